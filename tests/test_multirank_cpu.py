"""The multi-GPU path of bench.py is replicas only: each rank runs its own
scenarios with no data-path collective, and timing uses a barrier plus the
maximum over ranks.  These world-size-2 gloo tests run that host logic on
CPU processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    # each rank reports its own elapsed time; the job time is the maximum
    t = bench.max_over_ranks(1.5 + rank, w, torch.device("cpu"))
    # replicas: each rank draws its own scenario mix (no shared data)
    mix = bench.serving_mix(6, seed=3 + rank)
    q.put((rank, t, [sc.seed for sc in mix], [sc.n for sc in mix]))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replicas_barrier_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert out[0][1] == out[1][1] == pytest.approx(2.5)
    # the two replicas work on independent scenario draws
    assert set(out[0][2]).isdisjoint(out[1][2])
