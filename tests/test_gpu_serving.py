"""Serving (continuous batching) on the GPU: admission by device-memory
budget, overlap of resident scenarios, and identical results alone and in a
mix of other scenarios."""
import time

import numpy as np
import pytest

from paper_2604_20731_gb300 import scenario as scn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _hp(solver_cls, steps_adam=20):
    return solver_cls.hybrid_params(n_sub=10, dt=1.0, dt_policy=1, cfl=0.1, src_frac=0.05,
                                    adam_iters=steps_adam, lr=1e-3)


def test_alone_equals_in_mix():
    from paper_2604_20731_gb300.solver import HybridSolver, Server
    hp = _hp(HybridSolver)
    target = scn.make_scenario(2, 48, seed=1200, rate=1.3)
    theta = scn.make_theta0(2, 64, 4, seed=7)
    srv = Server(hbm_budget=4 << 30, max_active=8, n_streams=4)
    rid = srv.submit(target, n_steps=4, hp=hp, pretrain_iters=50, theta0=theta)
    S_alone, P_alone, info = srv.wait(rid)
    assert info["steps"] == 4
    # the same scenario among others of different sizes, arriving while they run
    ids = []
    for k, n in enumerate((32, 64, 96, 40)):
        sc = scn.make_scenario(2, n, seed=1300 + k, sigma=0.5 + 0.4 * k, rate=0.5 + 0.4 * k)
        ids.append(srv.submit(sc, n_steps=6, hp=hp, pretrain_iters=50, theta0=theta))
        if k == 1:
            time.sleep(0.02)
            rid2 = srv.submit(target, n_steps=4, hp=hp, pretrain_iters=50, theta0=theta)
    S_mix, P_mix, info2 = srv.wait(rid2)
    for i in ids:
        S, P, inf = srv.wait(i)
        assert inf["steps"] == 6 and np.isfinite(S).all()
    assert np.array_equal(S_mix, S_alone)
    assert np.array_equal(P_mix, P_alone)
    st = srv.stats()
    assert st["completed"] == 6 and st["p99_step_ms"] >= st["p50_step_ms"] > 0
    assert st["peak_active"] >= 2  # the mix really overlapped
    srv.close()


def test_admission_respects_budget_and_rejects_oversize():
    import ctypes as C
    from paper_2604_20731_gb300 import _lib
    from paper_2604_20731_gb300.solver import HybridSolver, Server, make_params
    hp = _hp(HybridSolver, steps_adam=5)
    lib = _lib.load()
    sc = scn.make_scenario(2, 64, seed=5)
    p = make_params(sc, "f32")
    crv = _lib.crvpinn_params(64, 4, _lib.ADS_BF16)
    est = lib.ads_hbm_estimate(C.byref(p), C.byref(crv))
    srv = Server(hbm_budget=int(2.5 * est), max_active=16, n_streams=4)
    ids = [srv.submit(scn.make_scenario(2, 64, seed=10 + i), n_steps=3, hp=hp, pretrain_iters=10)
           for i in range(6)]
    for i in ids:
        srv.wait(i)
    st = srv.stats()
    assert st["completed"] == 6
    assert st["peak_active"] <= 2
    assert st["peak_bytes"] <= 2.5 * est
    big = scn.make_scenario(2, 256, seed=1)
    with pytest.raises(_lib.AdsError):
        srv.submit(big, n_steps=1, hp=hp)
    srv.close()


def test_hybrid_step_batch_equals_per_context_steps():
    """hybrid_step_batch over a batch of three contexts of different sizes,
    each on its own stream, gives bit for bit what hybrid_step gives for each
    context alone (the same kernels in the same order on each context's
    stream), twice in a row, with the step statistics of each."""
    import torch
    from paper_2604_20731_gb300.solver import HybridSolver, hybrid_step_batch
    hp = _hp(HybridSolver, steps_adam=10)
    theta = scn.make_theta0(2, 64, 4, seed=7)
    scs = [scn.make_scenario(2, n, seed=1400 + n, sigma=0.8, rate=1.1) for n in (24, 40, 33)]
    dev = torch.device("cuda", 0)

    def make(sc):
        s = HybridSolver(sc, width=64, crv_dtype="bf16", ads_dtype="f32", stream=torch.cuda.Stream(device=dev))
        s.set_theta(theta)
        s.pretrain(20, 1e-3)
        return s

    batch = [make(sc) for sc in scs]
    alone = [make(sc) for sc in scs]
    try:
        for _ in range(2):
            st_b = hybrid_step_batch(batch, hp, stats=True)
            st_a = [s.hybrid_step(hp) for s in alone]
            for b, a, sb, sa in zip(batch, alone, st_b, st_a):
                for f in ("S", "P", "THETA"):
                    assert np.array_equal(b.get(f), a.get(f)), f
                assert sb["dt_used"] == sa["dt_used"] and sb["mass_total"] == sa["mass_total"]
                assert sb["loss_last"] == sa["loss_last"]
    finally:
        for s in batch + alone:
            s.close()


def test_grouped_batch_training_equals_per_context_steps():
    """Contexts of the grouped shape (2D, width-64 tensor-core network, FFT
    Gram solve in its three-pass form: the contexts are told they share the
    GPU) are trained by grouped launches, each training kernel once for the
    whole batch.  S, P, the parameters, the step statistics and the loss log
    are bit for bit those of each context's own hybrid step, over mixed sizes
    and two steps; the launch counts show the grouped path ran."""
    import torch
    from paper_2604_20731_gb300.solver import HybridSolver, hybrid_step_batch
    hp = _hp(HybridSolver, steps_adam=12)
    theta = scn.make_theta0(2, 64, 4, seed=7)
    sizes = (32, 128, 64, 256, 64)
    scs = [scn.make_scenario(2, n, seed=1500 + i, sigma=0.9, rate=0.7 + 0.2 * i) for i, n in enumerate(sizes)]
    dev = torch.device("cuda", 0)

    def make(sc):
        s = HybridSolver(sc, width=64, crv_dtype="bf16", ads_dtype="f32", stream=torch.cuda.Stream(device=dev))
        s.set_concurrency(len(sizes))
        s.set_theta(theta)
        s.pretrain(20, 1e-3)
        return s

    batch = [make(sc) for sc in scs]
    alone = [make(sc) for sc in scs]
    try:
        for step in range(2):
            l0 = [s.kernel_launches() for s in batch]
            a0 = [s.kernel_launches() for s in alone]
            st_b = hybrid_step_batch(batch, hp, stats=True)
            st_a = [s.hybrid_step(hp) for s in alone]
            dl = [s.kernel_launches() - v for s, v in zip(batch, l0)]
            da = [s.kernel_launches() - v for s, v in zip(alone, a0)]
            # an Adam iteration is 8 kernels per context alone; grouped, 8 for
            # the whole batch (counted on the first context)
            assert dl[0] == da[0] and all(d == e - 8 * hp.adam_iters for d, e in zip(dl[1:], da[1:])), (dl, da)
            for b, a, sb, sa in zip(batch, alone, st_b, st_a):
                for f in ("S", "P", "THETA", "LOSS_LOG"):
                    assert np.array_equal(b.get(f), a.get(f)), (step, f)
                assert sb["dt_used"] == sa["dt_used"] and sb["mass_total"] == sa["mass_total"]
                assert sb["loss_last"] == sa["loss_last"]
    finally:
        for s in batch + alone:
            s.close()


def test_grouped_batch_plans_follow_their_members():
    """A batch with a member outside the grouped shape is stepped context by
    context; a batch plan goes with a destroyed member, and is made again when
    a member's launch shape changes; the results stay those of the contexts'
    own steps throughout."""
    import torch
    from paper_2604_20731_gb300.solver import HybridSolver, hybrid_step_batch
    hp = _hp(HybridSolver, steps_adam=6)
    theta = scn.make_theta0(2, 64, 4, seed=7)
    dev = torch.device("cuda", 0)

    def make(n, seed, conc=4):
        s = HybridSolver(scn.make_scenario(2, n, seed=seed), width=64, crv_dtype="bf16", ads_dtype="f32",
                         stream=torch.cuda.Stream(device=dev))
        s.set_concurrency(conc)
        s.set_theta(theta)
        s.pretrain(10, 1e-3)
        return s

    def launches(ss):
        return [s.kernel_launches() for s in ss]

    def same(b, a):
        for f in ("S", "P", "THETA"):
            assert np.array_equal(b.get(f), a.get(f)), f

    A, B, C, D = make(64, 1), make(32, 2), make(128, 3), make(24, 4)  # D: N = 24, no FFT Gram solve
    A2, B2, C2, D2 = make(64, 1), make(32, 2), make(128, 3), make(24, 4)
    try:
        # a member outside the shape: every context steps on its own (8 kernels per iteration each)
        l0, m0 = launches([A, B, C, D]), launches([A2, B2, C2, D2])
        hybrid_step_batch([A, B, C, D], hp)
        for s in (A2, B2, C2, D2):
            s.hybrid_step(hp, stats=False)
        assert [x - y for x, y in zip(launches([A, B, C, D]), l0)] == \
               [x - y for x, y in zip(launches([A2, B2, C2, D2]), m0)]
        for b, a in zip((A, B, C, D), (A2, B2, C2, D2)):
            same(b, a)
        # grouped, then a member destroyed: the remaining pair gets a plan of its own
        l0 = launches([A, B, C])
        hybrid_step_batch([A, B, C], hp)
        for s in (A2, B2, C2):
            s.hybrid_step(hp, stats=False)
        assert launches([A, B, C])[1] - l0[1] < 8 * hp.adam_iters  # B's training ran grouped
        B.close()
        B2.close()
        l0 = launches([A, C])
        hybrid_step_batch([A, C], hp)
        for s in (A2, C2):
            s.hybrid_step(hp, stats=False)
        assert launches([A, C])[1] - l0[1] < 8 * hp.adam_iters
        # a member reshaped (another concurrency): the plan is made again
        for s in (C, C2):
            s.set_concurrency(2)
        hybrid_step_batch([A, C], hp)
        for s in (A2, C2):
            s.hybrid_step(hp, stats=False)
        for b, a in zip((A, C, D), (A2, C2, D2)):
            same(b, a)
    finally:
        for s in (A, B, C, D, A2, B2, C2, D2):
            s.close()


def test_grouped_batches_from_two_threads_with_plan_eviction():
    """Two host threads step batches of their own contexts at once, through
    24 distinct lists (more than the 16 kept plans, so plans are evicted
    while the other thread steps); every context ends bit-identical to a twin
    stepped alone the same number of times."""
    import itertools
    import threading
    import torch
    from paper_2604_20731_gb300.solver import HybridSolver, hybrid_step_batch
    hp = HybridSolver.hybrid_params(n_sub=1, dt=1.0, dt_policy=1, cfl=0.1, src_frac=0.05, adam_iters=2, lr=1e-3)
    theta = scn.make_theta0(2, 64, 4, seed=7)
    dev = torch.device("cuda", 0)

    def make(n, seed):
        s = HybridSolver(scn.make_scenario(2, n, seed=seed), width=64, crv_dtype="bf16", ads_dtype="f32",
                         stream=torch.cuda.Stream(device=dev))
        s.set_concurrency(4)
        s.set_theta(theta)
        return s

    sizes = (32, 64, 32, 64, 32, 64)
    ctx = [make(n, 1700 + i) for i, n in enumerate(sizes)]
    twin = [make(n, 1700 + i) for i, n in enumerate(sizes)]
    groups = [ctx[:3], ctx[3:]]
    lists = [[list(p) for p in itertools.permutations(g, 2)] + [list(p) for p in itertools.permutations(g, 3)]
             for g in groups]
    errors = []

    def work(k):
        try:
            for lst in lists[k]:
                hybrid_step_batch(lst, hp)
        except Exception as e:  # reported below
            errors.append(e)

    try:
        th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors, errors
        for s, t in zip(ctx, twin):
            steps = sum(lst.count(s) for ls in lists for lst in ls)
            assert steps == 10
            for _ in range(steps):
                t.hybrid_step(hp, stats=False)
            for f in ("S", "P", "THETA"):
                assert np.array_equal(s.get(f), t.get(f)), f
    finally:
        for s in ctx + twin:
            s.close()
