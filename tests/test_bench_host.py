"""Host-side pieces of bench.py that decide what a run reports: the clock
summary that rejects throttled runs, and the per-point work of the network."""
import pytest

import bench


def _line(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 850.20, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_max_and_reasons():
    lines = [_line(2070, 2070), _line(1980, 2070, cap="Active"), _line(2055, 2070),
             "garbage", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = bench.clock_summary(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_nothing_parsed():
    out = bench.clock_summary([_line(1500, 2070, hwt="Active", swt="Active")])
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert bench.clock_summary([]) is None
    assert bench.clock_summary(["index, clocks.sm"]) is None


def test_network_flops_per_point():
    # 2-64x4-1: forward 2(2W + 3W^2 + W), backward 2(6W^2 + W + 2W)
    fwd, bwd = bench.mlp_flops_per_point(2, 64)
    assert fwd == 24960
    assert bwd == 2 * (6 * 64 * 64 + 64 + 2 * 64)
    assert bench.mlp_flops_per_point(3, 128)[0] == 2 * (3 * 128 + 3 * 128 * 128 + 128)


def test_oracle_workers_are_single_threaded_and_time_a_step():
    """The CPU-baseline workers are spawned with one BLAS thread each and
    return (non-network seconds, seconds per Adam iteration, threads)."""
    from paper_2604_20731_gb300 import scenario as scn
    jobs = [(scn.make_scenario(2, n, seed=1000 + n), 2, 4, 2, 1e-3, 64) for n in (8, 12)]
    with bench._oracle_pool(2) as pool:
        res = pool.map(bench._oracle_step, jobs, chunksize=1)
    for t_sat, t_iter, threads in res:
        assert t_sat > 0 and t_iter > 0
        assert threads in (None, 1)


@pytest.mark.parametrize("groups,nstreams", [(2, 16), (3, 16), (4, 16), (2, 5), (1, 16), (8, 4)])
def test_batches_follow_the_streams(groups, nstreams):
    """Every scenario is in exactly one batch, and the scenarios sharing a
    stream share a batch, for any batch count against any stream count."""
    sizes = [128, 256, 512] * 21 + [128]
    on = bench.stream_assignment(sizes, nstreams, "rr")
    items = list(range(len(sizes)))
    batches = bench.batches_by_stream(items, on, groups)
    assert sorted(x for b in batches for x in b) == items
    assert all(b for b in batches) and len(batches) <= groups
    batch_of = {x: k for k, b in enumerate(batches) for x in b}
    for st in set(on):
        assert len({batch_of[i] for i in items if on[i] == st}) == 1
    assert bench.batches_by_stream(items, on, 0) == []
