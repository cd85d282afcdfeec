"""The allocation-free saturation step (ads_saturation_step_noalloc) against
the context-based entry point, through the C ABI.

It serves callers that cannot allocate device memory (their own allocator
owns the budget, or they must avoid the synchronisation an allocation can
cause).  The caller provides inputs and outputs; the step's working memory
is a fixed array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_step_matches_context_step_twice():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from paper_2604_20731_gb300 import _lib
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import HybridSolver, make_params

    lib = _lib.load()
    n = 96
    sc = scn.make_scenario(2, n, seed=77, S0="random", grav=0.4)
    sc.phi_map = 0.1 + 0.3 * np.random.default_rng(5).uniform(size=(n + 1, n + 1))
    P = np.random.default_rng(6).normal(size=(n + 2, n + 2))
    dt = 2e-4
    s = HybridSolver(sc, width=None, ads_dtype="f64")
    s.set_pressure(P)
    dev = torch.device("cuda", 0)
    K = torch.from_numpy(np.ascontiguousarray(sc.K)).to(dev)
    phi = torch.from_numpy(np.ascontiguousarray(sc.phi_map)).to(dev)
    S0 = torch.from_numpy(np.ascontiguousarray(sc.S0)).to(dev)
    Pd = torch.from_numpy(P).to(dev)
    out1 = torch.empty_like(S0)
    out2 = torch.empty_like(S0)
    params = make_params(sc, "f64")
    stream = torch.cuda.Stream(device=dev)
    h = C.c_void_p(stream.cuda_stream)
    torch.cuda.synchronize()
    # two calls in a row: S1 = step(S0), S2 = step(S1)
    rc = lib.ads_saturation_step_noalloc(C.byref(params), K.data_ptr(), phi.data_ptr(),
                                         S0.data_ptr(), Pd.data_ptr(), dt, out1.data_ptr(), h)
    assert rc == 0
    rc = lib.ads_saturation_step_noalloc(C.byref(params), K.data_ptr(), phi.data_ptr(),
                                         out1.data_ptr(), Pd.data_ptr(), dt, out2.data_ptr(), h)
    assert rc == 0
    stream.synchronize()
    s.saturation_step(dt, 1)
    ref1 = s.get("S")
    s.saturation_step(dt, 1)
    ref2 = s.get("S")
    got1, got2 = out1.cpu().numpy(), out2.cpu().numpy()
    for got, ref in ((got1, ref1), (got2, ref2)):
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # the status word covers both steps: no wait gave up, int S stayed finite
    flags = C.c_int(-1)
    assert lib.ads_saturation_step_noalloc_status(h, C.byref(flags)) == 0
    assert flags.value == 0
    # sizes beyond the fixed scratch are refused; input == output is refused
    params.n = 513
    assert lib.ads_saturation_step_noalloc(C.byref(params), K.data_ptr(), None, S0.data_ptr(),
                                           Pd.data_ptr(), dt, out1.data_ptr(), h) == 1
    params.n = n
    assert lib.ads_saturation_step_noalloc(C.byref(params), K.data_ptr(), None, S0.data_ptr(),
                                           Pd.data_ptr(), dt, S0.data_ptr(), h) == 1
    s.close()


def test_noalloc_step_at_the_largest_mesh_against_the_oracle():
    """n = 512 (the largest mesh the fixed array takes) with eight sources
    and no porosity map: the step against the FP64 oracle's step and against
    the context-based step, then the status word."""
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from oracle.ads import AdsOracle
    from paper_2604_20731_gb300 import _lib
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import HybridSolver, make_params

    lib = _lib.load()
    n = 512
    sc = scn.make_scenario(2, n, seed=81, S0="random", grav=0.7)
    rng = np.random.default_rng(9)
    sc.sources = [scn.Source(center=tuple(rng.uniform(0.1, 0.9, size=2)), rate=float(rng.uniform(0.5, 2)),
                             sigma=float(rng.uniform(0.02, 0.06)), kind=int(i % 2)) for i in range(8)]
    P = rng.normal(size=(n + 2, n + 2)) / n  # O(1) gradients
    dt = 2e-5
    dev = torch.device("cuda", 0)
    K = torch.from_numpy(np.ascontiguousarray(sc.K)).to(dev)
    S0 = torch.from_numpy(np.ascontiguousarray(sc.S0)).to(dev)
    Pd = torch.from_numpy(P).to(dev)
    out = torch.empty_like(S0)
    params = make_params(sc, "f64")
    assert params.n_src == 8
    stream = torch.cuda.Stream(device=dev)
    h = C.c_void_p(stream.cuda_stream)
    torch.cuda.synchronize()
    rc = lib.ads_saturation_step_noalloc(C.byref(params), K.data_ptr(), None, S0.data_ptr(),
                                         Pd.data_ptr(), dt, out.data_ptr(), h)
    assert rc == 0
    flags = C.c_int(-1)
    assert lib.ads_saturation_step_noalloc_status(h, C.byref(flags)) == 0
    assert flags.value == 0
    got = out.cpu().numpy()
    ref = AdsOracle(sc).step(sc.S0, P, dt)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    s = HybridSolver(sc, width=None, ads_dtype="f64")
    try:
        s.set_pressure(P)
        s.saturation_step(dt, 1)
        ctx = s.get("S")
    finally:
        s.close()
    assert np.abs(got - ctx).max() <= 1e-12 * np.abs(ctx).max()
