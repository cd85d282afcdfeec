"""Interfaces around the kernels, through the C ABI: the loss as a
torch.autograd.Function, and the host-side deadline of a wait.  Collected
after every other file, so that a run stopping at the first failure has
already run the rest.

Bounds: the autograd loss and gradient are the kernels' own, so they meet
the FP64 bounds of the direct loss/gradient parity test (loss 1e-9 relative,
gradient 1e-8 relative L2).
"""
import numpy as np
import pytest

from oracle.crvpinn import CrvOracle, MLP
from paper_2604_20731_gb300 import scenario as scn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _case(n=8, width=64, seed=21):
    from paper_2604_20731_gb300.solver import HybridSolver
    sc = scn.make_scenario(2, n, seed=seed, S0="random", grav=0.6)
    theta = scn.make_theta0(2, width, 4, seed=seed) + 0.01 * np.random.default_rng(seed).normal(
        size=scn.mlp_num_params(2, width, 4))
    s = HybridSolver(sc, width=width, crv_dtype="f64")
    s.set_theta(theta)
    s.update_coefficients()
    return sc, s, theta


def test_autograd_function_fp64():
    torch = pytest.importorskip("torch")
    from paper_2604_20731_gb300.torch_loss import crvpinn_loss
    sc, s, theta = _case()
    try:
        t = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        loss = crvpinn_loss(s, t)
        loss.backward()
        crv = CrvOracle(sc)
        alpha, f = crv.coefficients(sc.S0)
        ref_loss, ref_grad, _ = crv.loss_grad(MLP(2, 64, 4), theta, alpha, f)
        assert loss.item() == pytest.approx(ref_loss, rel=1e-9)
        g = t.grad.numpy()
        assert np.linalg.norm(g - ref_grad) <= 1e-8 * np.linalg.norm(ref_grad)
    finally:
        s.close()


def test_host_wait_deadline_reports_timeout_and_context_survives():
    """A wait whose deadline passes while queued work runs returns
    ADS_ERR_TIMEOUT; the context stays usable and a later wait succeeds."""
    from paper_2604_20731_gb300._lib import AdsError
    sc, s, theta = _case(n=64)
    try:
        s.pressure_update(2000, 1e-3, sync=False)  # enqueued, not waited for
        with pytest.raises(AdsError, match="timeout"):
            s.sync(1e-6)
        s.sync(600.0)
        assert np.isfinite(s.get("LOSS")).all()
    finally:
        s.close()


def test_device_wait_expiry_is_reported_and_the_context_carries_on():
    """A device-side mbarrier wait with no producer runs out: the probe kernel
    (the kernels' own bounded wait, with tensor memory held and a bulk copy in
    flight) records the timeout bit and returns ADS_ERR_TIMEOUT after its
    limit; with a producer the same wait completes.  The context's state and
    status are untouched: the loss is bit-identical afterwards and a hybrid
    step reads a clean status."""
    import ctypes as C
    import time
    from paper_2604_20731_gb300.solver import HybridSolver
    n = 33
    sc = scn.make_scenario(2, n, seed=5, S0="random")
    s = HybridSolver(sc, width=64, crv_dtype="bf16", ads_dtype="f32")
    try:
        s.set_theta(scn.make_theta0(2, 64, 4, seed=7))
        s.update_coefficients()
        l0 = s.loss_grad()
        bits = C.c_int(-1)
        t0 = time.perf_counter()
        assert s.lib.ads_probe_wait_expiry(s.ctx, 0.05, 0, C.byref(bits)) == 5  # ADS_ERR_TIMEOUT
        assert time.perf_counter() - t0 >= 0.05
        assert bits.value == 8
        assert s.lib.ads_probe_wait_expiry(s.ctx, 0.05, 1, C.byref(bits)) == 0
        assert bits.value == 0
        assert s.loss_grad() == l0
        st = s.hybrid_step(HybridSolver.hybrid_params(n_sub=2, adam_iters=5, lr=1e-3))
        assert np.isfinite(st["loss_last"])
    finally:
        s.close()


def test_profiles_time_every_kernel_and_advance_like_updates():
    """The per-kernel profiles replay a captured iteration (sub-step): the
    times are positive and finite, and the parameters advance exactly as
    through crvpinn_pressure_update (same kernels, same order)."""
    from paper_2604_20731_gb300.solver import HybridSolver
    n = 33
    sc = scn.make_scenario(2, n, seed=5, S0="random")
    theta = scn.make_theta0(2, 64, 4, seed=7)
    a = HybridSolver(sc, width=64, crv_dtype="bf16", ads_dtype="f32")
    b = HybridSolver(sc, width=64, crv_dtype="bf16", ads_dtype="f32")
    try:
        for s in (a, b):
            s.set_theta(theta)
            s.update_coefficients()
            s.pressure_update(1, 1e-3)  # sets the learning rate the profile uses
        ms = a.profile_train(3)
        b.pressure_update(3, 1e-3)
        assert len(ms) == 8 and all(np.isfinite(v) and v >= 0 for v in ms.values())
        assert ms["mlp_fwd"] > 0 and ms["mlp_bwd"] > 0
        assert np.array_equal(a.get("THETA"), b.get("THETA"))
        sat = a.profile_saturation(2)
        assert all(np.isfinite(v) and v > 0 for v in sat.values())
    finally:
        a.close()
        b.close()
