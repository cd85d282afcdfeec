"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  * saturation (FP64 path): relative L-inf <= 1e-12; (FP32 path) <= 1e-5 --
    the bounds stated for the method's precision policy;
  * step size, mass balance, coefficients: FP64 round-off bounds;
  * robust loss / gradient with the FP32 network: the residual is a
    difference of neighbouring network values, so FP32 rounding of u
    (~1e-7 relative) is amplified by ~1/(h |grad u|); the bounds below
    (loss 1e-3 relative, gradient 2e-2 relative L2) follow from that
    amplification at the tested sizes, and are checked tighter in FP64.
"""
import numpy as np
import pytest

from oracle.ads import AdsOracle
from oracle.crvpinn import Adam, CrvOracle, MLP, embed_interior
from oracle.hybrid import HybridOracle, project_nodal
from paper_2604_20731_gb300 import scenario as scn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def solver(sc, **kw):
    from paper_2604_20731_gb300.solver import HybridSolver
    return HybridSolver(sc, **kw)


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _scenario(n, seed=3, grav=0.0, phi_map=False, grav_sign=1.0):
    sc = scn.make_scenario(2, n, seed=seed, S0="random", grav=grav)
    sc.grav_sign = grav_sign
    # exercise the clamp inside the mobilities
    rng = np.random.default_rng(seed + 1)
    sc.S0 = rng.uniform(-0.15, 1.15, size=(n + 2, n + 2))
    if phi_map:
        sc.phi_map = 0.1 + 0.3 * rng.uniform(size=(n + 1, n + 1))
    return sc


# ----------------------------------------------------------------------------
# saturation step: quadrature (a1) + Kronecker solve (a2) + mass balance (a3)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 7, 31, 33, 64, 257])
@pytest.mark.parametrize("grav,phi_map,gsign", [(0.0, False, 1.0), (0.9, True, 1.0), (0.9, False, -1.0)])
def test_saturation_step_fp64(n, grav, phi_map, gsign):
    sc = _scenario(n, seed=n, grav=grav, phi_map=phi_map, grav_sign=gsign)
    P = np.random.default_rng(n + 7).normal(size=(n + 2, n + 2))
    dt = 3e-4
    s = solver(sc, width=None, ads_dtype="f64")
    s.set_pressure(P)
    s.saturation_step(dt, 1)
    got = s.get("S")
    ref = AdsOracle(sc).step(sc.S0, P, dt)
    assert rel_inf(got, ref) <= 1e-12
    s.close()


@pytest.mark.parametrize("n", [3, 33, 128])
def test_saturation_step_fp32(n):
    sc = _scenario(n, seed=n + 100, grav=0.5)
    P = np.random.default_rng(1).normal(size=(n + 2, n + 2))
    dt = 3e-4
    s = solver(sc, width=None, ads_dtype="f32")
    s.set_pressure(P)
    s.saturation_step(dt, 1)
    assert rel_inf(s.get("S"), AdsOracle(sc).step(sc.S0, P, dt)) <= 1e-5
    s.close()


@pytest.mark.parametrize("n,dtype,tol", [(600, "f64", 1e-12), (2, "f64", 1e-12), (700, "f32", 1e-5)])
def test_saturation_step_four_wells(n, dtype, tol):
    """More than two sources (the general source path of the quadrature) on
    meshes whose lines the sweeps split into several chunks."""
    sc = _scenario(n, seed=n + 11, grav=0.4)
    sc.sources = [
        scn.Source(center=(0.2, 0.3), rate=1.3, kind=scn.SRC_INJECT),
        scn.Source(center=(0.7, 0.25), rate=0.6, sigma=0.05, kind=scn.SRC_INJECT),
        scn.Source(center=(0.8, 0.8), rate=1.1, kind=scn.SRC_PRODUCE),
        scn.Source(center=(0.3, 0.75), rate=0.8, sigma=0.04, kind=scn.SRC_PRODUCE),
    ]
    P = np.random.default_rng(n).normal(size=(n + 2, n + 2))
    dt = 2e-4
    s = solver(sc, width=None, ads_dtype=dtype)
    s.set_pressure(P)
    # FP32: one step (the random pressure makes a second step ill-conditioned:
    # |S| grows to ~1e4 and FP32 rounding of the first step is amplified)
    steps = 2 if dtype == "f64" else 1
    s.saturation_step(dt, steps)
    a = AdsOracle(sc)
    ref = sc.S0
    for _ in range(steps):
        ref = a.step(ref, P, dt)
    assert rel_inf(s.get("S"), ref) <= tol
    mass = s.get("MASS")
    if dtype == "f64":
        assert mass[0] == pytest.approx(a.mesh.integral(ref), rel=1e-12)
    else:
        # |int (S - S_ref)| <= max |S - S_ref| times the area of the unit
        # square (the basis integrals sum to 1): the saturation tolerance
        # bounds the mass error.  The random pressure drives S far from its
        # mean, so a bound relative to the mass itself would be rounding luck.
        assert abs(mass[0] - a.mesh.integral(ref)) <= tol * np.abs(ref).max()
    s.close()


def test_ten_steps_and_mass_balance_fp64():
    n = 48
    sc = _scenario(n, seed=9, grav=0.3)
    P = np.random.default_rng(2).normal(size=(n + 2, n + 2))
    dt = 2e-4
    s = solver(sc, width=None)
    s.set_pressure(P)
    s.saturation_step(dt, 10)
    a = AdsOracle(sc)
    S = sc.S0
    src = 0.0
    for _ in range(10):
        src += a.source_integral(S, dt)
        S = a.step(S, P, dt)
    assert rel_inf(s.get("S"), S) <= 1e-12
    mass = s.get("MASS")  # [int S, accumulated mass error, accumulated source]
    assert mass[0] == pytest.approx(a.mesh.integral(S), rel=1e-12)
    assert abs(mass[1]) <= 1e-13 * max(1.0, abs(mass[0]))
    assert mass[2] == pytest.approx(src, rel=1e-12, abs=1e-15)
    # odd and even step counts end in the right buffer
    s.saturation_step(dt, 3)
    for _ in range(3):
        S = a.step(S, P, dt)
    assert rel_inf(s.get("S"), S) <= 1e-12
    s.close()


def test_cfl_dt_matches_oracle():
    n = 40
    sc = _scenario(n, seed=4, grav=0.7, phi_map=True)
    P = 5.0 * np.random.default_rng(3).normal(size=(n + 2, n + 2))
    s = solver(sc, width=None)
    s.set_pressure(P)
    dt = s.cfl_dt(0.1, 0.05, 1.0)
    assert dt == pytest.approx(AdsOracle(sc).cfl_dt(P, 0.1, 0.05, 1.0), rel=1e-12)
    # source-limited branch
    s.set_pressure(np.zeros_like(P))
    sc.grav = 0.0
    s2 = solver(sc, width=None)
    assert s2.cfl_dt(0.1, 0.05, 1.0) == pytest.approx(AdsOracle(sc).cfl_dt(np.zeros_like(P), 0.1, 0.05, 1.0), rel=1e-12)
    s.close(); s2.close()


# ----------------------------------------------------------------------------
# CRVPINN: coefficients (a5), network (a6), residual (a7), Gram (a8),
# adjoint (a9), backward (a10), Adam (a11)
# ----------------------------------------------------------------------------

def _crv_case(n, dtype, width=64, grav=0.6, seed=21):
    sc = _scenario(n, seed=seed, grav=grav)
    theta = scn.make_theta0(2, width, 4, seed=seed) + 0.01 * np.random.default_rng(seed).normal(
        size=scn.mlp_num_params(2, width, 4))
    s = solver(sc, width=width, crv_dtype=dtype)
    s.set_theta(theta)
    s.update_coefficients()
    crv = CrvOracle(sc)
    alpha, f = crv.coefficients(sc.S0)
    return sc, s, crv, theta, alpha, f


@pytest.mark.parametrize("n", [3, 4, 17, 65])
def test_coefficients_fp64(n):
    sc, s, crv, theta, alpha, f = _crv_case(n, "f64")
    assert rel_inf(s.get("ALPHA").ravel(), alpha.ravel()) <= 1e-13
    assert rel_inf(s.get("F"), f) <= 1e-12
    s.close()


# N a power of two (8, 64, 128) takes the FFT sine-transform Gram solve; the
# other sizes the dense-transform + tridiagonal route
@pytest.mark.parametrize("n", [3, 5, 8, 33, 64, 96, 128])
def test_loss_and_gradient_fp64(n):
    sc, s, crv, theta, alpha, f = _crv_case(n, "f64")
    loss = s.loss_grad()
    ref_loss, ref_grad, parts = crv.loss_grad(MLP(2, 64, 4), theta, alpha, f)
    assert rel_inf(s.get("U"), parts["u"]) <= 1e-12
    assert rel_inf(s.get("RES"), parts["r"]) <= 1e-9
    assert rel_inf(s.get("Z"), parts["z"]) <= 1e-9
    assert rel_inf(s.get("GU"), parts["g"]) <= 1e-9
    assert loss == pytest.approx(ref_loss, rel=1e-9)
    assert rel_l2(s.get("GRAD"), ref_grad) <= 1e-8
    s.close()


@pytest.mark.parametrize("n,width", [(3, 64), (8, 64), (33, 64), (64, 64), (65, 128), (128, 128),
                                     (130, 64)])
def test_loss_and_gradient_fp32(n, width):
    sc, s, crv, theta, alpha, f = _crv_case(n, "f32", width=width)
    assert rel_inf(s.get("ALPHA").ravel(), alpha.ravel()) <= 1e-6
    loss = s.loss_grad()
    ref_loss, ref_grad, parts = crv.loss_grad(MLP(2, width, 4), theta, alpha, f)
    assert np.abs(s.get("U") - parts["u"]).max() <= 2e-5 * max(1.0, np.abs(parts["u"]).max())
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    assert rel_l2(s.get("GRAD"), ref_grad) <= 2e-2
    s.close()


def test_adam_trajectory_fp64():
    """Five Adam iterations in FP64 follow the oracle (bias-corrected Adam)."""
    n = 12
    sc, s, crv, theta, alpha, f = _crv_case(n, "f64", seed=5)
    lr = 1e-3
    s.pressure_update(5, lr)
    mlp = MLP(2, 64, 4)
    opt = Adam(theta.size)
    th = theta.copy()
    for _ in range(5):
        _, g, _ = crv.loss_grad(mlp, th, alpha, f)
        th = opt.step(th, g, lr)
    assert np.abs(s.get("THETA") - th).max() <= 1e-9
    s.close()


def test_projection_fp64():
    n = 20
    sc, s, crv, theta, alpha, f = _crv_case(n, "f64", seed=8)
    s.project_pressure()
    u, _ = MLP(2, 64, 4).forward(theta, crv.X)
    ref = project_nodal(AdsOracle(sc).mesh, embed_interior(u, 2, n))
    assert rel_inf(s.get("P"), ref) <= 1e-12
    s.close()


def test_hybrid_step_fp64_matches_oracle():
    n = 16
    sc, s, crv, theta, alpha, f = _crv_case(n, "f64", seed=13, grav=0.0)
    sc.S0 = np.random.default_rng(3).uniform(0, 0.5, size=(n + 2, n + 2))
    s.set_saturation(sc.S0)
    hp = s.hybrid_params(n_sub=3, dt=1.0, dt_policy=1, cfl=0.1, src_frac=0.05, adam_iters=4, lr=1e-3)
    st = s.hybrid_step(hp)
    h = HybridOracle(sc, width=64)
    opt = Adam(theta.size)
    S, P, th, dt, losses = h.hybrid_step(sc.S0, theta, opt, n_sub=3, adam_iters=4, lr=1e-3,
                                         cfl=0.1, dt_cap=1.0)
    assert st["dt_used"] == pytest.approx(dt, rel=1e-12)
    assert rel_inf(s.get("P"), P) <= 1e-11
    assert rel_inf(s.get("S"), S) <= 1e-11
    assert np.abs(s.get("THETA") - th).max() <= 1e-9
    assert st["loss_last"] == pytest.approx(losses[-1], rel=1e-8)
    s.close()


# ----------------------------------------------------------------------------
# full-size configuration (256^2, FP64 saturation + FP32 network 2-64x4-1),
# the launch configuration the benchmark times
# ----------------------------------------------------------------------------

def test_full_size_256_saturation_and_loss():
    n = 256
    sc = scn.make_scenario(2, n, seed=1000, S0="random")
    P = np.random.default_rng(0).normal(size=(n + 2, n + 2))
    s = solver(sc, width=64, crv_dtype="f32", ads_dtype="f64")
    s.set_pressure(P)
    s.saturation_step(1e-4, 1)
    ref = AdsOracle(sc).step(sc.S0, P, 1e-4)
    assert rel_inf(s.get("S"), ref) <= 1e-12
    theta = scn.make_theta0(2, 64, 4, seed=7)
    s.set_theta(theta)
    s.update_coefficients()
    loss = s.loss_grad()
    crv = CrvOracle(sc)
    alpha, f = crv.coefficients(ref)
    ref_loss, ref_grad, _ = crv.loss_grad(MLP(2, 64, 4), theta, alpha, f)
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    assert rel_l2(s.get("GRAD"), ref_grad) <= 2e-2
    s.close()


# ----------------------------------------------------------------------------
# edge cases and error statuses
# ----------------------------------------------------------------------------

def test_edge_cases_and_errors():
    from paper_2604_20731_gb300 import _lib
    sc = scn.make_scenario(2, 3, seed=1, S0="random")
    s = solver(sc, width=64, crv_dtype="f32")
    S0 = s.get("S")
    s.saturation_step(1e-3, 0)  # no-op
    assert np.array_equal(s.get("S"), S0)
    with pytest.raises(_lib.AdsError):
        s.saturation_step(1e-3, -1)
    with pytest.raises(_lib.AdsError):
        s.set_pressure(np.full((5, 5), np.nan))
    with pytest.raises(_lib.AdsError):
        s.pressure_update(1, -1.0)
    # no sources, zero pressure: step size is the cap
    sc2 = scn.make_scenario(2, 8, seed=1)
    sc2.sources = []
    s2 = solver(sc2, width=None)
    assert s2.cfl_dt(0.1, 0.05, 0.25) == 0.25
    with pytest.raises(_lib.AdsError):
        s2.update_coefficients()  # no network in this context
    s.close(); s2.close()


def test_pretrain_reduces_loss_and_approaches_direct_solution():
    """Measured, not a parity claim: the trained network against the unique
    zero-residual solution (relative L2 over interior nodes is reported)."""
    n = 32
    sc = scn.make_scenario(2, n, seed=1000)
    s = solver(sc, width=64, crv_dtype="f32")
    s.set_theta(scn.make_theta0(2, 64, 4, seed=7))
    s.update_coefficients()
    l0 = s.loss_grad()
    l1 = s.pretrain(1500, 1e-3)
    assert l1 < 0.05 * l0
    crv = CrvOracle(sc)
    alpha, f = crv.coefficients(sc.S0_or_zero())
    ustar = crv.direct_solution(alpha, f)
    s.project_pressure()
    err = rel_l2(s.get("U"), ustar)
    print(f"pressure rel L2 vs direct after 1500 Adam iterations: {err:.3e}")
    assert err < 0.2
    s.close()


# ----------------------------------------------------------------------------
# BF16 tensor-core network (tcgen05): operands rounded to BF16 (unit
# round-off 2^-9 ~ 2e-3), FP32 accumulation.  Each stored activation and
# weight carries ~2e-3 relative rounding, so the loss and gradient are
# compared at 1e-2 (loss) and 2e-2 (gradient, relative L2), and the gradient
# direction must agree to cosine >= 0.9995.
# ----------------------------------------------------------------------------

# 256: 509 point tiles over at most one CTA per SM, so CTAs run several tiles
# (the prefetching path of the backward)
@pytest.mark.parametrize("n", [3, 9, 16, 33, 64, 130, 256])
def test_loss_and_gradient_bf16_tensor_cores(n):
    sc, s, crv, theta, alpha, f = _crv_case(n, "bf16", width=64)
    loss = s.loss_grad()
    ref_loss, ref_grad, parts = crv.loss_grad(MLP(2, 64, 4), theta, alpha, f)
    assert np.abs(s.get("U") - parts["u"]).max() <= 2e-2 * max(1.0, np.abs(parts["u"]).max())
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    g = s.get("GRAD")
    assert rel_l2(g, ref_grad) <= 2e-2
    assert g @ ref_grad / (np.linalg.norm(g) * np.linalg.norm(ref_grad)) >= 0.9995
    s.close()


def _bf16_rn(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def _tc_effective_theta(theta, din, w):
    """The parameters the tensor-core forward evaluates: the hidden layers'
    weights as bf16(s W) / s and their biases as (bf16(s b) + bf16(s b -
    bf16(s b))) / s, with s = -2 log2 e in FP32 (the kernels fold s into the
    staged operands); the first and the output layer stay in FP32."""
    s32 = np.float32(-2.8853900817779268)
    th = np.asarray(theta, dtype=np.float64).copy()
    sizes = [din, w, w, w, w, 1]
    o = 0
    for l in range(5):
        fi, fo = sizes[l], sizes[l + 1]
        Wl = th[o:o + fo * fi]
        bl = th[o + fo * fi:o + fo * fi + fo]
        if 1 <= l <= 3:
            sw = np.float32(Wl.astype(np.float32) * s32)
            th[o:o + fo * fi] = _bf16_rn(sw).astype(np.float64) / float(s32)
            sb = np.float32(bl.astype(np.float32) * s32)
            hi = _bf16_rn(sb)
            lo = _bf16_rn(np.float32(sb - hi))
            th[o + fo * fi:o + fo * fi + fo] = (hi.astype(np.float64) + lo.astype(np.float64)) / float(s32)
        o += fo * fi + fo
    return th


@pytest.mark.parametrize("n,width", [(33, 64), (256, 64), (70, 128)])
def test_bf16_forward_on_its_effective_weights(n, width):
    """The tensor-core forward against the FP64 network on the weights it
    actually multiplies (BF16-rounded, see _tc_effective_theta).  What is left
    is the forward's own arithmetic: hidden activations carried as BF16
    hi + lo (about 2^-17 relative each), FP32 accumulation and the ex2/rcp
    tanh (about 2^-21).  A wrong bias, scale, column or layer shows up as an
    error of order 1e-2 or more."""
    sc, s, crv, theta, alpha, f = _crv_case(n, "bf16", width=width)
    s.loss_grad()
    u_ref, _ = MLP(2, width, 4).forward(_tc_effective_theta(theta, 2, width), crv.X)
    err = np.abs(s.get("U") - u_ref).max() / max(1.0, np.abs(u_ref).max())
    print(f"BF16 forward vs the FP64 network on its effective weights, n={n}, W={width}: {err:.2e}")
    assert err <= 2e-4
    s.close()


def test_bf16_training_converges_to_direct_solution():
    n = 64
    sc = scn.make_scenario(2, n, seed=1000)
    s = solver(sc, width=64, crv_dtype="bf16", ads_dtype="f32")
    s.set_theta(scn.make_theta0(2, 64, 4, seed=7))
    s.update_coefficients()
    l0 = s.loss_grad()
    l1 = s.pretrain(3000, 1e-3)
    assert l1 < 0.02 * l0
    crv = CrvOracle(sc)
    alpha, f = crv.coefficients(sc.S0_or_zero())
    ustar = crv.direct_solution(alpha, f)
    s.project_pressure()
    err = rel_l2(s.get("U"), ustar)
    print(f"BF16 network: pressure rel L2 vs direct after 3000 Adam iterations: {err:.3e}")
    assert err < 0.15
    s.close()


def test_bf16_hybrid_step_runs_and_conserves_mass():
    n = 48
    sc = scn.make_scenario(2, n, seed=1001)
    s = solver(sc, width=64, crv_dtype="bf16", ads_dtype="f32")
    s.set_theta(scn.make_theta0(2, 64, 4, seed=7))
    s.pretrain(200, 1e-3)
    hp = s.hybrid_params(n_sub=10, dt=1.0, dt_policy=1, adam_iters=20, lr=1e-3)
    for _ in range(3):
        st = s.hybrid_step(hp)
    assert np.isfinite(st["loss_last"]) and st["dt_used"] > 0
    assert abs(st["mass_err"]) <= 1e-5 * max(st["mass_total"], 1e-3)
    s.close()


# ----------------------------------------------------------------------------
# hand-written adjoint (the FP64 GPU gradient) against central finite
# differences of the oracle's FP64 loss along 16 random unit directions
# ----------------------------------------------------------------------------

def test_adjoint_vs_finite_differences_16_directions():
    n = 24
    sc, s, crv, theta, alpha, f = _crv_case(n, "f64", seed=11)
    s.loss_grad()
    g = s.get("GRAD")
    mlp = MLP(2, 64, 4)
    rng = np.random.default_rng(11)
    scale = np.linalg.norm(theta)
    for eps_rel in (1e-2, 1e-3):
        errs = []
        for _ in range(16):
            d = rng.normal(size=theta.size)
            d /= np.linalg.norm(d)
            eps = eps_rel * scale / np.sqrt(theta.size)
            lp = crv.loss_grad(mlp, theta + eps * d, alpha, f, with_grad=False)[0]
            lm = crv.loss_grad(mlp, theta - eps * d, alpha, f, with_grad=False)[0]
            fd = (lp - lm) / (2 * eps)
            errs.append(abs(g @ d - fd) / max(abs(fd), 1e-12 * np.linalg.norm(g)))
        print(f"FD check eps_rel={eps_rel}: max relative deviation {max(errs):.2e}")
        assert max(errs) < 1e-3
    s.close()


@pytest.mark.parametrize("n", [3, 17, 70])
def test_loss_and_gradient_bf16_width128(n):
    """Width-128 tensor-core network (the 2-128x4-1 network of the 1024^2
    mixed-precision configuration): dW of the hidden layers on the tensor
    cores, the small gradients as FP32 sums on the CUDA cores."""
    sc, s, crv, theta, alpha, f = _crv_case(n, "bf16", width=128)
    loss = s.loss_grad()
    ref_loss, ref_grad, parts = crv.loss_grad(MLP(2, 128, 4), theta, alpha, f)
    assert np.abs(s.get("U") - parts["u"]).max() <= 2e-2 * max(1.0, np.abs(parts["u"]).max())
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    g = s.get("GRAD")
    assert rel_l2(g, ref_grad) <= 2e-2
    assert g @ ref_grad / (np.linalg.norm(g) * np.linalg.norm(ref_grad)) >= 0.9995
    s.close()


@pytest.mark.parametrize("n,width", [(33, 64), (256, 64), (70, 128)])
def test_concurrency_launch_shape_same_results(n, width):
    """ads_set_concurrency > 1 launches the network kernels on fewer CTAs with
    more tiles each (256: 509 tiles on 16 backward CTAs).  The network values
    and the loss are the same bit for bit; the gradient partials are summed in
    another grouping, so the gradient agrees to FP32 rounding."""
    sc, s, crv, theta, alpha, f = _crv_case(n, "bf16", width=width)
    loss1 = s.loss_grad()
    u1, g1 = s.get("U"), s.get("GRAD")
    s.set_concurrency(8)
    loss8 = s.loss_grad()
    u8, g8 = s.get("U"), s.get("GRAD")
    assert np.array_equal(u1, u8)
    assert loss8 == loss1
    assert rel_l2(g8, g1) <= 1e-5
    ref_loss, ref_grad, _ = crv.loss_grad(MLP(2, width, 4), theta, alpha, f)
    assert g8 @ ref_grad / (np.linalg.norm(g8) * np.linalg.norm(ref_grad)) >= 0.9995
    with pytest.raises(Exception):
        s.set_concurrency(0)
    s.close()


@pytest.mark.parametrize("n", [8, 64, 128])
def test_gram_solve_cluster_and_three_pass_forms_agree(n):
    """A context alone at N <= 128 solves G z = RES in one thread-block
    cluster (rows, columns through distributed shared memory, rows); with
    ads_set_concurrency > 1 it takes the three-pass form.  Both are the same
    sine-transform solve in another order of rounding: z, the residual and the
    loss agree to FP32 rounding, and z agrees with the oracle's direct solve."""
    sc, s, crv, theta, alpha, f = _crv_case(n, "f32", width=64)
    loss1 = s.loss_grad()
    z1, r1 = s.get("Z"), s.get("RES")
    s.set_concurrency(4)
    loss4 = s.loss_grad()
    z4, r4 = s.get("Z"), s.get("RES")
    assert np.array_equal(r1, r4)
    assert rel_l2(z1, z4) <= 1e-5
    assert loss1 == pytest.approx(loss4, rel=1e-5)
    _, _, parts = crv.loss_grad(MLP(2, 64, 4), theta, alpha, f)
    assert rel_l2(z1, parts["z"]) <= 1e-4
    s.close()


@pytest.mark.parametrize("n,width,chunks", [(64, 64, 3), (256, 64, 4), (70, 128, 2)])
def test_activation_recomputation_same_results(n, width, chunks):
    """act_chunks > 1: the iteration's forward stores no activations; the
    backward runs chunk by chunk, each chunk's forward storing only that
    chunk's (the last chunk shorter when the tiles do not divide).  Network
    values and loss are the same bit for bit; the gradient partials are
    grouped by chunk, so the gradient agrees to FP32 rounding; and an Adam
    trajectory stays together."""
    sc, s1, crv, theta, alpha, f = _crv_case(n, "bf16", width=width)
    s2 = solver(sc, width=width, crv_dtype="bf16", act_chunks=chunks)
    s2.set_theta(theta)
    s2.update_coefficients()
    loss1, loss2 = s1.loss_grad(), s2.loss_grad()
    assert loss1 == loss2
    assert np.array_equal(s1.get("U"), s2.get("U"))
    assert rel_l2(s2.get("GRAD"), s1.get("GRAD")) <= 1e-5
    s1.pressure_update(20, 1e-3)
    s2.pressure_update(20, 1e-3)
    assert rel_l2(s2.get("THETA"), s1.get("THETA")) <= 1e-4
    s1.close()
    s2.close()


def test_config3_mesh_1024_mixed_precision():
    """1024^2 elements, FP32 saturation step vs the FP64 oracle (1e-5) and the
    BF16 width-128 network's loss and gradient vs the FP64 oracle at the
    1025^2 collocation grid (1,046,529 interior points)."""
    n = 1024
    sc = scn.make_scenario(2, n, seed=1000, S0="random")
    P = np.random.default_rng(0).normal(size=(n + 2, n + 2))
    s = solver(sc, width=128, crv_dtype="bf16", ads_dtype="f32")
    s.set_pressure(P)
    s.saturation_step(1e-5, 1)
    S1 = s.get("S")
    assert rel_inf(S1, AdsOracle(sc).step(sc.S0, P, 1e-5)) <= 1e-5
    theta = scn.make_theta0(2, 128, 4, seed=7)
    s.set_theta(theta)
    s.update_coefficients()
    loss = s.loss_grad()
    crv = CrvOracle(sc)
    alpha, f = crv.coefficients(S1)
    ref_loss, ref_grad, _ = crv.loss_grad(MLP(2, 128, 4), theta, alpha, f, gram="fd")
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    g = s.get("GRAD")
    assert g @ ref_grad / (np.linalg.norm(g) * np.linalg.norm(ref_grad)) >= 0.999
    s.close()


def test_adjoint_vs_finite_differences_1024_fp64():
    """The FP64 GPU gradient against central differences of the GPU's own FP64
    loss on 16 random unit directions at 1024^2 (a property at any size)."""
    n = 1024
    sc = scn.make_scenario(2, n, seed=1000, S0="random")
    theta = scn.make_theta0(2, 64, 4, seed=7) + 0.01 * np.random.default_rng(1).normal(
        size=scn.mlp_num_params(2, 64, 4))
    s = solver(sc, width=64, crv_dtype="f64", ads_dtype="f64")
    s.set_theta(theta)
    s.update_coefficients()
    s.loss_grad()
    g = s.get("GRAD")
    rng = np.random.default_rng(11)
    eps = 1e-3 * np.linalg.norm(theta) / np.sqrt(theta.size)
    worst = 0.0
    for _ in range(16):
        d = rng.normal(size=theta.size)
        d /= np.linalg.norm(d)
        s.set_theta(theta + eps * d)
        lp = s.loss_grad()
        s.set_theta(theta - eps * d)
        lm = s.loss_grad()
        fd = (lp - lm) / (2 * eps)
        worst = max(worst, abs(g @ d - fd) / max(abs(fd), 1e-6 * np.linalg.norm(g)))
    print(f"1024^2 FD check: max relative deviation {worst:.2e}")
    assert worst < 1e-4
    s.close()


@pytest.mark.parametrize("conc", [1, 4])
def test_gram_solve_at_512_against_the_direct_solve(conc):
    """The three-pass sine-transform solve at N = 512 in FP32: z must solve
    G z = RES for the GPU's own RES (the oracle's sparse LU of G, FP64) to
    FP32 rounding, the loss must be RES . z, and the residual, loss and
    gradient must agree with the oracle's within the FP32 network's error;
    alone and in the shared launch shape."""
    sc, s, crv, theta, alpha, f = _crv_case(512, "f32", width=64)
    s.set_concurrency(conc)
    loss = s.loss_grad()
    z, r = s.get("Z").astype(np.float64), s.get("RES").astype(np.float64)
    z_ref = crv.gram_solve_lu(r)
    assert rel_l2(z, z_ref) <= 1e-5
    assert loss == pytest.approx(float(r @ z), rel=1e-5)
    ref_loss, ref_grad, parts = crv.loss_grad(MLP(2, 64, 4), theta, alpha, f)
    assert rel_l2(r, parts["r"]) <= 1e-2
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    assert rel_l2(s.get("GRAD"), ref_grad) <= 2e-2
    s.close()
