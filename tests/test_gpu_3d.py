"""3D (unit cube) parity of the CUDA path with the FP64 oracle: the
Kronecker mass solve gains a z factor, the collocation residual is the
7-point stencil (vertical differences weighted by kz_ratio), and G^-1 is
applied by sine transforms along x and y plus shifted tridiagonal sweeps
along z.  Tolerances as in the 2D tests."""
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


def _sc3(n, seed=3, grav=0.7, phi_map=True, kz=0.3):
    sc = scn.make_scenario(3, n, seed=seed, S0="random", grav=grav, kz_ratio=kz)
    rng = np.random.default_rng(seed + 5)
    sc.S0 = rng.uniform(-0.15, 1.15, size=(n + 2,) * 3)
    sc.sources[0].sigma = sc.sources[1].sigma = 0.15  # resolved on the small test meshes
    if phi_map:
        sc.phi_map = 0.1 + 0.3 * rng.uniform(size=(n + 1,) * 3)
    return sc


@pytest.mark.parametrize("n", [2, 3, 5, 12])
def test_saturation_step_3d_fp64(n):
    sc = _sc3(n, seed=n)
    P = np.random.default_rng(n).normal(size=(n + 2,) * 3)
    s = solver(sc, width=None, ads_dtype="f64")
    s.set_pressure(P)
    s.saturation_step(4e-4, 1)
    assert rel_inf(s.get("S"), AdsOracle(sc).step(sc.S0, P, 4e-4)) <= 1e-12
    s.close()


def test_saturation_steps_3d_fp32_and_mass():
    n = 16
    sc = _sc3(n, seed=31)
    P = np.random.default_rng(2).normal(size=(n + 2,) * 3)
    s = solver(sc, width=None, ads_dtype="f32")
    s.set_pressure(P)
    s.saturation_step(3e-4, 3)
    a = AdsOracle(sc)
    S = sc.S0
    src = 0.0
    for _ in range(3):
        src += a.source_integral(S, 3e-4)
        S = a.step(S, P, 3e-4)
    assert rel_inf(s.get("S"), S) <= 1e-5
    m = s.get("MASS")
    assert m[0] == pytest.approx(a.mesh.integral(S), rel=1e-5)
    assert abs(m[1]) <= 1e-5 * max(1.0, abs(m[0]))
    s.close()


def test_cfl_3d():
    n = 7
    sc = _sc3(n, seed=9)
    P = 3 * np.random.default_rng(4).normal(size=(n + 2,) * 3)
    s = solver(sc, width=None)
    s.set_pressure(P)
    assert s.cfl_dt(0.1, 0.05, 1.0) == pytest.approx(AdsOracle(sc).cfl_dt(P, 0.1, 0.05, 1.0), rel=1e-12)
    s.close()


def _crv3(n, dtype, width=64, seed=21):
    sc = _sc3(n, seed=seed, phi_map=False)
    theta = scn.make_theta0(3, width, 4, seed=seed) + 0.01 * np.random.default_rng(seed).normal(
        size=scn.mlp_num_params(3, width, 4))
    s = solver(sc, width=width, crv_dtype=dtype)
    s.set_theta(theta)
    s.update_coefficients()
    crv = CrvOracle(sc)
    alpha, f = crv.coefficients(sc.S0)
    return sc, s, crv, theta, alpha, f


# 8 and 16 are powers of two: the Gram solve takes the FFT sine transforms
# (the others the dense transforms)
@pytest.mark.parametrize("n", [3, 6, 8, 9, 16])
def test_coefficients_loss_gradient_3d_fp64(n):
    sc, s, crv, theta, alpha, f = _crv3(n, "f64")
    assert rel_inf(s.get("ALPHA").ravel(), alpha.ravel()) <= 1e-13
    assert rel_inf(s.get("F"), f) <= 1e-12
    loss = s.loss_grad()
    ref_loss, ref_grad, parts = crv.loss_grad(MLP(3, 64, 4), theta, alpha, f, gram="fd")
    assert rel_inf(s.get("U"), parts["u"]) <= 1e-12
    assert rel_inf(s.get("RES"), parts["r"]) <= 1e-9
    assert rel_inf(s.get("Z"), parts["z"]) <= 1e-9
    assert loss == pytest.approx(ref_loss, rel=1e-9)
    assert rel_l2(s.get("GRAD"), ref_grad) <= 1e-8
    s.close()


@pytest.mark.parametrize("n", [17, 32])  # 32: the FFT route
@pytest.mark.parametrize("dtype,width,tol_loss,tol_grad", [("f32", 64, 1e-3, 2e-2), ("f32", 128, 1e-3, 2e-2),
                                                            ("bf16", 64, 1e-2, 2e-2)])
def test_loss_gradient_3d_reduced_precision(dtype, width, tol_loss, tol_grad, n):
    sc, s, crv, theta, alpha, f = _crv3(n, dtype, width=width)
    loss = s.loss_grad()
    ref_loss, ref_grad, _ = crv.loss_grad(MLP(3, width, 4), theta, alpha, f, gram="fd")
    assert loss == pytest.approx(ref_loss, rel=tol_loss)
    assert rel_l2(s.get("GRAD"), ref_grad) <= tol_grad
    s.close()


def test_projection_3d_fp64():
    n = 7
    sc, s, crv, theta, alpha, f = _crv3(n, "f64", seed=8)
    s.project_pressure()
    u, _ = MLP(3, 64, 4).forward(theta, crv.X)
    ref = project_nodal(AdsOracle(sc).mesh, embed_interior(u, 3, n))
    assert rel_inf(s.get("P"), ref) <= 1e-12
    s.close()


def test_hybrid_step_3d_fp64_matches_oracle():
    n = 6
    sc, s, crv, theta, alpha, f = _crv3(n, "f64", seed=13)
    sc.S0 = np.random.default_rng(3).uniform(0, 0.5, size=(n + 2,) * 3)
    s.set_saturation(sc.S0)
    hp = s.hybrid_params(n_sub=3, dt=1.0, dt_policy=1, adam_iters=3, lr=1e-3)
    st = s.hybrid_step(hp)
    h = HybridOracle(sc, width=64)
    h.crv.gram_solve_lu = h.crv.gram_solve_fd
    S, P, th, dt, losses = h.hybrid_step(sc.S0, theta, Adam(theta.size), n_sub=3, adam_iters=3,
                                         lr=1e-3, cfl=0.1, dt_cap=1.0)
    assert st["dt_used"] == pytest.approx(dt, rel=1e-12)
    assert rel_inf(s.get("P"), P) <= 1e-11
    assert rel_inf(s.get("S"), S) <= 1e-11
    assert np.abs(s.get("THETA") - th).max() <= 1e-9
    s.close()


def test_config5_mesh_saturation_step_fp32():
    """128^3 elements (2.2 M B-spline coefficients), FP32, layered
    anisotropic permeability (kz = 0.1): one explicit step against the FP64
    oracle on the same inputs."""
    n = 128
    sc = scn.make_scenario(3, n, seed=1000, S0="random", kz_ratio=0.1)
    P = np.random.default_rng(1).normal(size=(n + 2,) * 3)
    s = solver(sc, width=None, ads_dtype="f32")
    s.set_pressure(P)
    s.saturation_step(1e-5, 1)
    assert rel_inf(s.get("S"), AdsOracle(sc).step(sc.S0, P, 1e-5)) <= 1e-5
    s.close()
