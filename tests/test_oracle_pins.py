"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms, invariants, brute force on tiny inputs written independently here, or
an independent library route.  They are chosen so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle.ads import AdsOracle, Mesh, gaussian_sources
from oracle.bspline import Axis1D, basis_derivatives, basis_values, gauss_rule, open_uniform_knots
from oracle.crvpinn import Adam, CrvOracle, MLP, embed_interior
from oracle.hybrid import HybridOracle, plain_step, project_nodal
from oracle.pressure import galerkin_pressure
from paper_2604_20731_gb300 import scenario as scn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# independent scalar helpers (written here, not imported from the oracle)
# ----------------------------------------------------------------------------

def bspline_scalar(knots, i, p, x):
    """Recursive Cox-de Boor for one function at one point (right end closed)."""
    if p == 0:
        lo, hi = knots[i], knots[i + 1]
        if lo <= x < hi:
            return 1.0
        if x == knots[-1] and hi == knots[-1] and lo < hi:
            return 1.0
        return 0.0
    out = 0.0
    d1 = knots[i + p] - knots[i]
    d2 = knots[i + p + 1] - knots[i + 1]
    if d1 > 0:
        out += (x - knots[i]) / d1 * bspline_scalar(knots, i, p - 1, x)
    if d2 > 0:
        out += (knots[i + p + 1] - x) / d2 * bspline_scalar(knots, i + 1, p - 1, x)
    return out


def bspline_scalar_deriv(knots, i, p, x, eps=1e-7):
    return (bspline_scalar(knots, i, p, x + eps) - bspline_scalar(knots, i, p, x - eps)) / (2 * eps)


# ----------------------------------------------------------------------------
# Sec. 8.1 parameters
# ----------------------------------------------------------------------------

def test_parameter_ratios():
    with open(os.path.join(GOLDEN, "sec81_parameters.json")) as f:
        t = json.load(f)
    assert scn.MU_W / scn.MU_G == pytest.approx(t["mu_w_Pa_s"] / t["mu_g_Pa_s"], rel=1e-14)
    assert scn.RHO_G / scn.RHO_W == pytest.approx(t["rho_g_kg_m3"] / t["rho_w_kg_m3"], rel=1e-14)
    # the source width ~ half the well radius relative to the domain
    assert scn.SOURCE_SIGMA == pytest.approx(0.5 * t["well_radius_m"] / t["domain_m"], rel=1e-12)


# ----------------------------------------------------------------------------
# B-splines and quadrature (Sec. 4)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 7, 16])
def test_partition_of_unity_and_derivative_sum(n):
    knots = open_uniform_knots(n, 2)
    x = np.random.default_rng(n).uniform(0, 1, 200)
    x = np.concatenate([x, [0.0, 1.0, 0.5]])
    B = basis_values(knots, 2, x)
    D = basis_derivatives(knots, 2, x)
    assert B.shape[1] == n + 2
    assert np.all(B >= -1e-15)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-11)


def test_basis_matches_scalar_recursion_and_fd_derivative():
    n = 5
    knots = open_uniform_knots(n, 2)
    x = np.array([0.0, 0.03, 0.21, 0.41, 0.63, 0.77, 0.95, 1.0])  # off the knots
    B = basis_values(knots, 2, x)
    D = basis_derivatives(knots, 2, x[1:-1])
    for i in range(n + 2):
        for k, xv in enumerate(x):
            assert B[k, i] == pytest.approx(bspline_scalar(knots, i, 2, xv), abs=1e-15)
        for k, xv in enumerate(x[1:-1]):
            assert D[k, i] == pytest.approx(bspline_scalar_deriv(knots, i, 2, xv), abs=1e-6)


@pytest.mark.parametrize("n", [1, 4, 9])
def test_basis_integrals_closed_form(n):
    """int B_i = (t_{i+p+1} - t_i)/(p+1)."""
    ax = Axis1D(n, 2)
    ints = ax.B.T @ ax.w
    t = ax.knots
    expect = np.array([(t[i + 3] - t[i]) / 3.0 for i in range(n + 2)])
    np.testing.assert_allclose(ints, expect, rtol=1e-14, atol=1e-16)


def test_gauss_rule_exact_to_degree_5():
    x, w = gauss_rule(3)
    for k in range(6):
        assert np.sum(w * x ** k) == pytest.approx(1.0 / (k + 1), rel=1e-14)
    assert abs(np.sum(w * x ** 6) - 1.0 / 7) > 1e-6  # and not beyond


def test_mass_matrix_closed_form():
    with open(os.path.join(GOLDEN, "bspline_quadratic_mass_row.json")) as f:
        row = np.array(json.load(f)["row_times_120_over_h"], dtype=float)
    n = 12
    ax = Axis1D(n, 2)
    M = ax.M
    h = 1.0 / n
    np.testing.assert_allclose(M, M.T, atol=1e-17)
    for i in range(3, n - 1):
        np.testing.assert_allclose(M[i, i - 2:i + 3] * 120 / h, row, rtol=1e-13)
        assert np.all(M[i, :i - 2] == 0) and np.all(M[i, i + 3:] == 0)
    np.testing.assert_allclose(M.sum(1), ax.B.T @ ax.w, rtol=1e-14)


def test_hat_interpolation_reproduces_linear():
    ax = Axis1D(6, 2)
    nodal = 0.3 + 1.7 * ax.nodes
    np.testing.assert_allclose(ax.H @ nodal, 0.3 + 1.7 * ax.x, atol=1e-14)


def test_knot_values_closed_form():
    """Value of a quadratic spline at knot k: (c_k + c_{k+1})/2 inside, end
    coefficients at the ends."""
    n = 9
    c = np.random.default_rng(3).normal(size=n + 2)
    ax = Axis1D(n, 2)
    vals = ax.values_at(ax.nodes) @ c
    expect = np.concatenate([[c[0]], 0.5 * (c[1:n] + c[2:n + 1]), [c[n + 1]]])
    np.testing.assert_allclose(vals, expect, atol=1e-14)


# ----------------------------------------------------------------------------
# Kronecker mass solve (Eq. 14) and the explicit step (Eqs. 6, 10a, 10b)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(2, 1), (2, 3), (2, 8), (3, 2), (3, 4)])
def test_kronecker_solve_equals_dense(dim, n):
    m = Mesh(dim, n)
    R = np.random.default_rng(dim * 10 + n).normal(size=(n + 2,) * dim)
    Xk = m.mass_solve_kron(R)
    Xd = m.mass_solve_dense(R)
    np.testing.assert_allclose(Xk, Xd, rtol=0, atol=1e-12 * np.abs(Xd).max())
    # residual of the assembled Kronecker product
    res = m.mass_dense() @ Xk.ravel() - R.ravel()
    assert np.abs(res).max() <= 1e-14 * np.abs(R).max() * 10


def _brute_rhs(sc, S, P, dt):
    """Element loop, pointwise scalar basis evaluation: the definition of the
    right-hand side of Eq. 10b with the gravity reading of the scenario, for
    B-splines of the scenario's degree with p + 1 Gauss points per axis."""
    n = sc.n
    deg = getattr(sc, "p", 2)
    knots = open_uniform_knots(n, deg)
    hat = open_uniform_knots(n, 1)
    xg, wg = np.polynomial.legendre.leggauss(deg + 1)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    h = 1.0 / n
    R = np.zeros((n + deg, n + deg))
    for ey in range(n):
        for ex in range(n):
            for qy in range(deg + 1):
                for qx in range(deg + 1):
                    x = (ex + xg[qx]) * h
                    y = (ey + xg[qy]) * h
                    w = wg[qx] * wg[qy] * h * h
                    bx = {i: bspline_scalar(knots, i, deg, x) for i in range(ex, ex + deg + 1)}
                    by = {j: bspline_scalar(knots, j, deg, y) for j in range(ey, ey + deg + 1)}
                    dbx = {i: bspline_scalar_deriv(knots, i, deg, x) for i in range(ex, ex + deg + 1)}
                    dby = {j: bspline_scalar_deriv(knots, j, deg, y) for j in range(ey, ey + deg + 1)}
                    s = sum(S[j, i] * by[j] * bx[i] for i in bx for j in by)
                    px = sum(P[j, i] * by[j] * dbx[i] for i in bx for j in by)
                    py = sum(P[j, i] * dby[j] * bx[i] for i in bx for j in by)
                    kk = sum(sc.K[j, i] * bspline_scalar(hat, j, 1, y) * bspline_scalar(hat, i, 1, x)
                             for i in (ex, ex + 1) for j in (ey, ey + 1))
                    st = min(max(s, 0.0), 1.0)
                    lg, lw = st / sc.mu_g, (1 - st) / sc.mu_w
                    qi = qp = 0.0
                    for src in sc.sources:
                        G = math.exp(-((x - src.center[0]) ** 2 + (y - src.center[1]) ** 2)
                                     / (2 * src.sigma ** 2)) / (2 * math.pi * src.sigma ** 2)
                        if src.kind == 0:
                            qi += src.rate * G
                        else:
                            qp += src.rate * G
                    qg = qi - lg / (lg + lw) * qp
                    phi = sc.phi
                    fx = kk * px
                    fy = kk * (py + sc.grav_sign * sc.rho_g * sc.grav)
                    for i in bx:
                        for j in by:
                            v = bx[i] * by[j]
                            vx = dbx[i] * by[j]
                            vy = bx[i] * dby[j]
                            R[j, i] += w * (s * v + dt / phi * (qg * v - lg * (fx * vx + fy * vy)))
    return R


@pytest.mark.parametrize("grav_sign", [1.0, -1.0])
def test_rhs_matches_element_loop(grav_sign):
    sc = scn.make_scenario(2, 4, seed=5, S0="random", grav=0.7)
    sc.grav_sign = grav_sign
    sc.sources[0].center = (0.3, 0.4)
    sc.sources[1].center = (0.6, 0.7)
    sc.sources[0].sigma = sc.sources[1].sigma = 0.2
    rng = np.random.default_rng(11)
    S = rng.uniform(-0.1, 1.1, size=(6, 6))  # exercises the clamp
    P = rng.normal(size=(6, 6))
    dt = 0.013
    R = AdsOracle(sc).rhs(S, P, dt)
    Rb = _brute_rhs(sc, S, P, dt)
    np.testing.assert_allclose(R, Rb, rtol=0, atol=2e-7 * np.abs(Rb).max())


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_constant_saturation_preserved(dim, n):
    sc = scn.make_scenario(dim, n, seed=2)
    sc.sources = []
    sc.grav = 0.0
    c = 0.37
    S = np.full((n + 2,) * dim, c)
    P = np.random.default_rng(0).normal(size=(n + 2,) * dim) * 0  # p = 0
    Sn = AdsOracle(sc).step(S, P, 0.01)
    np.testing.assert_allclose(Sn, c, atol=1e-13)


@pytest.mark.parametrize("dim,n,grav", [(2, 7, 0.0), (2, 6, 1.0), (3, 3, 1.0)])
def test_mass_balance(dim, n, grav):
    sc = scn.make_scenario(dim, n, seed=3, S0="random", grav=grav)
    sc.phi_map = 0.1 + 0.3 * np.random.default_rng(9).uniform(size=(n + 1,) * dim)
    P = np.random.default_rng(4).normal(size=(n + 2,) * dim)
    a = AdsOracle(sc)
    Sn = a.step(sc.S0, P, 0.002)
    total = a.mesh.integral(Sn)
    err = a.mass_error(sc.S0, Sn, 0.002)
    assert abs(err) <= 1e-13 * max(1.0, abs(total))
    # and int S_{n+1} equals the sum of the right-hand side
    assert total == pytest.approx(a.rhs(sc.S0, P, 0.002).sum(), rel=1e-13)


def test_flux_direction_outward_from_pressure_peak():
    """Gas flows down the pressure gradient: with a pressure maximum at the
    centre and uniform S, S decreases at the centre and increases around it."""
    n = 16
    sc = scn.make_scenario(2, n, seed=1)
    sc.K = np.ones_like(sc.K)
    sc.sources = []
    m = Mesh(2, n)
    xs = (np.arange(n + 2) - 0.5) / n  # rough Greville-like abscissae
    X, Y = np.meshgrid(xs, xs)
    P = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / 0.02)
    S = np.full((n + 2, n + 2), 0.5)
    Sn = AdsOracle(sc).step(S, P, 1e-4)
    assert Sn[n // 2 + 1, n // 2 + 1] < 0.5
    assert Sn[n // 2 + 1, n // 2 + 5] > 0.5


def test_gravity_moves_gas_down_without_pressure_support():
    """With p = 0 the gas flux is lambda_g K rho_g g downwards (Eq. 2 with g
    pointing down): the top row loses gas, the bottom row gains it; with the
    printed sign of Eq. 9 it is the other way round."""
    n = 8
    for sign, top_change in ((1.0, -1), (-1.0, 1)):
        sc = scn.make_scenario(2, n, seed=1, grav=1.0)
        sc.sources = []
        sc.grav_sign = sign
        S = np.full((n + 2, n + 2), 0.5)
        Sn = AdsOracle(sc).step(S, np.zeros_like(S), 1e-3)
        assert np.sign(Sn[-1, n // 2] - 0.5) == top_change
        assert np.sign(Sn[0, n // 2] - 0.5) == -top_change


def test_cfl_dt_rule():
    sc = scn.make_scenario(2, 8, seed=1)
    a = AdsOracle(sc)
    P = np.zeros((10, 10))
    # no flow: the source limit decides
    dt = a.cfl_dt(P)
    qi, _ = gaussian_sources(sc, a.coords)
    assert dt == pytest.approx(0.05 * sc.phi / qi.max(), rel=1e-14)
    # strong linear pressure: the velocity limit decides
    xs = np.linspace(0, 1, 10)
    sc.sources = []
    sc.K = np.full_like(sc.K, 2.0)
    Pl = np.tile(xs * 100.0, (10, 1))  # p = 100 x at the Greville abscissae -> dp/dx = 100
    knots = open_uniform_knots(8, 2)
    grev = np.array([(knots[i + 1] + knots[i + 2]) / 2 for i in range(10)])
    Pl = np.tile(100.0 * grev, (10, 1))
    dt = AdsOracle(sc).cfl_dt(Pl)
    vmax = 2.0 * 100.0 / (sc.mu_g * sc.phi)
    assert dt == pytest.approx(0.1 * (1 / 8) / vmax, rel=1e-12)


# ----------------------------------------------------------------------------
# Galerkin pressure (Sec. 4 / Sec. 7)
# ----------------------------------------------------------------------------

def test_galerkin_pressure_manufactured_h3():
    """Homogeneous K, S = 0, no gravity, p* = sin(pi x) sin(pi y) with its
    source q = 2 pi^2 lambda_w p*: L2 error falls like h^3."""
    errs = []
    for n in (8, 16, 32):
        sc = scn.make_scenario(2, n, seed=1)
        sc.K = np.ones_like(sc.K)
        lam = 1.0 / sc.mu_w

        # replace the sources by the manufactured one through a custom object
        class Src:
            pass
        m = Mesh(2, n)
        coords = m.gauss_coords()
        import oracle.pressure as pr
        orig = pr.gaussian_sources
        pr.gaussian_sources = lambda s, c: (2 * np.pi ** 2 * lam * np.sin(np.pi * c[0]) * np.sin(np.pi * c[1]),
                                            np.zeros_like(c[0]))
        try:
            P = galerkin_pressure(sc, np.zeros((n + 2, n + 2)))
        finally:
            pr.gaussian_sources = orig
        ph = m.at_gauss(P)
        ex = np.sin(np.pi * coords[0]) * np.sin(np.pi * coords[1])
        errs.append(math.sqrt(np.sum(m.gauss_weights() * (ph - ex) ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 2.7, (errs, rates)


def test_galerkin_pressure_manufactured_3d_h3():
    """3D with anisotropy K_z = kz K: p* = sin(pi x) sin(pi y) sin(2 pi z) with
    its source q = (2 + 4 kz) pi^2 lambda_w p* (a kz on another axis would
    give another source); the L2 error falls like h^3."""
    import oracle.pressure as pr
    kz = 0.3
    errs = []
    for n in (4, 8, 16):
        sc = scn.make_scenario(3, n, seed=1, kz_ratio=kz)
        sc.K = np.ones_like(sc.K)
        lam = 1.0 / sc.mu_w
        m = Mesh(3, n)
        coords = m.gauss_coords()
        orig = pr.gaussian_sources
        pr.gaussian_sources = lambda s, c: ((2 + 4 * kz) * np.pi ** 2 * lam * np.sin(np.pi * c[0])
                                            * np.sin(np.pi * c[1]) * np.sin(2 * np.pi * c[2]),
                                            np.zeros_like(c[0]))
        try:
            P = galerkin_pressure(sc, np.zeros((n + 2,) * 3))
        finally:
            pr.gaussian_sources = orig
        ph = m.at_gauss(P)
        ex = np.sin(np.pi * coords[0]) * np.sin(np.pi * coords[1]) * np.sin(2 * np.pi * coords[2])
        errs.append(math.sqrt(np.sum(m.gauss_weights() * (ph - ex) ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 2.6, (errs, rates)


def test_galerkin_pressure_matches_element_loop():
    """The Galerkin system assembled element by element with scalar basis
    evaluation: (lambda K grad B_kl, grad B_ij) p = (q_w + q_g, B_ij)
    - (g K (rho_w lambda_w + rho_g lambda_g), dB_ij/dy) over interior i, j,
    with a saturation that puts both mobilities to work (and the clamp) and
    gravity on -- the cases the S = 0 pins above cannot tell apart."""
    n = 4
    sc = scn.make_scenario(2, n, seed=9, S0="random", grav=0.8)
    sc.sources[0].center = (0.3, 0.4)
    sc.sources[1].center = (0.6, 0.7)
    sc.sources[0].sigma = sc.sources[1].sigma = 0.2
    S = np.random.default_rng(13).uniform(-0.2, 1.2, size=(n + 2, n + 2))
    knots = open_uniform_knots(n, 2)
    hat = open_uniform_knots(n, 1)
    xg, wg = np.polynomial.legendre.leggauss(3)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    h = 1.0 / n
    nb = n + 2
    A = np.zeros((nb * nb, nb * nb))
    F = np.zeros(nb * nb)
    for ey in range(n):
        for ex in range(n):
            for qy in range(3):
                for qx in range(3):
                    x, y = (ex + xg[qx]) * h, (ey + xg[qy]) * h
                    w = wg[qx] * wg[qy] * h * h
                    fn = [(j, i) for j in range(ey, ey + 3) for i in range(ex, ex + 3)]
                    val = {(j, i): bspline_scalar(knots, i, 2, x) * bspline_scalar(knots, j, 2, y) for j, i in fn}
                    gx = {(j, i): bspline_scalar_deriv(knots, i, 2, x) * bspline_scalar(knots, j, 2, y) for j, i in fn}
                    gy = {(j, i): bspline_scalar(knots, i, 2, x) * bspline_scalar_deriv(knots, j, 2, y) for j, i in fn}
                    s = min(max(sum(S[j, i] * val[j, i] for j, i in fn), 0.0), 1.0)
                    kk = sum(sc.K[j, i] * bspline_scalar(hat, j, 1, y) * bspline_scalar(hat, i, 1, x)
                             for i in (ex, ex + 1) for j in (ey, ey + 1))
                    lg, lw = s / sc.mu_g, (1 - s) / sc.mu_w
                    q = 0.0
                    for src in sc.sources:
                        G = math.exp(-((x - src.center[0]) ** 2 + (y - src.center[1]) ** 2)
                                     / (2 * src.sigma ** 2)) / (2 * math.pi * src.sigma ** 2)
                        q += src.rate * G if src.kind == 0 else -src.rate * G
                    for a in fn:
                        ia = a[0] * nb + a[1]
                        F[ia] += w * (q * val[a] - sc.grav * kk * (sc.rho_w * lw + sc.rho_g * lg) * gy[a])
                        for b in fn:
                            A[ia, b[0] * nb + b[1]] += w * (lg + lw) * kk * (gx[a] * gx[b] + gy[a] * gy[b])
    inner = [j * nb + i for j in range(1, nb - 1) for i in range(1, nb - 1)]
    p = np.linalg.solve(A[np.ix_(inner, inner)], F[inner])
    expect = np.zeros(nb * nb)
    expect[inner] = p
    P = galerkin_pressure(sc, S)
    # the scalar derivative is a central difference (error ~1e-9); a dropped
    # mobility or swapped density moves P by O(1e-2) or more
    np.testing.assert_allclose(P.ravel(), expect, rtol=0, atol=1e-7 * np.abs(expect).max())


def test_galerkin_pressure_sign():
    """An injector raises the pressure (Eq. 5: div(lambda K grad p) = -q)."""
    sc = scn.make_scenario(2, 16, seed=1)
    P = galerkin_pressure(sc, np.zeros((18, 18)))
    m = Mesh(2, 16)
    vals = m.ax.values_at([0.25, 0.75])
    pv = vals @ P @ vals.T  # [y][x] at (0.25,0.25),(0.75,0.25),...
    assert pv[0, 0] > 0 and pv[1, 1] < 0


# ----------------------------------------------------------------------------
# Higher spline degree (p = 3, 4): the same discretisation of Secs. 3-4 with
# B-splines of degree p, n + p functions per axis and p + 1 Gauss points
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("p,n", [(3, 1), (3, 6), (4, 2), (4, 9)])
def test_partition_of_unity_higher_degree(p, n):
    knots = open_uniform_knots(n, p)
    x = np.concatenate([np.random.default_rng(n + p).uniform(0, 1, 150), [0.0, 1.0, 0.5]])
    B = basis_values(knots, p, x)
    D = basis_derivatives(knots, p, x)
    assert B.shape[1] == n + p
    assert np.all(B >= -1e-15)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-10)
    xi = np.array([0.07, 0.33, 0.61, 0.94])
    Bi = basis_values(knots, p, xi)
    for i in range(n + p):
        for k, xv in enumerate(xi):
            assert Bi[k, i] == pytest.approx(bspline_scalar(knots, i, p, xv), abs=1e-14)


@pytest.mark.parametrize("p,n", [(3, 2), (3, 7), (4, 3), (4, 8)])
def test_basis_integrals_higher_degree(p, n):
    """int B_i = (t_{i+p+1} - t_i)/(p+1), with p + 1 Gauss points."""
    ax = Axis1D(n, p)
    t = ax.knots
    expect = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(n + p)])
    np.testing.assert_allclose(ax.B.T @ ax.w, expect, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_mass_rows_are_cardinal_bspline_values(p):
    with open(os.path.join(GOLDEN, "bspline_mass_rows_p234.json")) as f:
        g = json.load(f)
    row = np.array(g["rows_times_factorial"][str(p)], dtype=float) / g["factorial"][str(p)]
    # the fixture is the closed form: N_{2p+1} at the integers, evaluated here
    m = 2 * p + 1
    card = [bspline_scalar(np.arange(m + 2, dtype=float), 0, m, float(k)) for k in range(1, m + 1)]
    np.testing.assert_allclose(card, row, rtol=1e-13)
    n = 20
    ax = Axis1D(n, p)
    M, h = ax.M, 1.0 / n
    np.testing.assert_allclose(M, M.T, atol=1e-17)
    for i in range(2 * p, n - p):
        np.testing.assert_allclose(M[i, i - p:i + p + 1] / h, row, rtol=1e-12)
        assert np.all(M[i, :i - p] == 0) and np.all(M[i, i + p + 1:] == 0)


@pytest.mark.parametrize("dim,n,p", [(2, 3, 3), (2, 6, 4), (3, 2, 3)])
def test_kronecker_solve_equals_dense_higher_degree(dim, n, p):
    m = Mesh(dim, n, p)
    R = np.random.default_rng(dim + n + p).normal(size=(n + p,) * dim)
    Xk = m.mass_solve_kron(R)
    np.testing.assert_allclose(Xk, m.mass_solve_dense(R), rtol=0, atol=1e-11 * np.abs(Xk).max())


@pytest.mark.parametrize("dim,n,p", [(2, 5, 3), (2, 4, 4), (3, 3, 3)])
def test_constant_and_mass_balance_higher_degree(dim, n, p):
    sc = scn.make_scenario(dim, n, seed=2, p=p)
    sc.sources = []
    sc.grav = 0.0
    S = np.full((n + p,) * dim, 0.37)
    np.testing.assert_allclose(AdsOracle(sc).step(S, np.zeros_like(S), 0.01), 0.37, atol=1e-12)
    sc = scn.make_scenario(dim, n, seed=3, S0="random", grav=1.0, p=p)
    sc.phi_map = 0.1 + 0.3 * np.random.default_rng(9).uniform(size=(n + 1,) * dim)
    P = np.random.default_rng(4).normal(size=(n + p,) * dim)
    a = AdsOracle(sc)
    Sn = a.step(sc.S0, P, 0.002)
    assert abs(a.mass_error(sc.S0, Sn, 0.002)) <= 1e-13 * max(1.0, abs(a.mesh.integral(Sn)))


@pytest.mark.parametrize("p", [3, 4])
def test_rhs_matches_element_loop_higher_degree(p):
    sc = scn.make_scenario(2, 3, seed=5, S0="random", grav=0.7, p=p)
    sc.sources[0].center = (0.3, 0.4)
    sc.sources[1].center = (0.6, 0.7)
    sc.sources[0].sigma = sc.sources[1].sigma = 0.2
    rng = np.random.default_rng(12)
    S = rng.uniform(-0.1, 1.1, size=(3 + p, 3 + p))
    P = rng.normal(size=(3 + p, 3 + p))
    R = AdsOracle(sc).rhs(S, P, 0.013)
    Rb = _brute_rhs(sc, S, P, 0.013)
    np.testing.assert_allclose(R, Rb, rtol=0, atol=2e-7 * np.abs(Rb).max())


def test_galerkin_pressure_manufactured_cubic_h4():
    """As the quadratic case, with cubic B-splines: the L2 error falls like
    h^(p+1) = h^4."""
    import oracle.pressure as pr
    errs = []
    for n in (4, 8, 16):
        sc = scn.make_scenario(2, n, seed=1, p=3)
        sc.K = np.ones_like(sc.K)
        lam = 1.0 / sc.mu_w
        m = Mesh(2, n, 3)
        coords = m.gauss_coords()
        orig = pr.gaussian_sources
        pr.gaussian_sources = lambda s, c: (2 * np.pi ** 2 * lam * np.sin(np.pi * c[0]) * np.sin(np.pi * c[1]),
                                            np.zeros_like(c[0]))
        try:
            P = galerkin_pressure(sc, np.zeros((n + 3, n + 3)))
        finally:
            pr.gaussian_sources = orig
        ph = m.at_gauss(P)
        ex = np.sin(np.pi * coords[0]) * np.sin(np.pi * coords[1])
        errs.append(math.sqrt(np.sum(m.gauss_weights() * (ph - ex) ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 3.6, (errs, rates)


def test_library_refuses_other_degrees():
    from paper_2604_20731_gb300.solver import make_params
    with pytest.raises(ValueError):
        make_params(scn.make_scenario(2, 4, p=3))


# ----------------------------------------------------------------------------
# CRVPINN (Sec. 5)
# ----------------------------------------------------------------------------

def test_operator_matches_stencil_brute_force():
    sc = scn.make_scenario(2, 5, seed=4, S0="random", grav=0.8)
    c = CrvOracle(sc)
    alpha, f = c.coefficients(sc.S0)
    rng = np.random.default_rng(2)
    u_int = rng.normal(size=c.M)
    u = embed_interior(u_int, 2, 5)
    N, h = 5, 0.2
    res = []
    for j in range(1, N):
        for i in range(1, N):
            r = (alpha[j, i - 1] * (u[j, i] - u[j, i - 1]) - alpha[j, i] * (u[j, i + 1] - u[j, i])
                 + alpha[j - 1, i] * (u[j, i] - u[j - 1, i]) - alpha[j, i] * (u[j + 1, i] - u[j, i]))
            res.append(r)
    np.testing.assert_allclose(c.residual(alpha, f, u_int), np.array(res) + h * h * f, atol=1e-13)


def test_rhs_closed_form_brute_force():
    """Eq. 23b at one interior node, written out by hand."""
    sc = scn.make_scenario(2, 6, seed=8, S0="random", grav=1.3)
    c = CrvOracle(sc)
    alpha, f = c.coefficients(sc.S0)
    j, i = 2, 3
    knots = open_uniform_knots(6, 2)

    def s_at(jj, ii):
        x, y = ii / 6, jj / 6
        v = sum(sc.S0[b, a] * bspline_scalar(knots, a, 2, x) * bspline_scalar(knots, b, 2, y)
                for a in range(8) for b in range(8))
        return min(max(v, 0), 1)

    def rl(jj, ii):
        s = s_at(jj, ii)
        return sc.K[jj, ii] * ((1 - s) / sc.mu_w * sc.rho_w + s / sc.mu_g * sc.rho_g)
    s = s_at(j, i)
    assert alpha[j, i] == pytest.approx(((1 - s) / sc.mu_w + s / sc.mu_g) * sc.K[j, i], rel=1e-13)
    x, y = i / 6, j / 6
    qi = sc.sources[0].rate * math.exp(-((x - .25) ** 2 + (y - .25) ** 2) / (2 * .03 ** 2)) / (2 * math.pi * .03 ** 2)
    qp = sc.sources[1].rate * math.exp(-((x - .75) ** 2 + (y - .75) ** 2) / (2 * .03 ** 2)) / (2 * math.pi * .03 ** 2)
    expect = -sc.grav * (rl(j + 1, i) - rl(j, i)) * 6 - (qi - qp)
    assert f[(j - 1) * 5 + (i - 1)] == pytest.approx(expect, rel=1e-12, abs=1e-12)


def test_gram_routes_and_dst():
    for dim, N in ((2, 9), (2, 16), (3, 6)):
        sc = scn.make_scenario(dim, N, seed=1)
        c = CrvOracle(sc)
        r = np.random.default_rng(N).normal(size=c.M)
        q1 = c.gram_solve_lu(r)
        q2 = c.gram_solve_fd(r)
        np.testing.assert_allclose(q1, q2, rtol=0, atol=1e-12 * np.abs(q1).max())
        np.testing.assert_allclose(c.gram() @ q1, r, atol=1e-10 * np.abs(r).max())
    k = np.arange(1, 16)
    S = np.sqrt(2 / 16) * np.sin(np.pi * np.outer(k, k) / 16)
    np.testing.assert_allclose(S @ S, np.eye(15), atol=1e-14)


def test_gram_is_eq26_stencil():
    sc = scn.make_scenario(2, 4, seed=1)
    c = CrvOracle(sc)
    G = c.gram().toarray() * c.h ** 2
    # interior 3x3 grid, centre node index 4
    assert G[4, 4] == 4 and G[4, 3] == -1 and G[4, 5] == -1 and G[4, 1] == -1 and G[4, 7] == -1
    assert G[0, 4] == 0 and G[0, 8] == 0


def test_loss_equals_discrete_h1_error_for_unit_alpha():
    """With alpha = 1 the robust loss is h^2 |u - u*|^2_{grad,h} exactly
    (the inf-sup equivalence of Sec. 5 with the h^-2 Gram scaling of Eq. 26)."""
    N = 12
    sc = scn.make_scenario(2, N, seed=6)
    c = CrvOracle(sc)
    alpha = np.ones((N + 1, N + 1))
    f = np.random.default_rng(1).normal(size=c.M)
    ustar = c.direct_solution(alpha, f)
    u = np.random.default_rng(2).normal(size=c.M)
    r = c.residual(alpha, f, u)
    loss = r @ c.gram_solve_lu(r)
    e = embed_interior(u - ustar, 2, N)
    h = c.h
    dx = (e[:, 1:] - e[:, :-1]) / h
    dy = (e[1:, :] - e[:-1, :]) / h
    norm2 = h * h * (np.sum(dx ** 2) + np.sum(dy ** 2))
    assert loss == pytest.approx(h * h * norm2, rel=1e-10)


def test_direct_solution_discrete_manufactured():
    """A f built from a known u by the stencil formula is inverted exactly."""
    N = 10
    sc = scn.make_scenario(2, N, seed=7, S0="random")
    c = CrvOracle(sc)
    alpha, _ = c.coefficients(sc.S0)
    X = c.X
    uex = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) + X[:, 0] * X[:, 1] * (1 - X[:, 0])
    u = embed_interior(uex, 2, N)
    h = c.h
    lap = []
    for j in range(1, N):
        for i in range(1, N):
            lap.append((alpha[j, i] * (u[j, i + 1] - u[j, i]) - alpha[j, i - 1] * (u[j, i] - u[j, i - 1])
                        + alpha[j, i] * (u[j + 1, i] - u[j, i]) - alpha[j - 1, i] * (u[j, i] - u[j - 1, i])) / h ** 2)
    f = np.array(lap)  # div_-(alpha grad_+ u) = f  <=>  RES = 0
    np.testing.assert_allclose(c.direct_solution(alpha, f), uex, atol=1e-12)
    assert np.abs(c.residual(alpha, f, uex)).max() < 1e-13


def test_direct_solution_continuous_manufactured_h2():
    errs = []
    for N in (16, 32, 64):
        sc = scn.make_scenario(2, N, seed=1)
        c = CrvOracle(sc)
        alpha = np.ones((N + 1, N + 1))
        X = c.X
        f = -2 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
        u = c.direct_solution(alpha, f)
        errs.append(np.abs(u - np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.9, errs


def test_mlp_matches_torch_layers():
    torch = pytest.importorskip("torch")
    mlp = MLP(2, 8, 4)
    th = scn.make_theta0(2, 8, 4, seed=3)
    th = th + 0.1 * np.random.default_rng(0).normal(size=th.size)
    X = np.random.default_rng(1).uniform(size=(17, 2))
    u, _ = mlp.forward(th, X)
    layers, o = [], 0
    sizes = mlp.sizes
    for i in range(len(sizes) - 1):
        lin = torch.nn.Linear(sizes[i], sizes[i + 1]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(th[o:o + sizes[i + 1] * sizes[i]].reshape(sizes[i + 1], sizes[i])))
            o += sizes[i + 1] * sizes[i]
            lin.bias.copy_(torch.from_numpy(th[o:o + sizes[i + 1]]))
            o += sizes[i + 1]
        layers.append(lin)
        if i < len(sizes) - 2:
            layers.append(torch.nn.Tanh())
    net = torch.nn.Sequential(*layers)
    ut = net(torch.from_numpy(2 * X - 1)).detach().numpy()[:, 0]
    np.testing.assert_allclose(u, ut, rtol=1e-13, atol=1e-14)


def _loss_only(c, mlp, th, alpha, f):
    return c.loss_grad(mlp, th, alpha, f, with_grad=False)[0]


def test_gradient_finite_differences():
    sc = scn.make_scenario(2, 8, seed=3, S0="random", grav=0.5)
    c = CrvOracle(sc)
    mlp = MLP(2, 6, 4)
    th = scn.make_theta0(2, 6, 4, seed=2) + 0.05
    alpha, f = c.coefficients(sc.S0)
    loss, g, _ = c.loss_grad(mlp, th, alpha, f)
    rng = np.random.default_rng(11)
    for _ in range(16):
        d = rng.normal(size=th.size)
        d /= np.linalg.norm(d)
        eps = 1e-4
        fd = (_loss_only(c, mlp, th + eps * d, alpha, f) - _loss_only(c, mlp, th - eps * d, alpha, f)) / (2 * eps)
        assert g @ d == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(loss))


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    sc = scn.make_scenario(2, 7, seed=4, S0="random")
    c = CrvOracle(sc)
    mlp = MLP(2, 5, 4)
    th = scn.make_theta0(2, 5, 4, seed=5) + 0.02
    alpha, f = c.coefficients(sc.S0)
    loss, g, _ = c.loss_grad(mlp, th, alpha, f)
    A = torch.from_numpy(c.operator(alpha).toarray())
    Ginv = torch.linalg.inv(torch.from_numpy(c.gram().toarray()))
    t = torch.from_numpy(th).requires_grad_(True)
    X = torch.from_numpy(2 * c.X - 1)
    a, o = X, 0
    sizes = mlp.sizes
    for i in range(len(sizes) - 1):
        W = t[o:o + sizes[i + 1] * sizes[i]].reshape(sizes[i + 1], sizes[i]); o += sizes[i + 1] * sizes[i]
        b = t[o:o + sizes[i + 1]]; o += sizes[i + 1]
        a = a @ W.T + b
        if i < len(sizes) - 2:
            a = torch.tanh(a)
    r = A @ a[:, 0] + c.h ** 2 * torch.from_numpy(f)
    lt = r @ (Ginv @ r)
    lt.backward()
    assert float(lt.detach()) == pytest.approx(loss, rel=1e-12)
    np.testing.assert_allclose(g, t.grad.numpy(), rtol=1e-9, atol=1e-12 * np.abs(g).max())


def test_adam_closed_form():
    """A constant gradient moves every parameter by lr*g/(|g|+eps) per step."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th0 = np.array([1.0, 2.0, 3.0, 4.0])
    opt = Adam(4)
    th = th0
    for _ in range(3):
        th = opt.step(th, g, 0.01)
    np.testing.assert_allclose(th, th0 - 3 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


# ----------------------------------------------------------------------------
# projection and the loops (Sec. 6, Sec. 7)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dim,p", [(2, 2), (3, 2), (2, 3), (2, 4), (3, 3)])
def test_projection_reproduces_multilinear(dim, p):
    n = 6
    m = Mesh(dim, n, p)
    nodes = np.arange(n + 1) / n
    grids = list(reversed(np.meshgrid(*([nodes] * dim), indexing="ij")))
    nodal = 0.4 + 1.3 * grids[0] - 0.7 * grids[1] + 2.1 * grids[0] * grids[1]
    P = project_nodal(m, nodal)
    pts = np.random.default_rng(1).uniform(size=(dim, 5))
    vals = [m.ax.values_at(pts[c]) for c in range(dim)]
    for k in range(5):
        mats = [vals[dim - 1 - a][k:k + 1] for a in range(dim)]
        from oracle.ads import along
        v = along(P, mats).ravel()[0]
        x, y = pts[0, k], pts[1, k]
        assert v == pytest.approx(0.4 + 1.3 * x - 0.7 * y + 2.1 * x * y, abs=1e-12)


@pytest.mark.parametrize("p", [2, 3])
def test_plain_step_mass_balance_over_ten_steps(p):
    sc = scn.make_scenario(2, 12, seed=1000, p=p)
    S0 = sc.S0_or_zero()
    S, P, dt = plain_step(sc, S0, 10)
    a = AdsOracle(sc)
    src = 0.0
    Sk = S0
    for _ in range(10):
        src += a.source_integral(Sk, dt)
        Sk = a.step(Sk, P, dt)
    np.testing.assert_allclose(Sk, S, atol=1e-15)
    assert a.mesh.integral(S) == pytest.approx(src, rel=1e-12)


def test_hybrid_short_run_reduces_loss():
    sc = scn.make_scenario(2, 8, seed=1000)
    h = HybridOracle(sc, width=8)
    th = scn.make_theta0(2, 8, 4)
    opt = Adam(th.size)
    th, losses = h.train(th, opt, sc.S0_or_zero(), 200, 1e-2)
    assert losses[-1] < 0.2 * losses[0]
    S, P, th2, dt, l2 = h.hybrid_step(sc.S0_or_zero(), th, opt, n_sub=2, adam_iters=3, lr=1e-2)
    assert np.isfinite(S).all() and dt > 0 and len(l2) == 3


# ----------------------------------------------------------------------------
# 3D with a vertical permeability K_z = kz K (reading R23): the flux of the
# saturation step, the 7-point operator and the gravity divergence of Eq. 23b
# ----------------------------------------------------------------------------

def _brute_rhs_3d(sc, S, P, dt):
    """Element loop over a 3D mesh with pointwise scalar basis evaluation: the
    right-hand side of Eq. 10b with the vertical (z, array axis 0) Darcy flux
    scaled by kz and gravity acting along -z."""
    n = sc.n
    knots = open_uniform_knots(n, 2)
    hat = open_uniform_knots(n, 1)
    xg, wg = np.polynomial.legendre.leggauss(3)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    h = 1.0 / n
    R = np.zeros((n + 2,) * 3)
    for ez in range(n):
        for ey in range(n):
            for ex in range(n):
                for qz in range(3):
                    for qy in range(3):
                        for qx in range(3):
                            x, y, z = (ex + xg[qx]) * h, (ey + xg[qy]) * h, (ez + xg[qz]) * h
                            w = wg[qx] * wg[qy] * wg[qz] * h ** 3
                            bx = {i: bspline_scalar(knots, i, 2, x) for i in range(ex, ex + 3)}
                            by = {j: bspline_scalar(knots, j, 2, y) for j in range(ey, ey + 3)}
                            bz = {k: bspline_scalar(knots, k, 2, z) for k in range(ez, ez + 3)}
                            dbx = {i: bspline_scalar_deriv(knots, i, 2, x) for i in bx}
                            dby = {j: bspline_scalar_deriv(knots, j, 2, y) for j in by}
                            dbz = {k: bspline_scalar_deriv(knots, k, 2, z) for k in bz}
                            idx = [(k, j, i) for k in bz for j in by for i in bx]
                            s = sum(S[k, j, i] * bz[k] * by[j] * bx[i] for k, j, i in idx)
                            px = sum(P[k, j, i] * bz[k] * by[j] * dbx[i] for k, j, i in idx)
                            py = sum(P[k, j, i] * bz[k] * dby[j] * bx[i] for k, j, i in idx)
                            pz = sum(P[k, j, i] * dbz[k] * by[j] * bx[i] for k, j, i in idx)
                            kk = sum(sc.K[k, j, i] * bspline_scalar(hat, k, 1, z) * bspline_scalar(hat, j, 1, y)
                                     * bspline_scalar(hat, i, 1, x)
                                     for k in (ez, ez + 1) for j in (ey, ey + 1) for i in (ex, ex + 1))
                            st = min(max(s, 0.0), 1.0)
                            lg, lw = st / sc.mu_g, (1 - st) / sc.mu_w
                            qi = qp = 0.0
                            for src in sc.sources:
                                r2 = (x - src.center[0]) ** 2 + (y - src.center[1]) ** 2 + (z - src.center[2]) ** 2
                                G = math.exp(-r2 / (2 * src.sigma ** 2)) / (2 * math.pi * src.sigma ** 2) ** 1.5
                                if src.kind == 0:
                                    qi += src.rate * G
                                else:
                                    qp += src.rate * G
                            qg = qi - lg / (lg + lw) * qp
                            fx = kk * px
                            fy = kk * py
                            fz = sc.kz_ratio * kk * (pz + sc.grav_sign * sc.rho_g * sc.grav)
                            for k, j, i in idx:
                                v = bx[i] * by[j] * bz[k]
                                vx = dbx[i] * by[j] * bz[k]
                                vy = bx[i] * dby[j] * bz[k]
                                vz = bx[i] * by[j] * dbz[k]
                                R[k, j, i] += w * (s * v + dt / sc.phi * (qg * v - lg * (fx * vx + fy * vy + fz * vz)))
    return R


def test_rhs_matches_element_loop_3d_anisotropic():
    """The 3D saturation right-hand side with K_z = 0.1 K, gravity on and the
    clamp active, against the element loop.  A K_z on the wrong axis or on the
    wrong velocity component changes R by far more than the tolerance."""
    sc = scn.make_scenario(3, 3, seed=12, S0="random", grav=0.9, kz_ratio=0.1)
    sc.sources[0].center = (0.3, 0.45, 0.6)
    sc.sources[1].center = (0.7, 0.35, 0.25)
    sc.sources[0].sigma = sc.sources[1].sigma = 0.25
    rng = np.random.default_rng(13)
    S = rng.uniform(-0.1, 1.1, size=(5, 5, 5))
    P = rng.normal(size=(5, 5, 5))
    dt = 0.011
    R = AdsOracle(sc).rhs(S, P, dt)
    Rb = _brute_rhs_3d(sc, S, P, dt)
    np.testing.assert_allclose(R, Rb, rtol=0, atol=2e-7 * np.abs(Rb).max())
    # the anisotropy is visible at this tolerance: the isotropic flux differs
    sc_iso = scn.make_scenario(3, 3, seed=12, S0="random", grav=0.9, kz_ratio=1.0)
    sc_iso.sources = sc.sources
    R_iso = AdsOracle(sc_iso).rhs(S, P, dt)
    assert np.abs(R_iso - Rb).max() > 1e-3 * np.abs(Rb).max()


def test_cfl_dt_rule_3d_vertical_gradient():
    """With p linear in z only, |K (grad p)| = kz K dp/dz: the velocity limit
    sees the vertical permeability, not K."""
    n = 4
    sc = scn.make_scenario(3, n, seed=1, kz_ratio=0.25)
    sc.sources = []
    sc.K = np.full_like(sc.K, 2.0)
    knots = open_uniform_knots(n, 2)
    grev = np.array([(knots[i + 1] + knots[i + 2]) / 2 for i in range(n + 2)])
    P = np.broadcast_to(100.0 * grev[:, None, None], (n + 2,) * 3).copy()  # p = 100 z
    dt = AdsOracle(sc).cfl_dt(P)
    vmax = 0.25 * 2.0 * 100.0 / (sc.mu_g * sc.phi)
    assert dt == pytest.approx(0.1 * (1 / n) / vmax, rel=1e-12)
    # the same gradient along x sees K itself
    Px = np.broadcast_to(100.0 * grev[None, None, :], (n + 2,) * 3).copy()
    dtx = AdsOracle(sc).cfl_dt(Px)
    assert dtx == pytest.approx(0.1 * (1 / n) / (2.0 * 100.0 / (sc.mu_g * sc.phi)), rel=1e-12)


def test_operator_matches_stencil_brute_force_3d_anisotropic():
    """7-point residual with the vertical differences weighted by kz."""
    N = 4
    sc = scn.make_scenario(3, N, seed=4, S0="random", grav=0.8, kz_ratio=0.3)
    c = CrvOracle(sc)
    alpha, f = c.coefficients(sc.S0)
    u_int = np.random.default_rng(2).normal(size=c.M)
    u = embed_interior(u_int, 3, N)
    h = 1.0 / N
    res = []
    for k in range(1, N):
        for j in range(1, N):
            for i in range(1, N):
                r = (alpha[k, j, i - 1] * (u[k, j, i] - u[k, j, i - 1])
                     - alpha[k, j, i] * (u[k, j, i + 1] - u[k, j, i])
                     + alpha[k, j - 1, i] * (u[k, j, i] - u[k, j - 1, i])
                     - alpha[k, j, i] * (u[k, j + 1, i] - u[k, j, i])
                     + 0.3 * (alpha[k - 1, j, i] * (u[k, j, i] - u[k - 1, j, i])
                              - alpha[k, j, i] * (u[k + 1, j, i] - u[k, j, i])))
                res.append(r)
    np.testing.assert_allclose(c.residual(alpha, f, u_int), np.array(res) + h * h * f, atol=1e-13)


def test_rhs_closed_form_brute_force_3d():
    """Eq. 23b at one interior 3D node, written out by hand: the gravity
    divergence is a forward difference along z of kz K (rho_w lambda_w +
    rho_g lambda_g), and the Gaussians carry the 3D normalisation."""
    N = 5
    sc = scn.make_scenario(3, N, seed=8, S0="random", grav=1.3, kz_ratio=0.2)
    c = CrvOracle(sc)
    alpha, f = c.coefficients(sc.S0)
    knots = open_uniform_knots(N, 2)
    k0, j0, i0 = 2, 1, 3

    def s_at(kk, jj, ii):
        x, y, z = ii / N, jj / N, kk / N
        v = sum(sc.S0[cz, b, a] * bspline_scalar(knots, a, 2, x) * bspline_scalar(knots, b, 2, y)
                * bspline_scalar(knots, cz, 2, z)
                for a in range(N + 2) for b in range(N + 2) for cz in range(N + 2))
        return min(max(v, 0), 1)

    def rl(kk, jj, ii):
        s = s_at(kk, jj, ii)
        return 0.2 * sc.K[kk, jj, ii] * ((1 - s) / sc.mu_w * sc.rho_w + s / sc.mu_g * sc.rho_g)
    s = s_at(k0, j0, i0)
    assert alpha[k0, j0, i0] == pytest.approx(((1 - s) / sc.mu_w + s / sc.mu_g) * sc.K[k0, j0, i0], rel=1e-13)
    x, y, z = i0 / N, j0 / N, k0 / N
    norm = (2 * math.pi * 0.03 ** 2) ** 1.5
    qi = sc.sources[0].rate * math.exp(-((x - .25) ** 2 + (y - .25) ** 2 + (z - .25) ** 2) / (2 * .03 ** 2)) / norm
    qp = sc.sources[1].rate * math.exp(-((x - .75) ** 2 + (y - .75) ** 2 + (z - .75) ** 2) / (2 * .03 ** 2)) / norm
    expect = -sc.grav * (rl(k0 + 1, j0, i0) - rl(k0, j0, i0)) * N - (qi - qp)
    m = N - 1
    assert f[((k0 - 1) * m + (j0 - 1)) * m + (i0 - 1)] == pytest.approx(expect, rel=1e-12, abs=1e-12)


def test_loss_equals_discrete_h1_error_for_unit_alpha_3d():
    """3D twin of the inf-sup identity: with alpha = 1 and kz = 1 the 7-point
    residual operator is h^2 G, so LOSS = h^2 sum over grid edges of the
    squared jump of u - u* (Eq. 26 with the {6, -1} stencil)."""
    N = 6
    sc = scn.make_scenario(3, N, seed=6)
    c = CrvOracle(sc)
    alpha = np.ones((N + 1,) * 3)
    f = np.random.default_rng(1).normal(size=c.M)
    ustar = c.direct_solution(alpha, f)
    u = np.random.default_rng(2).normal(size=c.M)
    r = c.residual(alpha, f, u)
    e = embed_interior(u - ustar, 3, N)
    jumps = sum(np.sum(np.diff(e, axis=a) ** 2) for a in range(3))
    h = c.h
    for loss in (r @ c.gram_solve_lu(r), r @ c.gram_solve_fd(r)):
        assert loss == pytest.approx(h * h * jumps, rel=1e-10)
