"""Parity of the GPU Galerkin pressure (the plain method of Sec. 7) with the
oracle's sparse direct solve of the same system (Sec. 4, Eqs. 15-20; weak form
Eq. 12a), and of the plain step (Galerkin pressure + explicit saturation
steps) with the oracle's.

Tolerances: both sides solve the same SPD system directly in FP64 (banded
Cholesky here, SuperLU in the oracle).  Their difference is bounded by
cond(A) * eps; at these sizes cond(A) <= ~1e5 (h^-2 times the permeability
contrast of a sigma = 1 field), so relative L-inf <= 1e-9 holds with margin.
FP32 inputs (ads_dtype f32) round S and K by 6e-8 relative and store P in FP32;
the bound there is 1e-5.  The saturation after the plain step inherits the
pressure's difference through the flux (dt |grad dp| with dt from the CFL
rule), so it is held to the same 1e-9.
"""
import numpy as np
import pytest

from oracle.ads import AdsOracle
from oracle.hybrid import plain_step
from oracle.pressure import galerkin_pressure
from paper_2604_20731_gb300 import scenario as scn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def solver(sc, **kw):
    from paper_2604_20731_gb300.solver import HybridSolver
    return HybridSolver(sc, width=None, **kw)


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _scenario(n, seed=5, grav=0.6):
    sc = scn.make_scenario(2, n, seed=seed, S0="random", grav=grav)
    # saturation outside [0, 1] exercises the clamp inside the mobilities
    rng = np.random.default_rng(seed + 1)
    sc.S0 = rng.uniform(-0.15, 1.15, size=(n + 2, n + 2))
    return sc


# n = 2, 3: fewer unknowns than the band; 32: configuration 1; 78 / 79: the
# last size with the shared-memory row window and the first without; 120:
# the triangular sweeps' vectors no longer fit in shared memory
@pytest.mark.parametrize("n", [2, 3, 8, 32, 78, 79, 120])
def test_galerkin_pressure_fp64(n):
    sc = _scenario(n, grav=0.6 if n % 2 == 0 else 0.0)
    ref = galerkin_pressure(sc, sc.S0)
    s = solver(sc, ads_dtype="f64")
    try:
        s.set_saturation(sc.S0)
        s.galerkin_pressure()
        P = s.get("P")
    finally:
        s.close()
    assert P.shape == ref.shape
    assert np.all(P[0, :] == 0) and np.all(P[-1, :] == 0) and np.all(P[:, 0] == 0) and np.all(P[:, -1] == 0)
    assert rel_inf(P, ref) <= 1e-9


def test_galerkin_pressure_fp32_storage():
    n = 32
    sc = _scenario(n)
    ref = galerkin_pressure(sc, sc.S0)
    s = solver(sc, ads_dtype="f32")
    try:
        s.set_saturation(sc.S0)
        s.galerkin_pressure()
        P = s.get("P")
    finally:
        s.close()
    assert rel_inf(P, ref) <= 1e-5


def test_galerkin_pressure_repeat_is_identical():
    """A second call reuses the workspace and gives the same bits."""
    sc = _scenario(16)
    s = solver(sc, ads_dtype="f64")
    try:
        s.set_saturation(sc.S0)
        s.galerkin_pressure()
        P1 = s.get("P")
        s.galerkin_pressure()
        P2 = s.get("P")
    finally:
        s.close()
    assert np.array_equal(P1, P2)


def test_plain_step_configuration_1():
    """Configuration 1: 32 x 32 elements, FP64, S0 = 0, 10 explicit steps with
    the CFL step size; two plain steps, so the second one's pressure sees a
    non-zero saturation."""
    n = 32
    sc = scn.make_scenario(2, n, seed=1000)
    S = sc.S0_or_zero()
    s = solver(sc, ads_dtype="f64")
    try:
        for _ in range(2):
            S, P, dt = plain_step(sc, S, 10, cfl=0.1)
            s.plain_step(10, cfl=0.1)
            assert rel_inf(s.get("P"), P) <= 1e-9
            assert abs(s.get("DT")[0] - dt) <= 1e-9 * dt
            assert rel_inf(s.get("S"), S) <= 1e-9
        mass = s.get("MASS")
    finally:
        s.close()
    # the explicit steps conserve mass whatever the pressure
    assert abs(mass[1]) <= 1e-12 * max(abs(mass[0]), 1.0)
    assert AdsOracle(sc).mesh.integral(S) == pytest.approx(mass[0], rel=1e-9)


def test_galerkin_pressure_3d_unsupported():
    from paper_2604_20731_gb300._lib import AdsError
    sc = scn.make_scenario(3, 4, seed=2)
    s = solver(sc, ads_dtype="f64")
    try:
        with pytest.raises(AdsError, match="unsupported"):
            s.galerkin_pressure()
        # the context stays usable
        s.saturation_step(1e-3, 1)
        assert np.isfinite(s.get("S")).all()
    finally:
        s.close()
