"""Host-side check of the chunked line-sweep design used by the GPU mass solves.

The GPU splits each banded LDL^T line solve (Eqs. 14-15) into chunks that start
their forward and backward substitutions from a zero state H rows outside the
chunk.  The truncation error is a solution of the homogeneous recurrence of
the unit lower factor; for the quadratic B-spline mass matrix it shrinks by
rho = 0.43058 per row, the root inside the unit circle of the symbol of the
interior row [1, 26, 66, 26, 1] / 120.  These tests emulate the chunking in
numpy (FP64) on the oracle's 1D mass matrix and check the bound for the
halo widths the kernels use (24 rows in FP32, 48 in FP64).
"""
import numpy as np
import pytest

from oracle.bspline import Axis1D


def _mass(n):
    M = Axis1D(n).M
    M = M() if callable(M) else M
    return np.asarray(M.todense() if hasattr(M, "todense") else M, dtype=np.float64)


def _ldlt_pentadiag(M):
    """Unit lower factor coefficients (l1, l2) and D of a symmetric
    pentadiagonal SPD matrix, written out directly."""
    nb = M.shape[0]
    l1 = np.zeros(nb + 2)
    l2 = np.zeros(nb + 2)
    D = np.zeros(nb)
    for i in range(nb):
        b = M[i, i - 2] / D[i - 2] if i >= 2 else 0.0
        a = (M[i, i - 1] - b * l1[i - 1] * D[i - 2]) / D[i - 1] if i >= 1 else 0.0
        D[i] = M[i, i] - a * a * (D[i - 1] if i >= 1 else 0) - b * b * (D[i - 2] if i >= 2 else 0)
        l1[i], l2[i] = a, b
    return l1, l2, D


def _chunked_solve(l1, l2, D, r, chunk, H):
    nb = r.size
    x = np.zeros(nb)
    y = np.zeros(nb)
    # forward substitution per chunk from a zero state H rows early
    for s in range(0, nb, chunk):
        e = min(nb, s + chunk)
        y1 = y2 = 0.0
        for l in range(max(0, s - H), e):
            v = r[l] - l1[l] * y1 - l2[l] * y2
            if l >= s:
                y[l] = v
            y2, y1 = y1, v
    # backward substitution per chunk from a zero state H rows late
    for s in range(0, nb, chunk):
        e = min(nb, s + chunk)
        x1 = x2 = 0.0
        for l in range(min(nb, e + H) - 1, s - 1, -1):
            v = y[l] / D[l] - l1[l + 1] * x1 - l2[l + 2] * x2
            if l < e:
                x[l] = v
            x2, x1 = x1, v
    return x


def test_decay_rate_is_the_symbol_root():
    roots = np.roots([1.0, 26.0, 66.0, 26.0, 1.0])
    rho = np.abs(roots[np.abs(roots) < 1]).max()
    assert rho == pytest.approx(0.4305753471, abs=1e-9)
    Minv = np.linalg.inv(_mass(200))
    col = np.abs(Minv[:, 100])
    # ratios of consecutive entries of the inverse's column approach rho
    assert col[121] / col[120] == pytest.approx(rho, rel=1e-6)


def test_factorisation_matches_dense():
    M = _mass(40)
    l1, l2, D = _ldlt_pentadiag(M)
    nb = M.shape[0]
    L = np.eye(nb)
    for i in range(nb):
        if i >= 1:
            L[i, i - 1] = l1[i]
        if i >= 2:
            L[i, i - 2] = l2[i]
    np.testing.assert_allclose(L @ np.diag(D) @ L.T, M, rtol=0, atol=1e-15)


@pytest.mark.parametrize("H,bound", [(24, 1e-7), (32, 1e-10), (48, 1e-15)])
@pytest.mark.parametrize("chunk", [64, 127])
def test_chunked_sweep_error_bound(H, bound, chunk):
    n = 700
    M = _mass(n)
    l1, l2, D = _ldlt_pentadiag(M)
    rng = np.random.default_rng(5)
    r = rng.standard_normal(n + 2)
    x = np.linalg.solve(M, r)
    xc = _chunked_solve(l1, l2, D, r, chunk, H)
    rel = np.abs(xc - x).max() / np.abs(x).max()
    # the unchunked sweep's own rounding error is the floor
    full = np.abs(_chunked_solve(l1, l2, D, r, n + 2, 0) - x).max() / np.abs(x).max()
    rho = 0.4305753471
    assert rel < bound
    assert rel <= full + 100 * rho ** H


def test_halo_zero_is_visibly_wrong():
    # the check has teeth: without a halo the chunk edges are far off
    n = 300
    M = _mass(n)
    l1, l2, D = _ldlt_pentadiag(M)
    r = np.random.default_rng(6).standard_normal(n + 2)
    x = np.linalg.solve(M, r)
    xc = _chunked_solve(l1, l2, D, r, 64, 0)
    assert np.abs(xc - x).max() / np.abs(x).max() > 1e-3


def test_single_chunk_is_exact():
    n = 50
    M = _mass(n)
    l1, l2, D = _ldlt_pentadiag(M)
    r = np.random.default_rng(7).standard_normal(n + 2)
    np.testing.assert_allclose(_chunked_solve(l1, l2, D, r, 127, 32), np.linalg.solve(M, r),
                               rtol=1e-12, atol=1e-12 * np.abs(r).max())


# ----------------------------------------------------------------------------
# Higher spline degree (p = 3, 4): halos the chunked sweeps will need.  The
# band has p sub-diagonals; the truncation shrinks by the root inside the unit
# circle of the interior row's symbol (the cardinal B-spline of degree 2p+1 at
# the integers).  Halos of 32 / 64 rows (p = 3) and 40 / 80 rows (p = 4) keep
# it below FP32 / FP64 rounding; the quadratic halos (24 / 48) do not.
# ----------------------------------------------------------------------------

HALOS = {3: (32, 64), 4: (40, 80)}


def _golden_row(p):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "bspline_mass_rows_p234.json")) as f:
        return np.array(json.load(f)["rows_times_factorial"][str(p)], dtype=float)


def _ldlt_band(M, p):
    """Unit lower factor L[i, k] = L_{i, i-k} (k = 1..p) and D of a symmetric
    banded SPD matrix, by the column recurrences written out directly."""
    nb = M.shape[0]
    L = np.zeros((nb, p + 1))
    D = np.zeros(nb)
    for i in range(nb):
        for k in range(p, 0, -1):
            j = i - k
            if j < 0:
                continue
            v = M[i, j] - sum(L[i, i - m] * L[j, j - m] * D[m] for m in range(max(0, i - p), j))
            L[i, k] = v / D[j]
        D[i] = M[i, i] - sum(L[i, k] ** 2 * D[i - k] for k in range(1, p + 1) if i - k >= 0)
    return L, D


def _chunked_band_solve(L, D, r, p, chunk, H):
    nb = r.size
    y = np.zeros(nb)
    x = np.zeros(nb)
    for s in range(0, nb, chunk):
        e = min(nb, s + chunk)
        st = {}
        for l in range(max(0, s - H), e):
            st[l] = r[l] - sum(L[l, k] * st.get(l - k, 0.0) for k in range(1, p + 1))
            if l >= s:
                y[l] = st[l]
    for s in range(0, nb, chunk):
        e = min(nb, s + chunk)
        st = {}
        for l in range(min(nb, e + H) - 1, s - 1, -1):
            st[l] = y[l] / D[l] - sum(L[l + k, k] * st.get(l + k, 0.0)
                                      for k in range(1, p + 1) if l + k < nb)
            if l < e:
                x[l] = st[l]
    return x


@pytest.mark.parametrize("p", [3, 4])
def test_decay_rate_higher_degree(p):
    roots = np.roots(_golden_row(p))
    rho = np.abs(roots[np.abs(roots) < 1]).max()
    Minv = np.linalg.inv(np.asarray(Axis1D(200, p).M))
    col = np.abs(Minv[:, 100])
    assert col[131] / col[130] == pytest.approx(rho, rel=1e-5)


@pytest.mark.parametrize("p", [3, 4])
def test_chunked_sweep_halos_higher_degree(p):
    n = 200
    M = np.asarray(Axis1D(n, p).M)
    L, D = _ldlt_band(M, p)
    r = np.random.default_rng(p).normal(size=M.shape[0])
    xe = np.linalg.solve(M, r)

    def err(H):
        x = _chunked_band_solve(L, D, r, p, 64, H)
        return np.abs(x - xe).max() / np.abs(xe).max()

    floor = err(n + p)  # no truncation: the emulation's own rounding
    h32, h64 = HALOS[p]
    assert err(h32) <= 2.0 ** -24 / 8
    assert err(h64) <= 2 * floor + 2.0 ** -53
    # the quadratic splines' halos are too short here
    assert err(24) > 2.0 ** -24 / 8
    assert err(48) > 8 * 2.0 ** -53
