"""Oracle: B-spline bases, Gauss rules and 1D mass matrices (Sec. 4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The saturation and pressure fields are tensor products of 1D B-splines of
degree r with C^{r-1} continuity on an open uniform knot vector (Sec. 4,
Eq. 11b).  Basis values come from the Cox-de Boor recursion, derivatives from
its standard derivative formula.  Gauss-Legendre points: r+1 per axis per
element (the paper does not name the rule; r+1 points integrate the mass
matrix exactly).
"""
from __future__ import annotations

import numpy as np


def open_uniform_knots(n: int, p: int) -> np.ndarray:
    """Knots 0 (p+1 times), 1/n, ..., (n-1)/n, 1 (p+1 times); n+p functions."""
    inner = np.arange(n + 1, dtype=np.float64) / n
    return np.concatenate([np.zeros(p), inner, np.ones(p)])


def _degree0(knots: np.ndarray, x: np.ndarray) -> np.ndarray:
    nb = len(knots) - 1
    B = np.zeros((x.size, nb))
    last = max(i for i in range(nb) if knots[i + 1] > knots[i])
    for i in range(nb):
        lo, hi = knots[i], knots[i + 1]
        if hi <= lo:
            continue
        inside = (x >= lo) & (x < hi)
        if i == last:  # close the last non-empty interval on the right
            inside |= (x == hi)
        B[:, i] = inside
    return B


def basis_values(knots: np.ndarray, p: int, x) -> np.ndarray:
    """Cox-de Boor: B_{i,p}(x) for all i, shape (len(x), len(knots)-p-1)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    B = _degree0(knots, x)
    for k in range(1, p + 1):
        nb = len(knots) - 1 - k
        Bn = np.zeros((x.size, nb))
        for i in range(nb):
            d1 = knots[i + k] - knots[i]
            d2 = knots[i + k + 1] - knots[i + 1]
            if d1 > 0:
                Bn[:, i] += (x - knots[i]) / d1 * B[:, i]
            if d2 > 0:
                Bn[:, i] += (knots[i + k + 1] - x) / d2 * B[:, i + 1]
        B = Bn
    return B


def basis_derivatives(knots: np.ndarray, p: int, x) -> np.ndarray:
    """B'_{i,p}(x) = p/(t_{i+p}-t_i) B_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) B_{i+1,p-1}."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    Bm = basis_values(knots, p - 1, x)
    nb = len(knots) - 1 - p
    D = np.zeros((x.size, nb))
    for i in range(nb):
        d1 = knots[i + p] - knots[i]
        d2 = knots[i + p + 1] - knots[i + 1]
        if d1 > 0:
            D[:, i] += p / d1 * Bm[:, i]
        if d2 > 0:
            D[:, i] -= p / d2 * Bm[:, i + 1]
    return D


def gauss_rule(npts: int):
    """Gauss-Legendre points and weights on [0, 1]."""
    xi, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (xi + 1.0), 0.5 * w


def gauss_points_1d(n: int, npts: int):
    """All quadrature points of a uniform n-element mesh of [0,1], element by
    element (element e holds points e*npts .. e*npts+npts-1), and weights."""
    xi, w = gauss_rule(npts)
    h = 1.0 / n
    e = np.arange(n)[:, None]
    x = (e + xi[None, :]) * h
    wq = np.broadcast_to(w[None, :] * h, x.shape)
    return x.ravel(), np.ascontiguousarray(wq).ravel()


class Axis1D:
    """Everything the oracle needs along one axis of a uniform mesh.

    B, dB: degree-p basis values/derivatives at every Gauss point,
           shape (n*(p+1), n+p).
    H:     degree-1 (hat) basis at every Gauss point, shape (n*(p+1), n+1);
           H @ nodal_values is the piecewise-linear interpolant, which the
           oracle uses for the nodal permeability/porosity maps and for the
           network pressure.
    x, w:  Gauss points and weights.
    M:     1D mass matrix M_ik = int B_i B_k (Eq. 14).
    """

    def __init__(self, n: int, p: int = 2):
        self.n, self.p = n, p
        self.h = 1.0 / n
        self.knots = open_uniform_knots(n, p)
        self.x, self.w = gauss_points_1d(n, p + 1)
        self.B = basis_values(self.knots, p, self.x)
        self.dB = basis_derivatives(self.knots, p, self.x)
        self.H = basis_values(open_uniform_knots(n, 1), 1, self.x)
        self.M = self.B.T @ (self.w[:, None] * self.B)
        self.nodes = np.arange(n + 1, dtype=np.float64) / n

    def values_at(self, x) -> np.ndarray:
        return basis_values(self.knots, self.p, x)


def mass_matrix(n: int, p: int = 2) -> np.ndarray:
    return Axis1D(n, p).M
