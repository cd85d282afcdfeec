"""Oracle: Galerkin B-spline pressure system (Sec. 4, Eqs. 15-20) solved by a
sparse direct factorisation -- the role MUMPS plays in the IGA-ADS-MUMPS
algorithm of Sec. 7.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

System: (lambda K grad B_ij, grad B_kl) p = (g K rho lambda, grad B_kl)
        + (q_w + q_g, B_kl) for interior test functions, i.e. the weak form
Eq. 12a.  Readings: Eqs. 15, 18 and 20 write a divergence of scalar basis
functions, read as the gradient; the source enters with the sign of Eq. 12a
(Eqs. 15/20 print the opposite sign, which contradicts Eq. 5).  Dirichlet
p = 0 on the whole boundary (Sec. 8.1): the first and last basis function of
every axis are removed.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .ads import Mesh, gaussian_sources, mobilities


def _kron_all(mats):
    out = sp.csr_matrix(mats[0])
    for m in mats[1:]:
        out = sp.kron(out, sp.csr_matrix(m), format="csr")
    return out


def galerkin_pressure(sc, S: np.ndarray) -> np.ndarray:
    """Pressure B-spline coefficients (n+p)^d with zero boundary ring."""
    d = sc.dim
    deg = getattr(sc, "p", 2)
    m = Mesh(d, sc.n, deg)
    ax = m.ax
    W = m.gauss_weights().ravel()
    coords = m.gauss_coords()
    Kq = m.nodal_at_gauss(np.asarray(sc.K, dtype=np.float64)).ravel()
    Sq = m.at_gauss(S).ravel()
    lam_g, lam_w = mobilities(sc, Sq)
    lam = lam_g + lam_w
    rho_lam = lam_w * sc.rho_w + lam_g * sc.rho_g
    q_inj, q_prod = gaussian_sources(sc, coords)
    q_tot = (q_inj - q_prod).ravel()

    Phi0 = _kron_all([ax.B] * d)
    Smat = None
    F = Phi0.T @ (W * q_tot)
    for c in range(d):
        a = d - 1 - c
        Phic = _kron_all([ax.dB if b == a else ax.B for b in range(d)])
        Kc = Kq * (sc.kz_ratio if (d == 3 and c == d - 1) else 1.0)
        term = Phic.T @ sp.diags(W * lam * Kc) @ Phic
        Smat = term if Smat is None else Smat + term
        if c == d - 1:  # g points down the vertical axis
            F = F + Phic.T @ (W * (-sc.grav) * Kc * rho_lam)
    nb = sc.n + deg
    interior = np.zeros((nb,) * d, dtype=bool)
    interior[tuple([slice(1, -1)] * d)] = True
    idx = np.flatnonzero(interior.ravel())
    A = Smat.tocsr()[idx][:, idx].tocsc()
    sol = spla.splu(A).solve(F[idx])
    P = np.zeros(nb ** d)
    P[idx] = sol
    return P.reshape((nb,) * d)
