"""Oracle: one explicit IGA-ADS saturation step (Secs. 2-4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The step is the isogeometric L2 projection of Sec. 4 (Eqs. 10b-13):

    (S_{n+1}, v) = (S_n, v) + tau * int( phi^-1 q_g v
                     - phi^-1 lambda_g(S_n) K (grad p_n + s rho_g g e_vert) . grad v )

for every tensor B-spline test function v, i.e. the weak form of Eq. 6
derived in Sec. 3 (Eqs. 7-10a).  Readings:
  * gravity sign: s = +1 follows from Eq. 2 with g pointing down (Sec. 3,
    before Eq. 9); s = -1 reproduces Eq. 9 as printed.  The scenario carries s.
  * phi is evaluated inside the integrand (it is a map in Sec. 6, step 1).
  * lambda_g = clamp(S,0,1)/mu_g; the coefficients S themselves are never
    clamped (the paper states no clamping; clamping only inside the mobility
    keeps the update exactly mass-conservative).
  * boundary: the full B-spline space, no degrees of freedom removed (the
    no-flux condition of Sec. 8.1), so the boundary term of Eq. 8 is dropped.
  * sources: normalised Gaussians; the producer's total rate is split into
    gas and water by the fractional flow f_g = lambda_g/(lambda_g+lambda_w).
  * K is the nodal map interpolated piecewise-(bi/tri)linearly; in 3D the
    vertical permeability is kz_ratio * K.

Fields at Gauss points are formed by applying the 1D collocation matrices of
oracle.bspline.Axis1D along each axis; the right-hand side is the transposed
application.  The mass matrix M = M_x (x) M_y (x) M_z (Eq. 14) is solved by
1D banded solves along each axis (the Kronecker route), and, for small
meshes, by a dense solve of the assembled Kronecker product.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .bspline import Axis1D


def along(arr: np.ndarray, mats) -> np.ndarray:
    """Apply mats[a] (shape rows x arr.shape[a]) along axis a, every axis."""
    out = arr
    for a, M in enumerate(mats):
        out = np.moveaxis(np.tensordot(M, out, axes=([1], [a])), 0, a)
    return out


class Mesh:
    """Tensor mesh of `dim` identical axes (array axis 0 is the vertical)."""

    def __init__(self, dim: int, n: int, p: int = 2):
        self.dim, self.n, self.p = dim, n, p
        self.ax = Axis1D(n, p)
        self.h = 1.0 / n

    def gauss_weights(self) -> np.ndarray:
        w = self.ax.w
        out = w
        for _ in range(self.dim - 1):
            out = np.multiply.outer(w, out)
        return out

    def gauss_coords(self):
        """Coordinates of the Gauss points; returns [x, y(, z)] arrays shaped
        like the Gauss grid ([y][x] or [z][y][x])."""
        grids = np.meshgrid(*([self.ax.x] * self.dim), indexing="ij")
        return list(reversed(grids))  # array axis a holds coordinate dim-1-a

    def at_gauss(self, coeffs: np.ndarray) -> np.ndarray:
        return along(coeffs, [self.ax.B] * self.dim)

    def grad_at_gauss(self, coeffs: np.ndarray):
        """[d/dx, d/dy(, d/dz)] of the spline at Gauss points."""
        out = []
        for c in range(self.dim):
            a = self.dim - 1 - c
            mats = [self.ax.dB if b == a else self.ax.B for b in range(self.dim)]
            out.append(along(coeffs, mats))
        return out

    def nodal_at_gauss(self, nodal: np.ndarray) -> np.ndarray:
        return along(nodal, [self.ax.H] * self.dim)

    def test_value(self, c: np.ndarray) -> np.ndarray:
        """sum_q c_q v_k(x_q) for every tensor test function v_k."""
        return along(c, [self.ax.B.T] * self.dim)

    def test_grad(self, cvec) -> np.ndarray:
        """sum_q c_q . grad v_k(x_q); cvec = [c_x, c_y(, c_z)]."""
        out = 0.0
        for c in range(self.dim):
            a = self.dim - 1 - c
            mats = [self.ax.dB.T if b == a else self.ax.B.T for b in range(self.dim)]
            out = out + along(cvec[c], mats)
        return out

    # ---- Kronecker mass solve (Eq. 14) ----
    def mass_solve_kron(self, R: np.ndarray) -> np.ndarray:
        M = self.ax.M
        p = self.p
        nb = M.shape[0]
        ab = np.zeros((2 * p + 1, nb))
        for k in range(-p, p + 1):
            diag = np.diagonal(M, k)
            if k >= 0:
                ab[p - k, k:] = diag
            else:
                ab[p - k, :nb + k] = diag
        X = R
        for a in range(self.dim):
            Xa = np.moveaxis(X, a, 0)
            shp = Xa.shape
            Xa = scipy.linalg.solve_banded((p, p), ab, Xa.reshape(nb, -1))
            X = np.moveaxis(Xa.reshape(shp), 0, a)
        return X

    def mass_dense(self) -> np.ndarray:
        M = self.ax.M
        out = M
        for _ in range(self.dim - 1):
            out = np.kron(M, out)  # axis 0 slowest
        return out

    def mass_solve_dense(self, R: np.ndarray) -> np.ndarray:
        return np.linalg.solve(self.mass_dense(), R.ravel()).reshape(R.shape)

    def integral(self, coeffs: np.ndarray) -> float:
        return float(np.sum(self.gauss_weights() * self.at_gauss(coeffs)))


def gaussian_sources(sc, coords):
    """Injected gas rate q_inj and produced total rate q_prod (both >= 0) at
    the given points; G_c(x) = exp(-|x-c|^2/(2 s^2)) / (2 pi s^2)^(d/2)."""
    q_inj = np.zeros_like(coords[0])
    q_prod = np.zeros_like(coords[0])
    d = sc.dim
    for s in sc.sources:
        r2 = sum((coords[c] - s.center[c]) ** 2 for c in range(d))
        G = np.exp(-r2 / (2.0 * s.sigma ** 2)) / (2.0 * np.pi * s.sigma ** 2) ** (d / 2.0)
        if s.kind == 0:
            q_inj = q_inj + s.rate * G
        else:
            q_prod = q_prod + s.rate * G
    return q_inj, q_prod


def mobilities(sc, S):
    St = np.clip(S, 0.0, 1.0)
    lam_g = St / sc.mu_g
    lam_w = (1.0 - St) / sc.mu_w
    return lam_g, lam_w


def gas_source(sc, S, coords):
    """q_g: injection minus the gas share f_g of production."""
    q_inj, q_prod = gaussian_sources(sc, coords)
    lam_g, lam_w = mobilities(sc, S)
    f_g = lam_g / (lam_g + lam_w)
    return q_inj - f_g * q_prod


class AdsOracle:
    """The explicit saturation step of Eq. 6 in the weak form of Eq. 10a/10b."""

    def __init__(self, sc):
        self.sc = sc
        self.mesh = Mesh(sc.dim, sc.n, getattr(sc, "p", 2))
        m = self.mesh
        self.W = m.gauss_weights()
        self.coords = m.gauss_coords()
        self.Kq = m.nodal_at_gauss(np.asarray(sc.K, dtype=np.float64))
        if sc.phi_map is not None:
            self.phiq = m.nodal_at_gauss(np.asarray(sc.phi_map, dtype=np.float64))
        else:
            self.phiq = np.full_like(self.Kq, float(sc.phi))

    def darcy_term(self, P: np.ndarray):
        """K (grad p + s rho_g g e_vert) at Gauss points, per coordinate."""
        sc, d = self.sc, self.sc.dim
        gp = self.mesh.grad_at_gauss(P)
        out = []
        for c in range(d):
            Kc = self.Kq * (sc.kz_ratio if (d == 3 and c == d - 1) else 1.0)
            term = gp[c]
            if c == d - 1:
                term = term + sc.grav_sign * sc.rho_g * sc.grav
            out.append(Kc * term)
        return out

    def rhs(self, S: np.ndarray, P: np.ndarray, dt: float) -> np.ndarray:
        sc = self.sc
        m = self.mesh
        Sq = m.at_gauss(S)
        lam_g, _ = mobilities(sc, Sq)
        q_g = gas_source(sc, Sq, self.coords)
        c0 = self.W * (Sq + dt / self.phiq * q_g)
        flux = self.darcy_term(P)
        cvec = [-self.W * dt / self.phiq * lam_g * f for f in flux]
        return m.test_value(c0) + m.test_grad(cvec)

    def step(self, S: np.ndarray, P: np.ndarray, dt: float, dense: bool = False):
        R = self.rhs(S, P, dt)
        Snew = self.mesh.mass_solve_dense(R) if dense else self.mesh.mass_solve_kron(R)
        return Snew

    def source_integral(self, S: np.ndarray, dt: float) -> float:
        """tau * int q_g / phi, by the same quadrature."""
        Sq = self.mesh.at_gauss(S)
        q_g = gas_source(self.sc, Sq, self.coords)
        return float(dt * np.sum(self.W * q_g / self.phiq))

    def mass_error(self, S_old, S_new, dt) -> float:
        """int S_{n+1} - int S_n - tau int q_g/phi (zero for an exact step)."""
        return (self.mesh.integral(S_new) - self.mesh.integral(S_old)
                - self.source_integral(S_old, dt))

    def cfl_dt(self, P: np.ndarray, cfl: float = 0.1, src_frac: float = 0.05,
               dt_cap: float = np.inf) -> float:
        """Step size: min(C h / v_max, src_frac / s_max, dt_cap) with
        v_max = max_q |K (grad p + s rho_g g e)| / (mu_g phi) and
        s_max = max_q q_inj / phi (the paper fixes tau; this rule is the
        reading used for the CFL-limited configurations)."""
        sc = self.sc
        flux = self.darcy_term(P)
        vmag = np.sqrt(sum(f * f for f in flux)) / (sc.mu_g * self.phiq)
        vmax = float(vmag.max())
        q_inj, _ = gaussian_sources(sc, self.coords)
        smax = float((q_inj / self.phiq).max())
        dt = dt_cap
        if vmax > 0:
            dt = min(dt, cfl * self.mesh.h / vmax)
        if smax > 0:
            dt = min(dt, src_frac / smax)
        return dt
