"""Oracle: the CRVPINN pressure solver (Sec. 5) in float64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Collocation grid Omega_h = {(ih, jh)}, h = 1/N, N = n (Eq. 21); nodes coincide
with the B-spline knots.  Unknowns live on the interior nodes; the boundary
value is 0 (the space D_{0,h}).  Interior nodes are packed row-major with x
fastest ([y][x], or [z][y][x] in 3D).

Definitions restated here:
  * forward/backward differences (Eq. 22) and the discrete products
    (u,v)_h = h^2 sum u v and (u,v)_{grad,h} = sum_dir (D+u, D+v)_h;
  * nodal coefficient alpha = lambda(S) K and RHS = D+ . (g K rho lambda)
    - (q_w + q_g) at the nodes (Eq. 23b), with S clamped to [0,1] inside
    lambda;
  * residual RES_k = (alpha D+ u, D+ delta_k)_h + (RHS, delta_k)_h.  Eq. 24/25
    print a minus before the RHS term; with that sign a zero residual would
    solve div(alpha grad p) = -f, the opposite of Eq. 5, so the oracle uses
    the sign that makes RES = 0 the discrete form of Eq. 5;
  * Gram matrix G = h^-2 {4 on the diagonal, -1 for the four neighbours}
    (Eq. 26) on the interior nodes, loss RES^T G^-1 RES (Eq. 27) evaluated
    through an LU factorisation and two triangular solves (Eq. 28);
  * the network: inputs mapped from [0,1]^d to [-1,1]^d, tanh hidden layers,
    linear output; flat parameters [W_1, b_1, ..., W_{L+1}, b_{L+1}] with W_l
    stored [out][in] row-major;
  * dLOSS/du = 2 A G^-1 RES (A = the residual's linear part, symmetric), then
    ordinary back-propagation through the network;
  * Adam (Kingma & Ba) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8 and bias
    correction, as named in Sec. 8.3.
In 3D the same formulas are used with the 7-point neighbourhood (the paper is
2D only): G = h^-2 {6, -1}, the vertical difference weighted by kz_ratio, and
the 2D h^2 scaling kept.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .ads import along, gaussian_sources
from .bspline import basis_values, open_uniform_knots


# ----------------------------------------------------------------------------
# grid helpers
# ----------------------------------------------------------------------------

def interior_coords(dim: int, N: int) -> np.ndarray:
    """Coordinates of the interior nodes, shape (M, dim), columns (x, y[, z]),
    rows in packed order (x fastest)."""
    idx = np.arange(1, N) / N
    grids = np.meshgrid(*([idx] * dim), indexing="ij")  # axis 0 slowest
    cols = [g.ravel() for g in reversed(grids)]       # x first
    return np.stack(cols, axis=1)


def interior_slice(dim: int):
    return tuple([slice(1, -1)] * dim)


def embed_interior(u_int: np.ndarray, dim: int, N: int) -> np.ndarray:
    u = np.zeros((N + 1,) * dim)
    u[interior_slice(dim)] = u_int.reshape((N - 1,) * dim)
    return u


# ----------------------------------------------------------------------------
# network (Sec. 5: PINN(x_ij) replaces the pressure)
# ----------------------------------------------------------------------------

class MLP:
    def __init__(self, in_dim: int, width: int, hidden_layers: int = 4):
        self.sizes = [in_dim] + [width] * hidden_layers + [1]
        self.nparams = sum(self.sizes[i + 1] * self.sizes[i] + self.sizes[i + 1]
                           for i in range(len(self.sizes) - 1))

    def unpack(self, theta):
        out, o = [], 0
        for i in range(len(self.sizes) - 1):
            fi, fo = self.sizes[i], self.sizes[i + 1]
            W = theta[o:o + fo * fi].reshape(fo, fi); o += fo * fi
            b = theta[o:o + fo]; o += fo
            out.append((W, b))
        assert o == theta.size
        return out

    def forward(self, theta, X):
        """X in [0,1]^d, shape (P, d); returns u (P,) and the activations."""
        a = 2.0 * X - 1.0
        acts = [a]
        layers = self.unpack(theta)
        for l, (W, b) in enumerate(layers):
            z = a @ W.T + b
            a = np.tanh(z) if l < len(layers) - 1 else z
            acts.append(a)
        return a[:, 0], acts

    def backward(self, theta, acts, g):
        """Given dL/du per point, return dL/dtheta (flat)."""
        layers = self.unpack(theta)
        delta = g[:, None]
        grads = [None] * len(layers)
        for l in range(len(layers) - 1, -1, -1):
            W, _ = layers[l]
            grads[l] = (delta.T @ acts[l], delta.sum(axis=0))
            if l > 0:
                delta = (delta @ W) * (1.0 - acts[l] ** 2)
        return np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])


# ----------------------------------------------------------------------------
# the discrete pressure problem
# ----------------------------------------------------------------------------

class CrvOracle:
    def __init__(self, sc):
        self.sc = sc
        self.dim = sc.dim
        self.N = sc.n
        self.h = 1.0 / self.N
        self.M = (self.N - 1) ** self.dim
        self.K = np.asarray(sc.K, dtype=np.float64)
        nodes = np.arange(self.N + 1) / self.N
        deg = getattr(sc, "p", 2)
        self.Bnode = basis_values(open_uniform_knots(sc.n, deg), deg, nodes)
        grids = np.meshgrid(*([nodes] * self.dim), indexing="ij")
        self.node_coords = list(reversed(grids))
        self.X = interior_coords(self.dim, self.N)
        self._G_lu = None

    # ---- Eq. 23b ----
    def nodal_saturation(self, S: np.ndarray) -> np.ndarray:
        return along(S, [self.Bnode] * self.dim)

    def coefficients(self, S: np.ndarray):
        """alpha on all nodes and RHS on the interior nodes (Eq. 23b)."""
        sc = self.sc
        St = np.clip(self.nodal_saturation(S), 0.0, 1.0)
        lam_w = (1.0 - St) / sc.mu_w
        lam_g = St / sc.mu_g
        alpha = (lam_w + lam_g) * self.K
        # D+ . (g K rho lambda): g points down the vertical (array axis 0)
        Kv = self.K * (sc.kz_ratio if self.dim == 3 else 1.0)
        Fv = -sc.grav * Kv * (lam_w * sc.rho_w + lam_g * sc.rho_g)
        divF = (Fv[1:] - Fv[:-1]) / self.h          # forward difference, nodes 0..N-1
        q_inj, q_prod = gaussian_sources(sc, self.node_coords)
        rhs_full = np.zeros_like(alpha)
        rhs_full[:-1] = divF
        rhs_full = rhs_full - (q_inj - q_prod)
        f_int = rhs_full[interior_slice(self.dim)].ravel()
        return alpha, f_int

    # ---- residual operator A: RES = A u + h^2 f ----
    def operator(self, alpha: np.ndarray) -> sp.csr_matrix:
        """A = h^2 sum_dir D+^T diag(alpha) D+, restricted to the interior
        (the bilinear form (alpha D+ u, D+ delta_k)_h of Eq. 24)."""
        N, h, d = self.N, self.h, self.dim
        n1 = N + 1
        d1 = sp.diags([-np.ones(N), np.ones(N)], [0, 1], shape=(N, n1)) / h
        eye = sp.identity(n1, format="csr")
        A = None
        for a in range(d):  # array axis a
            mats = [d1 if b == a else eye for b in range(d)]
            D = mats[0]
            for mtx in mats[1:]:
                D = sp.kron(D, mtx)
            # alpha at the first node of each forward difference along axis a
            sl = [slice(None)] * d
            sl[a] = slice(0, N)
            coef = alpha[tuple(sl)]
            if d == 3 and a == 0:
                coef = coef * self.sc.kz_ratio
            term = D.T @ sp.diags(coef.ravel()) @ D
            A = term if A is None else A + term
        A = (h * h) * A
        interior = np.zeros((n1,) * d, dtype=bool)
        interior[interior_slice(d)] = True
        idx = np.flatnonzero(interior.ravel())
        return A.tocsr()[idx][:, idx].tocsr()

    def residual(self, alpha, f_int, u_int):
        return self.operator(alpha) @ u_int + self.h ** 2 * f_int

    # ---- Gram matrix (Eq. 26) and its inverse (Eq. 28) ----
    def gram(self) -> sp.csr_matrix:
        """h^-2 {2d on the diagonal, -1 for each interior neighbour}."""
        n = self.N - 1
        d = self.dim
        shape = (n,) * d
        M = self.M
        rows, cols, vals = [], [], []
        idx = np.arange(M).reshape(shape)
        rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(np.full(M, 2.0 * d))
        for a in range(d):
            sl_lo = [slice(None)] * d; sl_hi = [slice(None)] * d
            sl_lo[a] = slice(0, n - 1); sl_hi[a] = slice(1, n)
            lo = idx[tuple(sl_lo)].ravel(); hi = idx[tuple(sl_hi)].ravel()
            rows += [lo, hi]; cols += [hi, lo]; vals += [-np.ones(lo.size), -np.ones(lo.size)]
        G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(M, M))
        return G / self.h ** 2

    def gram_solve_lu(self, r: np.ndarray) -> np.ndarray:
        """q = G^-1 r by one LU factorisation and forward/back substitution
        (Eq. 28; the factorisation is kept for later calls)."""
        if self._G_lu is None:
            self._G_lu = spla.splu(self.gram().tocsc())
        return self._G_lu.solve(r)

    def gram_solve_fd(self, r: np.ndarray) -> np.ndarray:
        """q = G^-1 r by fast diagonalisation: G = h^-2 (T (+) T (+) ...) with
        T = tridiag(-1,2,-1) = S Lambda S, S_ik = sqrt(2/N) sin(pi i k/N).
        Sine transforms along every axis but the vertical one, then shifted
        tridiagonal solves along the vertical axis."""
        N, d, h = self.N, self.dim, self.h
        n = N - 1
        k = np.arange(1, N)
        S = np.sqrt(2.0 / N) * np.sin(np.pi * np.outer(k, k) / N)
        lam = 4.0 * np.sin(np.pi * k / (2.0 * N)) ** 2
        R = r.reshape((n,) * d)
        mats = [np.eye(n)] + [S] * (d - 1)
        Rh = along(R, mats)
        shift = np.zeros((n,) * (d - 1))
        for a in range(d - 1):
            shp = [1] * (d - 1); shp[a] = n
            shift = shift + lam.reshape(shp)
        flat_shift = shift.ravel()
        Rf = np.ascontiguousarray(Rh).reshape(n, -1)
        Zf = np.empty_like(Rf)
        for c in range(Rf.shape[1]):
            ab = np.zeros((3, n))
            ab[0, 1:] = -1.0
            ab[1, :] = 2.0 + flat_shift[c]
            ab[2, :-1] = -1.0
            Zf[:, c] = scipy.linalg.solve_banded((1, 1), ab, Rf[:, c])
        Z = along(Zf.reshape(Rh.shape), mats)
        return (h * h) * Z.ravel()

    # ---- loss, gradient ----
    def loss_grad(self, mlp: MLP, theta, alpha, f_int, with_grad=True, gram="lu"):
        u, acts = mlp.forward(theta, self.X)
        A = self.operator(alpha)
        r = A @ u + self.h ** 2 * f_int
        z = self.gram_solve_lu(r) if gram == "lu" else self.gram_solve_fd(r)
        loss = float(r @ z)
        if not with_grad:
            return loss, None, dict(u=u, r=r, z=z)
        g = 2.0 * (A @ z)
        grad = mlp.backward(theta, acts, g)
        return loss, grad, dict(u=u, r=r, z=z, g=g)

    def direct_solution(self, alpha, f_int) -> np.ndarray:
        """The unique zero-residual pressure u* (A u* = -h^2 f) by sparse LU."""
        A = self.operator(alpha)
        return spla.spsolve(A.tocsc(), -self.h ** 2 * f_int)


class Adam:
    """Adam with bias correction (Kingma & Ba), the optimiser of Sec. 8.3."""

    def __init__(self, nparams: int, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(nparams)
        self.v = np.zeros(nparams)
        self.t = 0
        self.b1, self.b2, self.eps = beta1, beta2, eps

    def step(self, theta, grad, lr):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        mhat = self.m / (1.0 - self.b1 ** self.t)
        vhat = self.v / (1.0 - self.b2 ** self.t)
        return theta - lr * mhat / (np.sqrt(vhat) + self.eps)
