"""Oracle: projection of the network pressure and the hybrid loop (Sec. 6).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 6, step 4 projects the nodal network pressure into the B-spline space by
an L2 projection.  Reading: the nodal values (boundary nodes 0) define the
piecewise-(bi/tri)linear interpolant on the knot grid, whose L2 projection is
(p, v) = (I_h u, v) for all B-spline test functions v, solved with the
Kronecker mass matrix.  Sec. 6, step 8 returns to step 5; the projection of
step 4 has to be repeated for the new pressure to reach the saturation update,
so each hybrid step is: project, 10 explicit saturation steps with that
pressure, recompute the collocation coefficients from the new saturation,
train the network (Adam) for a fixed number of iterations.
"""
from __future__ import annotations

import numpy as np

from .ads import AdsOracle, Mesh
from .crvpinn import Adam, CrvOracle, MLP, embed_interior
from .pressure import galerkin_pressure


def project_nodal(mesh: Mesh, nodal: np.ndarray) -> np.ndarray:
    Pq = mesh.nodal_at_gauss(nodal)
    F = mesh.test_value(mesh.gauss_weights() * Pq)
    return mesh.mass_solve_kron(F)


class HybridOracle:
    def __init__(self, sc, width: int, hidden_layers: int = 4):
        self.sc = sc
        self.ads = AdsOracle(sc)
        self.crv = CrvOracle(sc)
        self.mlp = MLP(sc.dim, width, hidden_layers)

    def nodal_pressure(self, theta) -> np.ndarray:
        u, _ = self.mlp.forward(theta, self.crv.X)
        return embed_interior(u, self.sc.dim, self.sc.n)

    def project(self, theta) -> np.ndarray:
        return project_nodal(self.ads.mesh, self.nodal_pressure(theta))

    def train(self, theta, adam: Adam, S, iters: int, lr: float):
        alpha, f = self.crv.coefficients(S)
        losses = []
        for _ in range(iters):
            loss, grad, _ = self.crv.loss_grad(self.mlp, theta, alpha, f)
            losses.append(loss)
            theta = adam.step(theta, grad, lr)
        return theta, losses

    def hybrid_step(self, S, theta, adam: Adam, n_sub: int, dt=None, adam_iters=100,
                    lr=1e-3, cfl=0.1, dt_cap=np.inf):
        P = self.project(theta)
        if dt is None:
            dt = self.ads.cfl_dt(P, cfl=cfl, dt_cap=dt_cap)
        for _ in range(n_sub):
            S = self.ads.step(S, P, dt)
        theta, losses = self.train(theta, adam, S, adam_iters, lr)
        return S, P, theta, dt, losses


def plain_step(sc, S, n_sub: int, dt=None, cfl=0.1, dt_cap=np.inf):
    """The IGA-ADS-MUMPS step of Sec. 7: direct Galerkin pressure, then n_sub
    explicit saturation steps with it."""
    ads = AdsOracle(sc)
    P = galerkin_pressure(sc, S)
    if dt is None:
        dt = ads.cfl_dt(P, cfl=cfl, dt_cap=dt_cap)
    for _ in range(n_sub):
        S = ads.step(S, P, dt)
    return S, P, dt
