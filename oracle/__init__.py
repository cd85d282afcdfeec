"""CPU FP64 oracle for the IGA-ADS + CRVPINN hybrid time step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method in float64 numpy/scipy, written to check the
CUDA path against.  Only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import it; the library's compute path never does, and the
two share no code.

Modules:
  bspline   -- knot vectors, Cox-de Boor basis values and derivatives, Gauss
               rules, 1D mass matrices                          (Sec. 4)
  ads       -- explicit saturation step: Galerkin RHS (Eq. 10a/10b), the
               Kronecker mass solve (Eq. 14), mass balance, CFL step size
  pressure  -- Galerkin pressure system (Eqs. 15-20, the direct-solver
               baseline of Sec. 7) and the discrete collocation pressure
               target (Eqs. 21-24) by sparse direct factorisation
  crvpinn   -- nodal coefficients (Eq. 23b), residual (Eq. 25), Gram matrix
               (Eq. 26), robust loss (Eqs. 27-28), MLP, adjoint gradient, Adam
  hybrid    -- projection of the network pressure (Sec. 6, step 4) and the
               hybrid loop (Sec. 6)
  maps      -- porosity and permeability maps given as images (Sec. 8.1),
               averaged over the nodes' dual cells

The spline degree follows the scenario (`p`, default 2: the quadratic C1
splines the configurations use): n + p functions per axis and p + 1 Gauss
points.  This is the general order-r, C^(r-1) basis of Eq. 11; the pins cover
p = 2, 3, 4.

Readings of the paper where it is silent or garbled are documented at each
function; the gravity sign, boundary conditions and residual sign follow the
derivation from Eqs. 1-5 (see each docstring).

Parity status: every function here is pinned by tests under tests/
(test_oracle_*.py) against closed forms, invariants, brute force or
independent library routes, except the multi-step saturation trajectory
beyond its invariants and the network training trajectory, which are
"parity unpinned" (no printed worked example exists in the paper).
"""
