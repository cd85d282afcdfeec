"""GB300-native hybrid IGA-ADS + CRVPINN time step (CO2 sequestration).

The compute path is the C-ABI CUDA library libadsgb.so (include/adsgb.h);
this package holds its Python binding (`solver`), the seeded scenario
generator (`scenario`) and the in-tree build (`build`).  Importing the
package does not load the library; the first solver does, and fails loudly if
it is missing.
"""
from . import scenario  # noqa: F401

__all__ = ["scenario", "HybridSolver", "hybrid_step_batch"]


def __getattr__(name):
    if name in ("HybridSolver", "hybrid_step_batch"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
