"""ads_init_with_allocator: the context's buffers come from the caller's
allocator (here PyTorch's caching allocator), results are the same as with
the library's own allocations, every block goes back, and misaligned or
missing memory is refused.  Needs a GPU."""
import numpy as np
import pytest

from paper_2604_20731_gb300 import scenario as scn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _solver(sc, **kw):
    from paper_2604_20731_gb300.solver import HybridSolver
    return HybridSolver(sc, **kw)


def test_caller_allocator_same_results_and_every_block_returned():
    import torch
    from paper_2604_20731_gb300.solver import HybridSolver
    live = {}

    def alloc(nbytes):
        p = torch.cuda.caching_allocator_alloc(nbytes)
        live[p] = nbytes
        return p

    def free(p):
        torch.cuda.caching_allocator_delete(p)
        live.pop(p)

    sc = scn.make_scenario(2, 64, seed=5, S0="random")
    theta = scn.make_theta0(2, 64, 4, seed=7)
    hp = HybridSolver.hybrid_params(n_sub=3, dt=1.0, dt_policy=1, cfl=0.1, src_frac=0.05,
                                    adam_iters=20, lr=1e-3)
    a = _solver(sc, width=64, crv_dtype="bf16", ads_dtype="f32", allocator=(alloc, free))
    assert len(live) > 20
    b = _solver(sc, width=64, crv_dtype="bf16", ads_dtype="f32")
    for s in (a, b):
        s.set_theta(theta)
        s.pretrain(10, 1e-3)
        s.hybrid_step(hp)
    for f in ("S", "P", "THETA", "U", "DT"):
        assert np.array_equal(a.get(f), b.get(f)), f
    a.close()
    b.close()
    assert not live


def test_misaligned_or_missing_memory_is_refused():
    import torch
    from paper_2604_20731_gb300._lib import AdsError
    sc = scn.make_scenario(2, 32, seed=5)
    base = {}

    def bad_alloc(nbytes):
        p = torch.cuda.caching_allocator_alloc(nbytes + 512)
        base[p + 16] = p
        return p + 16

    def bad_free(p):
        torch.cuda.caching_allocator_delete(base.pop(p))

    with pytest.raises(AdsError):
        _solver(sc, width=None, ads_dtype="f32", allocator=(bad_alloc, bad_free))
    assert not base
    with pytest.raises(AdsError):
        _solver(sc, width=None, ads_dtype="f32", allocator=(lambda n: 0, lambda p: None))
