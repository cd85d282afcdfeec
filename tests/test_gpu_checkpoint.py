"""Checkpoint / resume (ads_save, ads_load): a context restored from a
checkpoint continues bit for bit as the saved one; files of another shape or
format are refused.  Needs a GPU."""
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


def _hp(adam_iters=20):
    from paper_2604_20731_gb300.solver import HybridSolver
    return HybridSolver.hybrid_params(n_sub=3, dt=1.0, dt_policy=1, cfl=0.1, src_frac=0.05,
                                      adam_iters=adam_iters, lr=1e-3)


@pytest.mark.parametrize("crv_dtype,ads_dtype,phi_map", [("bf16", "f32", False), ("f64", "f64", True)])
def test_resume_continues_bit_for_bit(tmp_path, crv_dtype, ads_dtype, phi_map):
    n = 32
    sc = scn.make_scenario(2, n, seed=11, S0="random")
    if phi_map:
        sc.phi_map = 0.1 + 0.3 * np.random.default_rng(5).uniform(size=(n + 1, n + 1))
    theta0 = scn.make_theta0(2, 64, 4, seed=7)
    hp = _hp()
    a = _solver(sc, width=64, crv_dtype=crv_dtype, ads_dtype=ads_dtype)
    a.set_theta(theta0)
    a.pretrain(20, 1e-3)
    a.hybrid_step(hp)  # (one step: Adam moments, step counter and the S buffer parity move)
    path = tmp_path / "ck.bin"
    a.save(path)
    a.hybrid_step(hp)
    ref = {f: a.get(f) for f in ("S", "P", "THETA", "U", "DT", "MASS", "LOSS")}
    a.close()

    b = _solver(sc, width=64, crv_dtype=crv_dtype, ads_dtype=ads_dtype)
    b.load(path)
    b.hybrid_step(hp)
    for f, v in ref.items():
        assert np.array_equal(b.get(f), v), f
    b.close()


def test_saturation_only_context_resumes(tmp_path):
    n = 24
    sc = scn.make_scenario(2, n, seed=3, S0="random")
    P = np.random.default_rng(1).normal(size=(n + 2, n + 2))
    a = _solver(sc, width=None, ads_dtype="f64")
    a.set_pressure(P)
    a.saturation_step(1e-4, 2)
    path = tmp_path / "sat.bin"
    a.save(path)
    a.saturation_step(1e-4, 3)
    S_ref = a.get("S")
    a.close()
    b = _solver(sc, width=None, ads_dtype="f64")
    b.load(path)
    b.saturation_step(1e-4, 3)
    assert np.array_equal(b.get("S"), S_ref)
    b.close()


def test_checkpoint_of_another_shape_or_format_is_refused(tmp_path):
    from paper_2604_20731_gb300._lib import AdsError
    sc = scn.make_scenario(2, 32, seed=11)
    a = _solver(sc, width=64, crv_dtype="f32", ads_dtype="f32")
    path = tmp_path / "ck.bin"
    a.save(path)
    for other in (_solver(scn.make_scenario(2, 16, seed=11), width=64, crv_dtype="f32", ads_dtype="f32"),
                  _solver(sc, width=128, crv_dtype="bf16", ads_dtype="f32"),
                  _solver(sc, width=None, ads_dtype="f32")):
        with pytest.raises(AdsError):
            other.load(path)
        other.close()
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NOTACKPT" + bytes(64))
    with pytest.raises(AdsError):
        a.load(bad)
    with pytest.raises(AdsError):
        a.load(tmp_path / "missing.bin")
    # a truncated file: short read
    trunc = tmp_path / "trunc.bin"
    trunc.write_bytes(path.read_bytes()[:100])
    with pytest.raises(AdsError):
        a.load(trunc)
    a.close()
