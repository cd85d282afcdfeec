"""Porosity and permeability pictures brought onto the vertex grid
(ads_map_from_image) against the FP64 oracle of the same reading, through the
C ABI.

The oracle (oracle/maps.py) is pinned on the CPU (test_oracle_maps.py).  Here
the GPU must agree with it to FP64 rounding for pictures finer and coarser
than the mesh in ragged ratios, both pixel types, both means, both row
orders and in 3D; at the full 1024^2 mesh from a 4096^2 picture on sampled
nodes and through the integral the dual cells keep; and a saturation step fed
with the GPU's maps must match the oracle's step fed with the oracle's maps.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import maps as om

pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__ as g
    g.build()
    from paper_2604_20731_gb300 import _lib
    return _lib, _lib.load()


def _picture(shape, ptype, seed):
    rng = np.random.default_rng(seed)
    if ptype == "u8":
        return rng.integers(0, 256, shape).astype(np.uint8)
    return rng.uniform(0.05, 3.0, shape).astype(np.float32)


CASES = [
    # picture shape ([D,] H, W), n (x, y[, z]), pixel type, flip_y, mean, scale, offset
    ((5, 7), (4, 6), "f32", True, "arithmetic", 1.0, 0.0),
    ((64, 48), (33, 20), "f32", False, "geometric", 1.0, 0.0),
    ((17, 13), (40, 50), "u8", True, "arithmetic", 0.35 / 255, 0.05),
    ((300, 400), (128, 96), "u8", True, "geometric", 2.0 / 255, 0.2),
    ((1, 1), (3, 2), "f32", True, "arithmetic", 1.0, 0.0),
    ((1000, 3), (1, 1), "f32", True, "geometric", 1.0, 0.0),
    ((9, 10, 11), (6, 5, 4), "f32", True, "arithmetic", 1.0, 0.0),
    ((12, 7, 20), (5, 9, 3), "u8", False, "geometric", 1.0 / 255, 0.01),
]


@pytest.mark.parametrize("shape,n,ptype,flip_y,mean,scale,offset", CASES)
def test_map_matches_oracle(shape, n, ptype, flip_y, mean, scale, offset):
    torch = pytest.importorskip("torch")
    _, lib = _lib()
    from paper_2604_20731_gb300.solver import map_from_image
    img = _picture(shape, ptype, seed=sum(shape) + 31 * len(n))
    dev = torch.device("cuda", 0)
    got = map_from_image(torch.from_numpy(img).to(dev), n, flip_y=flip_y, mean=mean, scale=scale,
                         offset=offset).cpu().numpy()
    m = om.MEAN_GEOMETRIC if mean == "geometric" else om.MEAN_ARITHMETIC
    ref = om.image_to_nodal(img, n, flip_y=flip_y, mean=m, scale=scale, offset=offset)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-13


@pytest.mark.parametrize("mean", ["arithmetic", "geometric"])
def test_full_mesh_from_a_4096_picture(mean):
    """1024^2 elements from a 4096^2 8-bit picture: 4 pixels per element, the
    boundary cells half as wide.  Sampled nodes (corners, edges, random)
    against the oracle one by one; the arithmetic mean keeps the integral."""
    torch = pytest.importorskip("torch")
    _, lib = _lib()
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import map_from_image
    n = 1024
    img = scn.make_map_image((4096, 4096), seed=21)
    scale, offset = 0.35 / 255, 0.05
    dev = torch.device("cuda", 0)
    got = map_from_image(torch.from_numpy(img).to(dev), n, mean=mean, scale=scale, offset=offset)
    rng = np.random.default_rng(4)
    nodes = [(0, 0), (n, 0), (0, n), (n, n), (0, 517), (n, 3), (511, 0), (2, n)]
    nodes += [tuple(int(v) for v in rng.integers(0, n + 1, 2)) for _ in range(200)]
    m = om.MEAN_GEOMETRIC if mean == "geometric" else om.MEAN_ARITHMETIC
    ref = om.nodal_at(img, n, nodes, mean=m, scale=scale, offset=offset)
    g = got.cpu().numpy()
    sample = np.array([g[j, i] for i, j in nodes])
    assert np.max(np.abs(sample - ref) / np.abs(ref)) <= 1e-13
    if mean == "arithmetic":
        w = torch.full((n + 1,), 1.0 / n, dtype=torch.float64, device=dev)
        w[0] = w[-1] = 0.5 / n
        integral = float((got * w[:, None] * w[None, :]).sum())
        expect = offset + scale * float(img.astype(np.float64).mean())
        assert integral == pytest.approx(expect, rel=1e-13)


def test_non_finite_values_are_reported_and_the_rest_written():
    torch = pytest.importorskip("torch")
    L, lib = _lib()
    dev = torch.device("cuda", 0)
    img = torch.full((32, 32), 2.0, dtype=torch.float32, device=dev)
    img[31, 31] = -1.0                       # bottom-right pixel, seen only by the corner node
    out = torch.empty((9, 9), dtype=torch.float64, device=dev)
    shape = (C.c_int * 3)(32, 32, 0)
    n = (C.c_int * 3)(8, 8, 0)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.ads_map_from_image(img.data_ptr(), L.ADS_PIXEL_F32, 2, shape, 1, n, L.ADS_MAP_GEOMETRIC, 1.0, 0.0,
                                out.data_ptr(), st)
    assert rc == 4                            # ADS_ERR_NONFINITE
    o = out.cpu().numpy()
    assert np.isnan(o[0, 8])
    o[0, 8] = 2.0
    assert np.allclose(o, 2.0, rtol=1e-15, atol=0)
    # the arithmetic mean of the same picture is finite
    rc = lib.ads_map_from_image(img.data_ptr(), L.ADS_PIXEL_F32, 2, shape, 1, n, L.ADS_MAP_ARITHMETIC, 1.0, 0.0,
                                out.data_ptr(), st)
    assert rc == 0
    img[0, 0] = float("nan")
    rc = lib.ads_map_from_image(img.data_ptr(), L.ADS_PIXEL_F32, 2, shape, 1, n, L.ADS_MAP_ARITHMETIC, 1.0, 0.0,
                                out.data_ptr(), st)
    assert rc == 4
    assert np.isnan(out.cpu().numpy()[8, 0])  # row 0 of the picture is the top edge


def test_saturation_step_on_maps_given_as_pictures():
    """A permeability picture (geometric mean) and a porosity picture
    (arithmetic mean) at another resolution than the mesh: each side brings
    them onto the vertex grid itself, then one degree-2 step each."""
    torch = pytest.importorskip("torch")
    _, lib = _lib()
    from oracle.ads import AdsOracle
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import DegreePlan, map_from_image
    n = 40
    k_img = scn.make_map_image((150, 130), seed=5)
    p_img = scn.make_map_image((90, 110), seed=6, corr_len=0.15)
    k_dec, p_dec = (3.0 / 255, 0.1), (0.35 / 255, 0.05)
    sc = scn.make_scenario(2, n, seed=1011, S0="random")
    sc.K = om.image_to_nodal(k_img, n, mean=om.MEAN_GEOMETRIC, scale=k_dec[0], offset=k_dec[1])
    sc.phi_map = om.image_to_nodal(p_img, n, scale=p_dec[0], offset=p_dec[1])
    rng = np.random.default_rng(9)
    S = sc.S0
    P = rng.normal(size=(n + 2, n + 2))
    dt = 5e-4
    ref = AdsOracle(sc).step(S, P, dt)

    dev = torch.device("cuda", 0)
    K = map_from_image(torch.from_numpy(k_img).to(dev), n, mean="geometric", scale=k_dec[0], offset=k_dec[1])
    phi = map_from_image(torch.from_numpy(p_img).to(dev), n, scale=p_dec[0], offset=p_dec[1])
    plan = DegreePlan(sc, 2)
    try:
        Sd = torch.from_numpy(np.ascontiguousarray(S)).to(dev)
        Pd = torch.from_numpy(P).to(dev)
        out = torch.empty_like(Sd)
        st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        plan.step(K, phi, Sd, Pd, dt, out, st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    finally:
        plan.close()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
