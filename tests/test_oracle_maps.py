"""Pins of the image-map oracle (porosity and permeability pictures, Sec. 8.1).

Each pin is independent of the oracle's overlap arithmetic: constants, the
integral the dual cells keep, linear fields whose dual-cell averages are known
in closed form, the orientation of a single bright pixel, and brute force over
a fine grid of equal sub-cells, each inside one pixel and one dual cell.
"""
import math

import numpy as np
import pytest

from oracle import maps


def brute(img, n, flip_y=True, mean=maps.MEAN_ARITHMETIC):
    """Average over a grid of equal sub-cells, lcm(2 n_a, pixels) per axis.
    A sub-cell's midpoint (2k+1)/(2L) lies in pixel floor((2k+1) m / 2L) and
    in the dual cell of node floor(((2k+1) n + L) / 2L)."""
    v = np.asarray(img, dtype=np.float64)
    if flip_y:
        v = v[..., ::-1, :]
    dim = v.ndim
    ns = (n,) * dim if np.isscalar(n) else tuple(n)
    pix, node = [], []
    for ax in range(dim):
        m = v.shape[dim - 1 - ax]
        L = math.lcm(2 * ns[ax], m)
        k = np.arange(L)
        pix.append(((2 * k + 1) * m) // (2 * L))
        node.append(((2 * k + 1) * ns[ax] + L) // (2 * L))
    if dim == 2:
        vals = v[np.ix_(pix[1], pix[0])]
        ids = node[1][:, None] * (ns[0] + 1) + node[0][None, :]
        shape = (ns[1] + 1, ns[0] + 1)
    else:
        vals = v[np.ix_(pix[2], pix[1], pix[0])]
        ids = ((node[2][:, None, None] * (ns[1] + 1) + node[1][None, :, None]) * (ns[0] + 1)
               + node[0][None, None, :])
        shape = (ns[2] + 1, ns[1] + 1, ns[0] + 1)
    if mean == maps.MEAN_GEOMETRIC:
        vals = np.log(vals)
    tot = np.bincount(ids.ravel(), weights=vals.ravel(), minlength=int(np.prod(shape)))
    cnt = np.bincount(ids.ravel(), minlength=int(np.prod(shape)))
    out = (tot / cnt).reshape(shape)
    return np.exp(out) if mean == maps.MEAN_GEOMETRIC else out


@pytest.mark.parametrize("mean", [maps.MEAN_ARITHMETIC, maps.MEAN_GEOMETRIC])
def test_constant_image_gives_constant_nodes(mean):
    out = maps.image_to_nodal(np.full((9, 13), 0.37), (5, 7), mean=mean)
    assert out.shape == (8, 6)
    assert np.allclose(out, 0.37, rtol=1e-15, atol=0)
    out3 = maps.image_to_nodal(np.full((3, 4, 5), 2.5), (2, 3, 4), mean=mean)
    assert out3.shape == (5, 4, 3)
    assert np.allclose(out3, 2.5, rtol=1e-15, atol=0)


@pytest.mark.parametrize("shape,n", [((5, 7), (4, 6)), ((13, 11), (3, 3)), ((4, 4), (9, 10)),
                                     ((3, 5, 7), (2, 3, 4)), ((6, 2, 3), (4, 5, 3))])
def test_arithmetic_average_keeps_the_integral(shape, n):
    """The dual cells tile the domain: sum(value x cell volume) is the image's
    mean, whether the picture is finer or coarser than the mesh."""
    img = np.random.default_rng(3).uniform(0.0, 1.0, shape)
    out = maps.image_to_nodal(img, n)
    vol = 1.0
    for ax, na in enumerate(n):
        w = np.full(na + 1, 1.0 / na)
        w[0] = w[-1] = 0.5 / na
        vol = np.multiply.outer(w, vol) if ax else w
    assert abs((out * vol).sum() - img.mean()) <= 1e-15 * 8


def test_linear_field_gives_its_value_at_the_dual_cell_centroid():
    """Pixels of width h/2k hold the pixel-average of f = a + b x + c y, and
    the dual cells are unions of whole pixels, so the node value is f at the
    cell's centroid: the node itself, h/4 inside the edge at the boundary."""
    nx, ny, kx, ky = 4, 6, 3, 2
    W, H = 2 * nx * kx, 2 * ny * ky
    a, b, c = 0.3, 1.7, -0.9
    xc = (np.arange(W) + 0.5) / W
    yc = 1.0 - (np.arange(H) + 0.5) / H          # row 0 at the top
    img = a + b * xc[None, :] + c * yc[:, None]
    out = maps.image_to_nodal(img, (nx, ny))

    def centroid(na):
        t = np.arange(na + 1) / na
        t[0], t[-1] = 0.25 / na, 1.0 - 0.25 / na
        return t

    ref = a + b * centroid(nx)[None, :] + c * centroid(ny)[:, None]
    assert np.max(np.abs(out - ref)) <= 1e-14
    # geometric mean of exp(f): exp(f at the centroid), the same argument in log space
    outg = maps.image_to_nodal(np.exp(img), (nx, ny), mean=maps.MEAN_GEOMETRIC)
    assert np.max(np.abs(np.log(outg) - ref)) <= 1e-14


def test_linear_field_3d():
    nx, ny, nz = 2, 3, 4
    W, H, D = 2 * nx * 2, 2 * ny, 2 * nz * 3
    xc = (np.arange(W) + 0.5) / W
    yc = (np.arange(H) + 0.5) / H               # row 0 at the bottom (flip_y False)
    zc = (np.arange(D) + 0.5) / D
    img = (0.5 + 2.0 * xc[None, None, :] - 1.0 * yc[None, :, None] + 3.0 * zc[:, None, None])
    out = maps.image_to_nodal(img, (nx, ny, nz), flip_y=False)

    def centroid(na):
        t = np.arange(na + 1) / na
        t[0], t[-1] = 0.25 / na, 1.0 - 0.25 / na
        return t

    ref = (0.5 + 2.0 * centroid(nx)[None, None, :] - 1.0 * centroid(ny)[None, :, None]
           + 3.0 * centroid(nz)[:, None, None])
    assert np.max(np.abs(out - ref)) <= 1e-14


@pytest.mark.parametrize("flip_y", [True, False])
def test_orientation_of_a_bright_corner_pixel(flip_y):
    """Pixel (row 0, column 0) is the top-left corner of a picture (flip_y) or
    the bottom-left corner of a bottom-up array."""
    img = np.zeros((8, 8))
    img[0, 0] = 1.0
    out = maps.image_to_nodal(img, 4, flip_y=flip_y)
    hot = np.argwhere(out > 0)
    assert hot.tolist() == ([[4, 0]] if flip_y else [[0, 0]])   # [y][x]
    assert out[tuple(hot[0])] == 1.0      # the corner node's cell is that pixel alone


@pytest.mark.parametrize("shape,n,flip_y,mean", [
    ((5, 7), (4, 6), True, maps.MEAN_ARITHMETIC),
    ((7, 5), (6, 4), False, maps.MEAN_ARITHMETIC),
    ((3, 2), (5, 7), True, maps.MEAN_GEOMETRIC),
    ((11, 9), (4, 3), True, maps.MEAN_GEOMETRIC),
    ((3, 5, 4), (2, 3, 5), True, maps.MEAN_ARITHMETIC),
    ((4, 3, 5), (3, 2, 2), False, maps.MEAN_GEOMETRIC),
])
def test_brute_force_over_equal_sub_cells(shape, n, flip_y, mean):
    img = np.random.default_rng(11).uniform(0.05, 2.0, shape)
    out = maps.image_to_nodal(img, n, flip_y=flip_y, mean=mean)
    ref = brute(img, n, flip_y=flip_y, mean=mean)
    assert np.max(np.abs(out - ref) / np.abs(ref)) <= 1e-13


def test_nodes_one_at_a_time_and_pixel_scaling():
    img = np.random.default_rng(5).integers(0, 256, (6, 10)).astype(np.uint8)
    full = maps.image_to_nodal(img, (7, 5), scale=0.5, offset=2.0)
    ref = 2.0 + 0.5 * brute(img, (7, 5))
    assert np.max(np.abs(full - ref)) <= 1e-12
    nodes = [(0, 0), (7, 5), (3, 2), (6, 1)]
    one = maps.nodal_at(img, (7, 5), nodes, scale=0.5, offset=2.0)
    assert np.array_equal(one, np.array([full[j, i] for i, j in nodes]))


def test_a_zero_pixel_makes_the_geometric_mean_zero_only_where_it_is_seen():
    img = np.full((8, 8), 2.0)
    img[7, 7] = 0.0                        # bottom-right corner of the picture
    out = maps.image_to_nodal(img, 4, mean=maps.MEAN_GEOMETRIC)
    assert out[0, 4] == 0.0
    mask = np.ones_like(out, dtype=bool)
    mask[0, 4] = False
    assert np.allclose(out[mask], 2.0, rtol=1e-15, atol=0)
