"""Oracle: porosity and permeability given as images (Sec. 8.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 8.1 gives the porosity (values 0 to 1) and the permeability (mDarcy,
used in SI units, 1 mDarcy ~ 1e-15 m^2) of each reservoir as a picture of the
domain.  The method reads K and phi as nodal values on the (n+1)^d vertex
grid (bi/trilinear at the Gauss points, the nodal value itself for the
collocation coefficient of Eq. 23b), so a map given as an image has to be
brought onto that grid.

Reading (the paper does not say how the pictures were sampled):
  * The image is a piecewise-constant field: pixel (row r, column c) of an
    H x W image holds one value over the square x in [c/W, (c+1)/W],
    y in [1 - (r+1)/H, 1 - r/H] when row 0 is the top edge of the picture
    (flip_y, the usual image convention), or y in [r/H, (r+1)/H] when row 0
    is the bottom edge.  3D maps are stacks of such images, slice s over
    z in [s/D, (s+1)/D].
  * A pixel value v becomes the physical value offset + scale * v.
  * The nodal value at vertex x_i = i/n is the average of the field over the
    node's dual cell, [x_i - h/2, x_i + h/2] per axis (clipped to [0, 1] at
    the boundary nodes): the arithmetic mean, or the geometric mean
    exp(avg log) often used to upscale log-normal permeability.  The dual
    cells tile the domain, so the arithmetic form keeps the integral of the
    map, and it works the same when the image is finer or coarser than the
    mesh.

The overlaps of dual cells and pixels are computed exactly: in units of
1/(2 n W) every endpoint is an integer, (2i -+ 1) W for the dual cell and
2 n c for the pixel.
"""
from __future__ import annotations

import numpy as np

MEAN_ARITHMETIC = 0
MEAN_GEOMETRIC = 1


def dual_overlap(n: int, m: int) -> np.ndarray:
    """(n+1) x m matrix of overlap lengths, in units of 1/(2 n m), between the
    dual cell of node i (of n elements on [0, 1]) and pixel c (of m pixels)."""
    lo = np.clip((2 * np.arange(n + 1) - 1) * m, 0, 2 * n * m)
    hi = np.clip((2 * np.arange(n + 1) + 1) * m, 0, 2 * n * m)
    c_lo = 2 * n * np.arange(m)
    c_hi = 2 * n * (np.arange(m) + 1)
    A = np.minimum(hi[:, None], c_hi[None, :]) - np.maximum(lo[:, None], c_lo[None, :])
    return np.maximum(A, 0).astype(np.int64)


def _prepare(img, n, flip_y, scale, offset):
    a = np.asarray(img, dtype=np.float64)
    dim = a.ndim
    if dim not in (2, 3):
        raise ValueError("image must be 2D or 3D")
    ns = (int(n),) * dim if np.isscalar(n) else tuple(int(v) for v in n)
    if len(ns) != dim:
        raise ValueError("one element count per axis")
    v = offset + scale * a
    if flip_y:
        v = v[..., ::-1, :]        # the row index now grows with y
    # overlaps per axis, x first: (n_a + 1) x (pixels along axis a)
    A = [dual_overlap(ns[ax], v.shape[dim - 1 - ax]) for ax in range(dim)]
    return v, ns, A


def _node_value(v, A, idx, mean):
    """Average of the field over the dual cell of node idx (x, y(, z)):
    only the pixels the cell overlaps enter, weighted by the overlap."""
    sel = [np.nonzero(A[ax][idx[ax]])[0] for ax in range(len(idx))]
    w = A[0][idx[0]][sel[0]].astype(np.float64)
    for ax in range(1, len(idx)):
        w = np.multiply.outer(A[ax][idx[ax]][sel[ax]].astype(np.float64), w)
    block = v[np.ix_(*sel[::-1])]  # [z][y][x] sub-block
    if mean == MEAN_ARITHMETIC:
        return float((w * block).sum() / w.sum())
    if mean == MEAN_GEOMETRIC:
        with np.errstate(divide="ignore", invalid="ignore"):
            return float(np.exp((w * np.log(block)).sum() / w.sum()))
    raise ValueError("mean")


def image_to_nodal(img, n, flip_y: bool = True, mean: int = MEAN_ARITHMETIC,
                   scale: float = 1.0, offset: float = 0.0) -> np.ndarray:
    """Nodal values of an image map.

    img: (H, W) for 2D or (D, H, W) for 3D (rows of a slice along y, columns
    along x), any numeric dtype.  n: elements per axis, an int or one per
    axis in x, y(, z) order.  Returns [y][x] (or [z][y][x]) float64 with
    n_a + 1 nodes along axis a.
    """
    v, ns, A = _prepare(img, n, flip_y, scale, offset)
    out = np.empty(tuple(m + 1 for m in ns[::-1]))
    for idx in np.ndindex(*out.shape):
        out[idx] = _node_value(v, A, idx[::-1], mean)
    return out


def nodal_at(img, n, nodes, flip_y: bool = True, mean: int = MEAN_ARITHMETIC,
             scale: float = 1.0, offset: float = 0.0) -> np.ndarray:
    """The nodal values at a list of nodes, each (i, j(, k)) in x, y(, z)
    order: the same definition, one node at a time, for large maps."""
    v, ns, A = _prepare(img, n, flip_y, scale, offset)
    return np.array([_node_value(v, A, tuple(int(t) for t in nd), mean) for nd in nodes])
