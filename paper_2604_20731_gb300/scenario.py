"""Seeded synthetic scenario generator.

This module only draws inputs: permeability fields, initial saturations,
source placements and initial network weights.  It contains none of the
solver's arithmetic (no basis functions, quadrature, residuals or updates), so
the CPU oracle and the CUDA path can both be fed from it without sharing any
of the method.

The paper's reservoir maps (its Sec. 8.1 porosity/permeability figures) are
not available, so a log-normal Gaussian random field stands in for them:
K = exp(sigma * Z), Z a zero-mean, unit-variance field with a Gaussian
correlation of length ``corr_len``.  Parameters are non-dimensional; the
viscosity and density ratios are those of the paper's parameter table
(Sec. 8.1): mu_w/mu_g = 25.35/3.95, rho_g/rho_w = 479/1045.

Array layout (shared by every consumer): row-major with x fastest, i.e.
2D arrays are [y][x] and 3D arrays are [z][y][x].
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Non-dimensional fluid parameters (ratios of the paper's Sec. 8.1 table).
MU_G = 1.0
MU_W = 25.35 / 3.95
RHO_W = 1.0
RHO_G = 479.0 / 1045.0
PHI = 0.2
SOURCE_SIGMA = 0.03  # ~ the paper's 3 m well radius in a 50 m domain, halved

SRC_INJECT = 0   # gas injector: q_g = rate * G
SRC_PRODUCE = 1  # producer: total rate split by fractional flow


@dataclasses.dataclass
class Source:
    center: Sequence[float]
    rate: float
    sigma: float = SOURCE_SIGMA
    kind: int = SRC_INJECT


@dataclasses.dataclass
class Scenario:
    """One reservoir scenario: grid, coefficients, sources and initial state."""

    dim: int
    n: int                      # elements per axis; collocation intervals N = n
    K: np.ndarray               # nodal permeability, (n+1)^dim, float64
    phi: float = PHI            # constant porosity ...
    phi_map: Optional[np.ndarray] = None  # ... or nodal porosity (n+1)^dim
    S0: Optional[np.ndarray] = None       # B-spline coefficients (n+p)^dim
    sources: List[Source] = dataclasses.field(default_factory=list)
    mu_w: float = MU_W
    mu_g: float = MU_G
    rho_w: float = RHO_W
    rho_g: float = RHO_G
    grav: float = 0.0
    grav_sign: float = 1.0      # +1: gravity term as derived from Eq. 2; -1: as printed in Eq. 9
    kz_ratio: float = 1.0       # 3D vertical/horizontal permeability ratio
    seed: int = 0
    p: int = 2                  # B-spline degree (the library implements p = 2)

    @property
    def nodes_shape(self):
        return (self.n + 1,) * self.dim

    @property
    def coeffs_shape(self):
        return (self.n + self.p,) * self.dim

    def S0_or_zero(self) -> np.ndarray:
        if self.S0 is None:
            return np.zeros(self.coeffs_shape)
        return self.S0


def gaussian_random_field(shape, corr_len, rng: np.random.Generator) -> np.ndarray:
    """Zero-mean unit-variance field on a grid of ``shape`` nodes over [0,1]^d.

    White noise on a padded periodic grid is convolved (by FFT) with a
    Gaussian kernel of correlation length ``corr_len`` (scalar or per axis),
    cropped and normalised.
    """
    dim = len(shape)
    if np.isscalar(corr_len):
        corr_len = (float(corr_len),) * dim
    h = [1.0 / max(s - 1, 1) for s in shape]
    pad = [int(math.ceil(3.0 * corr_len[a] / h[a])) for a in range(dim)]
    big = [shape[a] + 2 * pad[a] for a in range(dim)]
    noise = rng.standard_normal(big)
    # periodic Gaussian kernel centred at index 0
    grids = np.meshgrid(*[np.minimum(np.arange(big[a]), big[a] - np.arange(big[a])) * h[a]
                          for a in range(dim)], indexing="ij")
    arg = sum((g / corr_len[a]) ** 2 for a, g in enumerate(grids))
    kernel = np.exp(-0.5 * arg)
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * np.fft.fftn(kernel)))
    crop = tuple(slice(pad[a], pad[a] + shape[a]) for a in range(dim))
    z = field[crop]
    z = z - z.mean()
    sd = z.std()
    return z / sd if sd > 0 else z


def make_scenario(dim: int = 2, n: int = 32, seed: int = 1000, sigma: float = 1.0,
                  corr_len=0.1, rate: float = 1.0, grav: float = 0.0,
                  kz_ratio: float = 1.0, S0: str = "zero", p: int = 2) -> Scenario:
    """Scenario shaped like the configurations: log-normal K, injector at
    (0.25,...) and producer at (0.75,...), constant porosity 0.2.

    S0: "zero" (the configurations' initial state) or "random" (coefficients
    uniform in [0, 0.6], used by the parity tests so that every term is live).
    p: B-spline degree, n + p coefficients per axis.
    """
    rng = np.random.default_rng(seed)
    shape = (n + 1,) * dim
    if dim == 3 and np.isscalar(corr_len):
        corr_len = (0.02, 0.2, 0.2)  # [z][y][x]: layered along z
    Z = gaussian_random_field(shape, corr_len, rng)
    K = np.exp(sigma * Z)
    if S0 == "zero":
        s0 = np.zeros((n + p,) * dim)
    elif S0 == "random":
        s0 = rng.uniform(0.0, 0.6, size=(n + p,) * dim)
    else:
        raise ValueError(S0)
    inj = Source(center=(0.25,) * dim, rate=rate, kind=SRC_INJECT)
    prod = Source(center=(0.75,) * dim, rate=rate, kind=SRC_PRODUCE)
    return Scenario(dim=dim, n=n, K=K, S0=s0, sources=[inj, prod], grav=grav,
                    kz_ratio=kz_ratio, seed=seed, p=p)


def mlp_layer_sizes(in_dim: int, width: int, hidden_layers: int = 4) -> List[int]:
    return [in_dim] + [width] * hidden_layers + [1]


def mlp_num_params(in_dim: int, width: int, hidden_layers: int = 4) -> int:
    s = mlp_layer_sizes(in_dim, width, hidden_layers)
    return sum(s[i + 1] * s[i] + s[i + 1] for i in range(len(s) - 1))


def make_theta0(in_dim: int, width: int, hidden_layers: int = 4, seed: int = 7) -> np.ndarray:
    """Xavier-uniform initial weights, zero biases.

    Flat layout: for each layer l = 1..L+1 in order, W_l as [out][in]
    row-major followed by b_l[out].
    """
    rng = np.random.default_rng(seed)
    sizes = mlp_layer_sizes(in_dim, width, hidden_layers)
    parts = []
    for i in range(len(sizes) - 1):
        fan_in, fan_out = sizes[i], sizes[i + 1]
        a = math.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-a, a, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)


def make_map_image(shape, seed: int, corr_len=0.08, contrast: float = 40.0) -> np.ndarray:
    """A synthetic 8-bit grey picture standing in for the paper's reservoir
    maps (Sec. 8.1), which are not available: a Gaussian random field on the
    pixel grid, 128 + contrast * Z clipped to 0..255.  shape: (H, W) or
    (D, H, W); row 0 is the picture's top edge.  Decode it as
    offset + scale * pixel (e.g. porosity 0.05 + 0.35 * pixel / 255)."""
    rng = np.random.default_rng(seed)
    Z = gaussian_random_field(tuple(shape), corr_len, rng)
    return np.clip(np.rint(128.0 + contrast * Z), 0, 255).astype(np.uint8)
