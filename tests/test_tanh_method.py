"""Host-side check of the reciprocal the tensor-core forward computes on the FP32
pipe for part of its activations (tanh z = 2 / (1 + 2^z') - 1 with
z' = -2 log2(e) z).

The forward takes 1/d, d = 1 + 2^z' >= 1, as Newton-Raphson from an integer
guess: R - bits(d), read as a float, with R = 0x7EF311C0, then three steps
y <- y + y (1 - d y).  These tests emulate the method in numpy and check:
- the guess is within 5.1 % of 1/d over a whole binade, every mantissa
  (the relative error of a guess depends on the mantissa only);
- in exact arithmetic three steps leave an error far below FP32 rounding;
- in FP32 arithmetic without fused multiply-adds, a stricter rounding than
  the kernel's fused steps, the result is within a few units in the last
  place over d in [1, 2^64];
- the tanh built on it agrees with numpy's tanh to FP32 rounding.
"""
import numpy as np

R = 0x7EF311C0


def _seed(d32):
    bits = d32.view(np.uint32).astype(np.int64)
    return (np.int64(R) - bits).astype(np.uint32).view(np.float32)


def test_seed_error_over_a_binade():
    m = np.arange(0, 1 << 23, dtype=np.int64)
    d = ((127 << 23) + m).astype(np.uint32).view(np.float32)
    y = _seed(d).astype(np.float64)
    err = np.abs(d.astype(np.float64) * y - 1.0)
    assert err.max() <= 0.0506
    # a neighbouring constant is worse: the search picked a minimum
    y2 = (np.int64(R + (1 << 16)) - d.view(np.uint32).astype(np.int64)).astype(np.uint32).view(np.float32)
    assert np.abs(d.astype(np.float64) * y2.astype(np.float64) - 1.0).max() > err.max()


def test_three_newton_steps_exact_arithmetic():
    rng = np.random.default_rng(3)
    d = (1.0 + np.exp2(rng.uniform(-30.0, 64.0, size=200_000))).astype(np.float32)
    y = _seed(d).astype(np.float64)
    dd = d.astype(np.float64)
    errs = []
    for _ in range(3):
        y = y + y * (1.0 - dd * y)
        errs.append(np.abs(dd * y - 1.0).max())
    assert errs[0] <= 2.6e-3 and errs[1] <= 6.6e-6 and errs[2] <= 1e-10


def test_fp32_steps_within_a_few_ulp():
    rng = np.random.default_rng(4)
    d = (1.0 + np.exp2(rng.uniform(-30.0, 64.0, size=200_000))).astype(np.float32)
    d = np.concatenate([d, np.float32([1.0, 2.0, 1.5, np.float32(2.0) ** 64 + 1])])
    y = _seed(d)
    one = np.float32(1.0)
    for _ in range(3):
        e = (one - d * y).astype(np.float32)
        y = (y + y * e).astype(np.float32)
    exact = 1.0 / d.astype(np.float64)
    ulp = np.spacing(exact.astype(np.float32)).astype(np.float64)
    assert (np.abs(y.astype(np.float64) - exact) / ulp).max() <= 3.0


def test_tanh_on_the_fp32_pipe():
    z = np.linspace(-40.0, 40.0, 400_001)  # z < -22.2 meets the cap z' = 64
    zs = np.minimum((-2.0 * np.log2(np.e) * z).astype(np.float32), np.float32(64.0))
    d = (np.float32(1.0) + np.exp2(zs).astype(np.float32)).astype(np.float32)
    y = _seed(d)
    for _ in range(3):
        y = (y + y * (np.float32(1.0) - d * y)).astype(np.float32)
    t = (np.float32(2.0) * y - np.float32(1.0)).astype(np.float32)
    assert np.abs(t.astype(np.float64) - np.tanh(z)).max() <= 4e-7
    assert np.all(t[z > 10.0] == 1.0) and np.all(t[z < -10.0] == -1.0)
