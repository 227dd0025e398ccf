"""The arithmetic behind the tensor-core sampler's error bound, checked on the CPU: a float
x is split into two TF32 numbers hi = rn(x), lo = rn(x - hi) (rn: round to nearest, ties
away from zero, to 10 explicit mantissa bits, as cvt.rna.tf32.f32 does), and a product
x y is formed as hi_x hi_y + hi_x lo_y + lo_x hi_y. The GPU parity test charges each such
product 12 u (u = 2^-24) of |x y|: the split leaves a rest below 2^-22 |x|, and the dropped
and rest terms total at most 3 * 2^-22 |x y|. Here TF32 rounding is emulated exactly on the
float32 bit patterns and both statements are checked on many random and edge values, and a
plain single TF32 product is shown to miss the bound (so the split is what keeps FP32
accuracy)."""
import numpy as np

U = 2.0 ** -24


def tf32_rna(x):
    """x (float32) rounded to TF32, ties away from zero: add half of the dropped 13-bit
    field's unit to the magnitude bits and clear the field (sign-magnitude, so one integer
    addition serves both signs; finite inputs far below the overflow threshold)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    sign = b & np.uint32(0x80000000)
    mag = b & np.uint32(0x7FFFFFFF)
    mag = (mag + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return (sign | mag).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = tf32_rna(x)
    lo = tf32_rna((x - hi).astype(np.float32))   # x - hi is exact in float32
    return hi, lo


def _values(n, seed):
    g = np.random.default_rng(seed)
    v = np.concatenate([g.normal(size=n), g.normal(size=n) * 1e-3, g.normal(size=n) * 1e3,
                        g.uniform(-1, 1, n) * 2.0 ** g.integers(-60, 60, n),
                        [1.0, -1.0, 1.0 + 2.0 ** -11, 1.0 + 2.0 ** -12, 1.0 + 3 * 2.0 ** -12,
                         -(1.0 + 2.0 ** -12), 0.0, 2.0 ** -100, 3.0e30]])
    return v.astype(np.float32)


def test_tf32_rounding_is_nearest_ties_away():
    # the TF32 unit at 1 is 2^-10: 1 + 2^-11 is a tie (away from zero, either sign), 1 + 2^-12
    # is below half a unit, 1 + 3 2^-12 above it
    x = np.array([1.0 + 2.0 ** -11, -(1.0 + 2.0 ** -11), 1.0 + 2.0 ** -12, 1.0 + 3 * 2.0 ** -12,
                  -(1.0 + 2.0 ** -12), 1.0 + 2.0 ** -11 - 2.0 ** -23], dtype=np.float32)
    want = np.array([1.0 + 2.0 ** -10, -(1.0 + 2.0 ** -10), 1.0, 1.0 + 2.0 ** -10, -1.0, 1.0],
                    dtype=np.float32)
    np.testing.assert_array_equal(tf32_rna(x), want)
    # every result has its low 13 mantissa bits clear and lies within half a TF32 unit
    v = _values(20000, 0)
    r = tf32_rna(v)
    assert np.all((r.view(np.uint32) & np.uint32(0x1FFF)) == 0)
    nz = v != 0
    assert np.all(np.abs(r[nz].astype(np.float64) - v[nz]) <= 2.0 ** -11 * np.abs(v[nz].astype(np.float64)))


def test_split_rest_below_2_pow_minus_22():
    v = _values(20000, 1)
    hi, lo = split(v)
    rest = v.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)
    assert np.all(np.abs(rest) <= 2.0 ** -22 * np.abs(v.astype(np.float64)))


def test_three_products_within_12u_and_one_product_is_not():
    x, y = _values(20000, 2), _values(20000, 3)[::-1].copy()
    keep = np.abs(x.astype(np.float64) * y) < 1e30
    x, y = x[keep], y[keep]
    hx, lx = split(x)
    hy, ly = split(y)
    exact = x.astype(np.float64) * y.astype(np.float64)
    three = (hx.astype(np.float64) * hy + hx.astype(np.float64) * ly + lx.astype(np.float64) * hy)
    assert np.all(np.abs(three - exact) <= 12 * U * np.abs(exact))
    one = hx.astype(np.float64) * hy
    assert np.max(np.abs(one - exact) / np.maximum(np.abs(exact), 1e-300)) > 100 * U
