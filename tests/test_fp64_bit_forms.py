"""The integer and bit-pattern forms the FP64 kernels use in place of FP64-pipe instructions,
checked on the host (numpy restatements of each identity; the GPU test in test_gpu_math.py
checks the device functions against the generic ones bit for bit):

* the uniform (w + 1/2) 2^-32 as (1 + u) assembled from w's bits, less 1;
* the logarithm's exponent and fraction bits of that uniform from the integer 2w + 1;
* the Box-Muller angle's reduction 256 v = j + f with j the nearest integer and
  f = (2 (w - j 2^24) + 1) 2^-25 (32-bit wrap-around giving the signed remainder at j = 256);
* the order keys (bit pattern with the magnitude bits of negative values flipped) sort doubles
  like the doubles, and the map is its own inverse;
* the -inf / NaN test and the |x| <= 708 test on bit patterns;
* lowering the exponent field by sh equals ldexp(v, -sh) when the result stays normal."""
import numpy as np

MASK52 = (1 << 52) - 1


def _bits(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).view(np.int64)


def _words(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    edge = [0, 1, 2, 3, (1 << 23) - 1, 1 << 23, (1 << 31) - 1, 1 << 31, (1 << 32) - 2, (1 << 32) - 1]
    return np.concatenate([rng.integers(0, 1 << 32, n, dtype=np.uint64), np.array(edge, dtype=np.uint64),
                           np.uint64(1) << np.arange(32, dtype=np.uint64),
                           np.arange(0, 512, dtype=np.uint64) << np.uint64(23)])


def test_uniform_from_its_bits():
    w = _words(200_000, 1)
    hi = (np.uint64(0x3FF00000) | (w >> np.uint64(12))) << np.uint64(32)
    lo = ((w << np.uint64(20)) & np.uint64(0xFFFFFFFF)) | np.uint64(1 << 19)
    one_u = (hi | lo).view(np.float64)
    assert np.all((one_u >= 1.0) & (one_u < 2.0))
    np.testing.assert_array_equal(one_u - 1.0, (w.astype(np.float64) + 0.5) * 2.0 ** -32)


def test_log_parts_of_the_uniform_from_the_integer():
    w = _words(200_000, 2)
    u = (w.astype(np.float64) + 0.5) * 2.0 ** -32
    v = 2 * w.astype(object) + 1                      # exact integers
    msb = np.array([int(x).bit_length() - 1 for x in v])
    e = msb - 33
    frac = np.array([(int(x) << (52 - int(b))) & MASK52 for x, b in zip(v, msb)], dtype=np.int64)
    b = _bits(u)
    np.testing.assert_array_equal(e, (b >> 52) - 1023)                     # the exponent
    np.testing.assert_array_equal(frac, b & MASK52)                        # the fraction bits
    m, ex = np.frexp(u)
    np.testing.assert_array_equal(e, ex - 1)


def test_angle_reduction_in_integers():
    w = _words(200_000, 3)
    t = (w.astype(np.float64) + 0.5) * 2.0 ** -24                         # 256 v, exact
    j = ((w >> np.uint64(23)) + np.uint64(1)) >> np.uint64(1)
    np.testing.assert_array_equal(j, np.floor(t + 0.5).astype(np.uint64))  # nearest (no ties)
    r32 = ((w - (j << np.uint64(24))) * np.uint64(2) + np.uint64(1)) & np.uint64(0xFFFFFFFF)
    r = r32.astype(np.int64) - ((r32 >> np.uint64(31)).astype(np.int64) << 32)   # as int32
    assert np.all(np.abs(r) < 1 << 24)
    np.testing.assert_array_equal(r.astype(np.float64) * 2.0 ** -25, t - j.astype(np.float64))
    assert set(np.unique(j)) <= set(range(257)) and 256 in j


def _order_key(x: np.ndarray) -> np.ndarray:
    b = _bits(x)
    return b ^ ((b >> 63) & np.int64(0x7FFFFFFFFFFFFFFF))


def test_order_keys_sort_like_the_doubles():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(100_000) * 10.0 ** rng.integers(-300, 300, 100_000),
                        [0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324, 1.0, -1.0, 2.2250738585072014e-308]])
    k = _order_key(x)
    order = np.argsort(k, kind="stable")
    assert np.all(np.diff(x[order]) >= 0)                                  # non-decreasing values
    back = (k ^ ((k >> 63) & np.int64(0x7FFFFFFFFFFFFFFF))).view(np.float64)
    np.testing.assert_array_equal(_bits(back), _bits(x))                   # its own inverse
    a, b = x[:50_000], x[50_000:100_000]                                  # the maximum of two keys
    km = np.maximum(_order_key(a), _order_key(b))
    np.testing.assert_array_equal((km ^ ((km >> 63) & np.int64(0x7FFFFFFFFFFFFFFF))).view(np.float64), np.maximum(a, b))


def test_range_tests_on_bit_patterns():
    x = np.array([0.0, -0.0, 1.0, -1.0, 708.0, -708.0, np.nextafter(708.0, np.inf), -np.nextafter(708.0, np.inf),
                  1e308, -1e308, np.inf, -np.inf, np.nan, -np.nan])
    b = _bits(x).view(np.uint64)
    above = ((b & np.uint64(0x7FFFFFFFFFFFFFFF)) <= np.uint64(0x7FF0000000000000)) & (b != np.uint64(0xFFF0000000000000))
    with np.errstate(invalid="ignore"):
        np.testing.assert_array_equal(above, x > -np.inf)
        np.testing.assert_array_equal((b & np.uint64(0x7FFFFFFFFFFFFFFF)) <= np.uint64(0x4086200000000000),
                                      np.abs(x) <= 708.0)
    assert _bits(np.array([708.0]))[0] == 0x4086200000000000


def test_exponent_lowering_equals_ldexp_when_normal():
    rng = np.random.default_rng(5)
    v = np.abs(rng.standard_normal(100_000)) * 10.0 ** rng.integers(-300, 300, 100_000)
    sh = rng.integers(0, 1100, 100_000)
    b = _bits(v)
    ex = (b >> 52).astype(np.int64)
    fast = (sh < ex) & (ex < 0x7FF)
    lowered = (b - (sh.astype(np.int64) << 52)).view(np.float64)
    np.testing.assert_array_equal(lowered[fast], np.ldexp(v, -sh)[fast])
    assert fast.mean() > 0.3 and (~fast).mean() > 0.1                      # both branches exercised
