"""The FP64 path's table-driven double exponential, logarithm and Box-Muller sine and cosine
(airpf_debug_math) against the host library's (numpy) and the device library's (torch on
CUDA): the exponential and logarithm within 2 ulp where the tables are used and the library's
values outside that range (infinities, NaN, zero, subnormals); sin and cos of 2 pi v within a
few 1e-16 of an extended-precision reference (2 ulp where |value| >= 1/4), exact at the
quarter turns; and the Box-Muller forms of a 32-bit word (the uniform assembled from its bits,
its logarithm and the angle reduced in integers) bit for bit equal to the generic functions of
that uniform."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
EXP, LOG, SIN2PI, COS2PI = 0, 1, 2, 3
UNIF_W, LOG_W, SIN2PI_W, COS2PI_W = 4, 5, 6, 7


def _tab(fn: int, x: np.ndarray) -> np.ndarray:
    from paper_2312_06484_gb300 import _binding
    lib = _binding.load()
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    _binding.check(lib.airpf_debug_math(fn, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()),
                                        xd.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _ulps(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distance in units in the last place (same-sign values)."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_exp_within_two_ulp_of_the_library_exponentials(gpu_lib):
    rng = np.random.default_rng(7)
    ln2_n = np.log(2.0) / 256
    x = np.concatenate([rng.uniform(-708.0, 708.0, 2_000_000), rng.uniform(-1.0, 1.0, 1_000_000),
                        rng.uniform(-40.0, 0.0, 1_000_000),            # the weights' range
                        np.arange(-100000, 100000) * ln2_n,            # table points
                        np.arange(-100000, 100000) * ln2_n + ln2_n / 2,   # and reduction boundaries
                        [0.0, -0.0, 1e-300, -1e-300, 708.0, -708.0]])
    got = _tab(EXP, x)
    assert _ulps(got, np.exp(x)).max() <= 2
    assert _ulps(got, torch.exp(torch.tensor(x, device="cuda")).cpu().numpy()).max() <= 2


def test_log_within_two_ulp_of_the_library_logarithms(gpu_lib):
    rng = np.random.default_rng(8)
    w = rng.integers(0, 2 ** 32, 2_000_000, dtype=np.uint64)
    u = (w.astype(np.float64) + 0.5) * 2.0 ** -32                       # the Box-Muller words
    edge = (np.array([0, 1, 2, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1], dtype=np.float64) + 0.5) * 2.0 ** -32
    near1 = 1.0 + rng.uniform(-1e-3, 1e-3, 500_000)
    wide = np.exp(rng.uniform(-700.0, 700.0, 1_000_000))
    grid = 1.0 + np.arange(0, 257) / 256.0                              # the table points and midpoints
    x = np.concatenate([u, edge, near1, wide, grid, grid / 2, [1.0, 2.0, 0.5, np.e, 2.2250738585072014e-308]])
    got = _tab(LOG, x)
    host = np.log(x)
    dev = torch.log(torch.tensor(x, device="cuda")).cpu().numpy()
    pos, neg = host > 0, host < 0                                       # compare same-sign values
    for ref in (host, dev):
        assert _ulps(got[pos], ref[pos]).max() <= 2 and _ulps(-got[neg], -ref[neg]).max() <= 2
    assert np.all(got[host == 0] == 0)


def test_outside_the_table_ranges_they_are_the_library_functions(gpu_lib):
    x = np.array([709.5, 710.0, 1e6, np.inf, -709.0, -740.0, -745.2, -746.0, -1e6, -np.inf, np.nan])
    got = _tab(EXP, x)
    np.testing.assert_array_equal(got, torch.exp(torch.tensor(x, device="cuda")).cpu().numpy())
    assert np.isnan(got[-1]) and got[3] == np.inf and got[9] == 0.0
    x = np.array([0.0, -0.0, -1.0, 1e-310, 5e-324, np.inf, np.nan])
    got = _tab(LOG, x)
    np.testing.assert_array_equal(got, torch.log(torch.tensor(x, device="cuda")).cpu().numpy())
    assert got[0] == -np.inf and np.isnan(got[2]) and got[5] == np.inf


def test_sin_cos_of_two_pi_v(gpu_lib):
    rng = np.random.default_rng(9)
    w = rng.integers(0, 2 ** 32, 1_000_000, dtype=np.uint64)
    v = (w.astype(np.float64) + 0.5) * 2.0 ** -32                       # the Box-Muller words
    grid = np.arange(0, 513) / 512.0                                    # table points and midpoints
    v = np.concatenate([v, grid, [2.0 ** -33, 1 - 2.0 ** -33]])
    # reference in extended precision: 2 pi as a double-double, the product and sine in long double
    two_pi = np.longdouble(6.283185307179586) + np.longdouble(2.4492935982947064e-16)
    ang = v.astype(np.longdouble) * two_pi
    s, c = _tab(SIN2PI, v), _tab(COS2PI, v)
    for got, ref in ((s, np.sin(ang)), (c, np.cos(ang))):
        err = np.abs(got.astype(np.longdouble) - ref).astype(np.float64)
        assert err.max() <= 3.4e-16                                     # a few 1e-16 absolute
        big = np.abs(ref) >= 0.25
        assert np.all(err[big] <= 2 * np.spacing(np.abs(ref[big]).astype(np.float64)))   # 2 ulp
    # and near the host library's values (whose argument 2 pi v is itself rounded)
    assert np.abs(s - np.sin(2 * np.pi * v)).max() <= 1e-15 and np.abs(c - np.cos(2 * np.pi * v)).max() <= 1e-15
    x = np.array([0.0, 0.25, 0.5, 0.75, 1.0])
    np.testing.assert_array_equal(_tab(SIN2PI, x), [0.0, 1.0, 0.0, -1.0, 0.0])
    np.testing.assert_array_equal(_tab(COS2PI, x), [1.0, 0.0, -1.0, 0.0, 1.0])


def test_word_forms_equal_the_generic_functions_of_the_uniform(gpu_lib):
    rng = np.random.default_rng(10)
    w = np.concatenate([rng.integers(0, 2 ** 32, 1_000_000, dtype=np.uint64),
                        np.arange(0, 4096, dtype=np.uint64),                    # small words: e down to -33
                        2 ** 32 - 1 - np.arange(0, 4096, dtype=np.uint64),      # the top: j = 256
                        (np.arange(0, 512, dtype=np.uint64) << 23),             # 512th boundaries
                        (np.arange(1, 513, dtype=np.uint64) << 23) - 1,
                        np.uint64(1) << np.arange(0, 32, dtype=np.uint64)])     # every exponent
    wd = w.astype(np.float64)
    u = _tab(UNIF_W, wd)
    np.testing.assert_array_equal(u, (wd + 0.5) * 2.0 ** -32)                   # exact
    for fw, fu in ((LOG_W, LOG), (SIN2PI_W, SIN2PI), (COS2PI_W, COS2PI)):
        np.testing.assert_array_equal(_tab(fw, wd).view(np.int64), _tab(fu, u).view(np.int64))
