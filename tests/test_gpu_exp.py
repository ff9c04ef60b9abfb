"""The FP64 path's table-driven exponential (airpf_debug_exp) against the host library's exp
(numpy) and the device library's (torch on CUDA): within 2 ulp over |x| <= 708, where the
table is used, and the same values outside it (infinities, NaN, subnormal results)."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _exp_tab(x: np.ndarray) -> np.ndarray:
    from paper_2312_06484_gb300 import _binding
    lib = _binding.load()
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    _binding.check(lib.airpf_debug_exp(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), xd.numel(),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _ulps(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_within_two_ulp_of_the_library_exponentials(gpu_lib):
    rng = np.random.default_rng(7)
    ln2_64 = np.log(2.0) / 64
    x = np.concatenate([rng.uniform(-708.0, 708.0, 2_000_000), rng.uniform(-1.0, 1.0, 1_000_000),
                        rng.uniform(-40.0, 0.0, 1_000_000),            # the weights' range
                        np.arange(-20000, 20000) * ln2_64,             # table boundaries
                        np.arange(-20000, 20000) * ln2_64 + ln2_64 / 2,
                        [0.0, -0.0, 1e-300, -1e-300, 708.0, -708.0]])
    got = _exp_tab(x)
    host = np.exp(x)
    dev = torch.exp(torch.tensor(x, device="cuda")).cpu().numpy()
    assert _ulps(got, host).max() <= 2
    assert _ulps(got, dev).max() <= 2


def test_outside_the_table_range_it_is_the_library_function(gpu_lib):
    x = np.array([709.5, 710.0, 1e6, np.inf, -709.0, -740.0, -745.2, -746.0, -1e6, -np.inf, np.nan])
    got = _exp_tab(x)
    dev = torch.exp(torch.tensor(x, device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(got, dev)
    assert np.isnan(got[-1]) and got[3] == np.inf and got[9] == 0.0
