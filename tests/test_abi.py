"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/airpf.h
declares; host-side argument checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2312_06484_gb300 import _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "airpf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(airpf_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = _binding.load()
    names = _declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_binding.SIGNATURES), "binding and header disagree"


def _cfg(**kw):
    base = dict(model=1, dx=1, dy=1, m=1024, M=256, T=1000, B=1, mode=2, tau=0.3, precision=1,
                record=0, seed=1, launch=0, reserved=0)
    base.update(kw)
    return _binding.AirpfConfig(**base)


def test_workspace_size_and_argument_checks():
    lib = _binding.load()
    n = ctypes.c_size_t()
    assert lib.airpf_workspace_bytes(ctypes.byref(_cfg()), ctypes.byref(n)) == 0
    # two particle stores of N floats plus small buffers
    assert 2 * 262144 * 4 <= n.value < 2 * 262144 * 4 + (1 << 20)
    bad = [dict(m=3), dict(m=131072), dict(M=0), dict(M=1025), dict(T=0), dict(B=0), dict(tau=0.0),
           dict(tau=1.01), dict(mode=3), dict(model=9), dict(dx=2), dict(model=3, dx=9),
           dict(precision=7), dict(record=64), dict(launch=5), dict(reserved=1),
           dict(ppt=3), dict(ppt=16), dict(ppt=8, precision=0), dict(ppt=8, model=0),
           dict(islands_per_cta=3), dict(islands_per_cta=-2),
           dict(tau_int=-0.1), dict(tau_int=1.5), dict(radix=3), dict(radix=1), dict(radix=8),
           dict(model=5), dict(model=5, dy=1)]
    for kw in bad:
        assert lib.airpf_workspace_bytes(ctypes.byref(_cfg(**kw)), ctypes.byref(n)) == 1, kw
        assert lib.airpf_last_error(None)
    out = ctypes.c_void_p()
    assert lib.airpf_create(ctypes.byref(_cfg(m=5)), None, 0, None, None, ctypes.byref(out)) == 1
    assert lib.airpf_create(ctypes.byref(_cfg()), None, 0, None, None, ctypes.byref(out)) == 3
    assert out.value is None
    assert lib.airpf_create(ctypes.byref(_cfg(model=3, dx=2, dy=2)), None, 0, None, None,
                            ctypes.byref(out)) == 1          # LGSSM without model data
    # valid: radix 4 and 1024 = 4^5 islands, adaptive internal resampling, the change-point model
    for kw in (dict(radix=4), dict(radix=1024), dict(tau_int=0.5), dict(model=5, dy=2)):
        assert lib.airpf_workspace_bytes(ctypes.byref(_cfg(**kw)), ctypes.byref(n)) == 0, kw
    # tau_int keeps one log-weight per particle per buffer (two buffers of N floats)
    base, air = ctypes.c_size_t(), ctypes.c_size_t()
    lib.airpf_workspace_bytes(ctypes.byref(_cfg()), ctypes.byref(base))
    lib.airpf_workspace_bytes(ctypes.byref(_cfg(tau_int=0.5)), ctypes.byref(air))
    assert air.value - base.value >= 2 * 262144 * 4
    assert lib.airpf_theta_dim(0, 1) == 4 and lib.airpf_theta_dim(3, 8) == 10 and lib.airpf_theta_dim(5, 1) == 3
    assert lib.airpf_status_string(4) == b"AIRPF_ERR_TIMEOUT"
    assert lib.airpf_run(None, None, None, 0, 0, None, None, None, None, None) == 1


def test_lineage_record_sizes_grow_workspace():
    lib = _binding.load()
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    lib.airpf_workspace_bytes(ctypes.byref(_cfg(m=16, M=64, T=100)), ctypes.byref(a))
    lib.airpf_workspace_bytes(ctypes.byref(_cfg(m=16, M=64, T=100, record=7)), ctypes.byref(b))
    assert b.value - a.value >= 100 * 1024 * 4


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built CUDA library the binding raises."""
    from paper_2312_06484_gb300 import _binding, build as _build
    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing" / "libairpf.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _binding.load(build_if_needed=False)


def test_moments_workspace_covers_the_small_grid_tiling():
    """With AIRPF_RECORD_MOMENTS the per-warp island sums are sized for the larger of the
    default tiling (4 particles a thread: 64 threads for M = 200) and the small-grid one
    (2 a thread: 128 threads, 4 warps per island), which a context of few CTAs takes."""
    lib = _binding.load()
    base, mom = ctypes.c_size_t(), ctypes.c_size_t()
    kw = dict(model=5, dy=2, m=64, M=200, T=50, B=3)
    assert lib.airpf_workspace_bytes(ctypes.byref(_cfg(**kw)), ctypes.byref(base)) == 0
    assert lib.airpf_workspace_bytes(ctypes.byref(_cfg(record=32, **kw)), ctypes.byref(mom)) == 0
    B, T, m, dx = 3, 50, 64, 1
    need = 8 * B * T * m * 2 + 8 * B * T * m * 4 * 4 * dx       # log W pairs, 4 warps x 4 dx sums
    assert need <= mom.value - base.value < need + 2 * 256


def test_run_static_checks_sizes_before_the_call():
    """run_static hands raw pointers to kernels that read theta[B*d] and y[T*dy] and write
    log_z[B]: short or misshapen tensors are refused on the host (no GPU needed here)."""
    import torch
    import paper_2312_06484_gb300 as gp
    f64 = dict(dtype=torch.float64)
    th, y, lz = torch.zeros(2 * 3, **f64), torch.zeros(10, **f64), torch.zeros(2, **f64)
    kw = dict(m=16, M=32, B=2)
    cases = [(torch.zeros(5, **f64), y, lz, {}, "theta holds"),
             (th, y, torch.zeros(1, **f64), {}, "log_z holds"),
             (th, torch.zeros(0, **f64), lz, {}, "y holds"),
             (th, torch.zeros(9, **f64), lz, dict(dy=2, model=5), "y holds")]
    for theta, yy, out, extra, msg in cases:
        model = extra.pop("model", gp.MODEL_SV)
        with pytest.raises(gp.AirpfError, match=msg):
            gp.run_static(model, theta, yy, out, **kw, **extra)
    # the LGSSM's model data: dx*dx + dy*dx values
    d = gp.theta_dim(gp.MODEL_LGSSM, 2)
    with pytest.raises(gp.AirpfError, match="model_data"):
        gp.run_static(gp.MODEL_LGSSM, torch.zeros(2 * d, **f64), torch.zeros(20, **f64), lz, dx=2, dy=2,
                      model_data=torch.zeros(5, **f64), **kw)
    # right sizes but host tensors: refused before any pointer reaches the library
    with pytest.raises(gp.AirpfError, match="CUDA tensors"):
        gp.run_static(gp.MODEL_SV, th, y, lz, **kw)
