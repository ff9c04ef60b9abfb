"""GB300 (sm_103a) Augmented Island Resampling Particle Filter.

Heine, "Augmented Island Resampling Particle Filters for Particle Markov Chain Monte
Carlo" (arXiv 2312.06484), Algorithm 1, run inside particle marginal Metropolis-
Hastings.  Every step of the filter runs in the CUDA kernels of ``csrc/`` behind the C
ABI of ``include/airpf.h``; this module only marshals torch tensors (device memory and
streams) into that ABI.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding
from ._binding import AirpfConfig, AirpfError

MODEL_AR1, MODEL_SV, MODEL_NGM, MODEL_LGSSM, MODEL_TOY, MODEL_CP = 0, 1, 2, 3, 4, 5
NEVER, ALWAYS, ADAPTIVE = 0, 1, 2
FP64, FP32_MIXED = 0, 1
RECORD_LINEAGE, RECORD_ENF, RECORD_TRACE, RECORD_TIMING, RECORD_GRAD, RECORD_MOMENTS = 1, 2, 4, 8, 16, 32
LAUNCH_AUTO, LAUNCH_STEPS, LAUNCH_PERSISTENT_CTA, LAUNCH_PERSISTENT_GRID, LAUNCH_STEPS_SPLIT = 0, 1, 2, 3, 4

_MODES = {"never": NEVER, "always": ALWAYS, "adaptive": ADAPTIVE}
_PREC = {"fp64": FP64, "fp32": FP32_MIXED, "fp32_mixed": FP32_MIXED}
_LAUNCH = {"auto": LAUNCH_AUTO, "steps": LAUNCH_STEPS, "cta": LAUNCH_PERSISTENT_CTA,
           "grid": LAUNCH_PERSISTENT_GRID, "split": LAUNCH_STEPS_SPLIT}


def theta_dim(model: int, dx: int = 1) -> int:
    return int(_binding.load().airpf_theta_dim(model, dx))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class AIRPF:
    """One context: B filters of m islands x M particles over T observations.

    Device workspace is a torch uint8 tensor; all work is enqueued on ``stream``
    (default: torch's current CUDA stream)."""

    def __init__(self, model: int, *, m: int, M: int, T: int, B: int = 1, dx: int = 1, dy: int = 1,
                 mode="adaptive", tau: float = 0.3, precision="fp64", seed: int = 0, record: int = 0,
                 model_data=None, stream=None, launch="auto", ppt: int = 0, islands_per_cta: int = 0,
                 ckpt: int = 0, tau_int: float = 0.0, radix: int = 2):
        import torch
        self._torch = torch
        self.lib = _binding.load()
        mode = _MODES[mode] if isinstance(mode, str) else int(mode)
        precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        launch = _LAUNCH[launch] if isinstance(launch, str) else int(launch)
        self.cfg = AirpfConfig(model=model, dx=dx, dy=dy, m=m, M=M, T=T, B=B, mode=mode, tau=tau,
                               precision=precision, record=record, seed=seed, launch=launch, reserved=0,
                               ppt=ppt, islands_per_cta=islands_per_cta, ckpt=ckpt, tau_int=tau_int, radix=radix)
        nbytes = ctypes.c_size_t()
        _binding.check(self.lib.airpf_workspace_bytes(ctypes.byref(self.cfg), ctypes.byref(nbytes)))
        self.workspace = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        md = None
        if model_data is not None:
            self._md = np.ascontiguousarray(np.asarray(model_data, dtype=np.float64))
            md = self._md.ctypes.data_as(ctypes.c_void_p)
        ctx = ctypes.c_void_p()
        _binding.check(self.lib.airpf_create(ctypes.byref(self.cfg), _ptr(self.workspace), nbytes.value, md,
                                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx)))
        self.ctx = ctx
        self.m, self.M, self.T, self.B, self.dx, self.dy = m, M, T, B, dx, dy
        self.N = m * M
        self.S = int(round(np.log2(m)))
        # interaction stages: S_r = log_r m for radix r (S for r = 2)
        self.S_r = self.S // max(1, int(round(np.log2(radix)))) if radix > 2 else self.S
        self.theta_dim = theta_dim(model, dx)
        self.record = record

    # -- runs -------------------------------------------------------------------------------
    def run(self, theta, y, *, chain0: int = 0, iter: int = 0, lineage=False, enf=False, trace=False):
        """One pass of Algorithm 1 for every filter of the batch.  theta: [B, d] float64 CUDA;
        y: [T*dy] float64 CUDA.  Returns dict of CUDA tensors (log_z [B], optional
        anc [B, T, N], enf [B, T, S_r+1], sstar [B, T], trace [B, T]; S_r the number of
        interaction stages, log_r m for radix r)."""
        torch = self._torch
        theta = theta.reshape(self.B, self.theta_dim).to(device="cuda", dtype=torch.float64).contiguous()
        y = y.reshape(-1).to(device="cuda", dtype=torch.float64).contiguous()
        out = {"log_z": torch.empty(self.B, dtype=torch.float64, device="cuda")}
        if lineage:
            out["anc"] = torch.empty((self.B, self.T, self.N), dtype=torch.int32, device="cuda")
        if enf:
            out["enf"] = torch.empty((self.B, self.T, self.S_r + 1), dtype=torch.float64, device="cuda")
            out["sstar"] = torch.empty((self.B, self.T), dtype=torch.int32, device="cuda")
        if trace:
            out["trace"] = torch.empty((self.B, self.T), dtype=torch.float64, device="cuda")
        self._keep = (theta, y)
        _binding.check(self.lib.airpf_run(self.ctx, _ptr(theta), _ptr(y), chain0, iter, _ptr(out["log_z"]),
                                          _ptr(out.get("anc")), _ptr(out.get("enf")), _ptr(out.get("sstar")),
                                          _ptr(out.get("trace"))), self.ctx)
        return out

    def run_host(self, theta: np.ndarray, y: np.ndarray, *, chain0: int = 0, iter: int = 0) -> np.ndarray:
        """Host buffers in and out; synchronises.  Returns log_z [B] (numpy)."""
        theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(self.B, self.theta_dim))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(-1))
        lz = np.empty(self.B, dtype=np.float64)
        _binding.check(self.lib.airpf_run_host(self.ctx, theta.ctypes.data_as(ctypes.c_void_p),
                                               y.ctypes.data_as(ctypes.c_void_p), chain0, iter,
                                               lz.ctypes.data_as(ctypes.c_void_p)), self.ctx)
        return lz

    # -- stepwise passes (the islands of one filter split over processes) -----------------
    def step_begin(self, theta, y, *, chain0: int = 0, iter: int = 0):
        """Copies theta and y in and runs the pass's prologue (airpf_step_begin)."""
        torch = self._torch
        theta = theta.reshape(self.B, self.theta_dim).to(device="cuda", dtype=torch.float64).contiguous()
        y = y.reshape(-1).to(device="cuda", dtype=torch.float64).contiguous()
        self._keep = (theta, y)
        _binding.check(self.lib.airpf_step_begin(self.ctx, _ptr(theta), _ptr(y), chain0, iter), self.ctx)

    def step_islands(self, t: int, cta0: int = 0, ncta: int = 0):
        """Island work of step t for CTAs cta0 .. cta0+ncta-1 (0: all) (airpf_step_islands)."""
        _binding.check(self.lib.airpf_step_islands(self.ctx, t, cta0, ncta), self.ctx)

    def step_cascade(self, t: int):
        """The cascade of step t over all CTA records (airpf_step_cascade)."""
        _binding.check(self.lib.airpf_step_cascade(self.ctx, t), self.ctx)

    def step_end(self):
        """Returns log Z^N_T as a [1] float64 CUDA tensor (airpf_step_end)."""
        out = self._torch.empty(1, dtype=self._torch.float64, device="cuda")
        _binding.check(self.lib.airpf_step_end(self.ctx, _ptr(out)), self.ctx)
        return out

    def step_regions(self, t: int):
        """Views of the workspace that step t's island launch writes, one uint8 tensor a
        region: CTA exponents, CTA block-sum subtrees, CTA sums of squares, then the particle
        rows of each state dimension (airpf_step_regions).  Each is ordered by CTA, so CTA
        range j of G equal ranges owns part j of G equal parts of every region."""
        n = 8 + self.dx
        offs, nb, cnt = (ctypes.c_size_t * n)(), (ctypes.c_size_t * n)(), ctypes.c_int32()
        _binding.check(self.lib.airpf_step_regions(self.ctx, t, offs, nb, ctypes.byref(cnt)), self.ctx)
        return [self.workspace[offs[i]:offs[i] + nb[i]] for i in range(cnt.value)]

    @property
    def ctas(self) -> int:
        """CTAs of one filter's island launch (one int32 exponent record each)."""
        return self.step_regions(0)[0].numel() // 4

    def step_levels(self) -> int:
        """Split steps: the binary interaction levels of the last cascade (airpf_step_levels;
        synchronises the stream)."""
        lv = ctypes.c_int32()
        _binding.check(self.lib.airpf_step_levels(self.ctx, ctypes.byref(lv)), self.ctx)
        return int(lv.value)

    def pmmh(self, y, state_theta, state_logz, *, step, lo, hi, iters: int, chain0: int = 0,
             iter0: int = 0, n_accept=None, record: bool = True):
        """Random-walk PMMH, one chain per filter, entirely on the device (airpf_pmmh).
        state_theta [B, d] and state_logz [B] are float64 CUDA tensors updated in place
        (NaN log Z: estimated first).  step/lo/hi: length-d sequences.  Returns dict with
        n_accept [B] (int32, accumulated into ``n_accept`` if given) and, with record,
        theta [iters, B, d] and log_z [iters, B]."""
        torch = self._torch
        d = self.theta_dim
        assert state_theta.dtype == torch.float64 and state_theta.is_cuda and state_theta.is_contiguous()
        assert state_logz.dtype == torch.float64 and state_logz.is_cuda and state_logz.numel() == self.B
        y = y.reshape(-1).to(device="cuda", dtype=torch.float64).contiguous()
        arrs = [np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(d)) for v in (step, lo, hi)]
        if n_accept is None:
            n_accept = torch.zeros(self.B, dtype=torch.int32, device="cuda")
        out = {"n_accept": n_accept}
        if record:
            out["theta"] = torch.empty((iters, self.B, d), dtype=torch.float64, device="cuda")
            out["log_z"] = torch.empty((iters, self.B), dtype=torch.float64, device="cuda")
        self._keep = (y, arrs)
        _binding.check(self.lib.airpf_pmmh(self.ctx, _ptr(y), *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                           _ptr(state_theta), _ptr(state_logz), chain0, iter0, iters,
                                           _ptr(out.get("theta")), _ptr(out.get("log_z")), _ptr(n_accept)),
                       self.ctx)
        return out

    def pmmh_langevin(self, y, state_theta, state_logz, state_grad, *, step, lo, hi, iters: int,
                      chain0: int = 0, iter0: int = 0, n_accept=None, record: bool = True):
        """PMMH with the Langevin proposal (airpf_pmmh_langevin; context with RECORD_GRAD).
        state_theta [B, d], state_logz [B] (NaN: estimated first) and state_grad [B, d] are
        float64 CUDA tensors updated in place."""
        torch = self._torch
        d = self.theta_dim
        for t in (state_theta, state_logz, state_grad):
            assert t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
        y = y.reshape(-1).to(device="cuda", dtype=torch.float64).contiguous()
        arrs = [np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(d)) for v in (step, lo, hi)]
        if n_accept is None:
            n_accept = torch.zeros(self.B, dtype=torch.int32, device="cuda")
        out = {"n_accept": n_accept}
        if record:
            out["theta"] = torch.empty((iters, self.B, d), dtype=torch.float64, device="cuda")
            out["log_z"] = torch.empty((iters, self.B), dtype=torch.float64, device="cuda")
        self._keep = (y, arrs)
        _binding.check(self.lib.airpf_pmmh_langevin(
            self.ctx, _ptr(y), *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs], _ptr(state_theta),
            _ptr(state_logz), _ptr(state_grad), chain0, iter0, iters, _ptr(out.get("theta")),
            _ptr(out.get("log_z")), _ptr(n_accept)), self.ctx)
        return out

    def grad(self, theta, y, *, chain0: int = 0, iter: int = 0):
        """airpf_grad (context created with RECORD_GRAD): returns dict of CUDA tensors log_z [B],
        grad [B, d] (adjoint with the lineage held fixed) and score [B, d] (Fisher-identity
        score along the lineages)."""
        torch = self._torch
        theta = theta.reshape(self.B, self.theta_dim).to(device="cuda", dtype=torch.float64).contiguous()
        y = y.reshape(-1).to(device="cuda", dtype=torch.float64).contiguous()
        out = {"log_z": torch.empty(self.B, dtype=torch.float64, device="cuda"),
               "grad": torch.empty((self.B, self.theta_dim), dtype=torch.float64, device="cuda"),
               "score": torch.empty((self.B, self.theta_dim), dtype=torch.float64, device="cuda")}
        self._keep = (theta, y)
        _binding.check(self.lib.airpf_grad(self.ctx, _ptr(theta), _ptr(y), chain0, iter, _ptr(out["log_z"]),
                                           _ptr(out["grad"]), _ptr(out["score"])), self.ctx)
        return out

    def moments(self):
        """Output measures of the last run (context created with RECORD_MOMENTS): a CUDA
        tensor [B, T, 2, 2, dx]; [:, t, 0] the prediction filter (mutated particles, weights
        before y_t), [:, t, 1] the filter (internally resampled particles, weights after y_t);
        [..., 0, d] E[x_d], [..., 1, d] E[x_d^2]."""
        torch = self._torch
        out = torch.empty((self.B, self.T, 2, 2, self.dx), dtype=torch.float64, device="cuda")
        _binding.check(self.lib.airpf_moments(self.ctx, _ptr(out)), self.ctx)
        return out

    def kernel_times(self):
        """(island-step kernels ms, cascade kernels ms) of the last run; needs RECORD_TIMING."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _binding.check(self.lib.airpf_kernel_times(self.ctx, ctypes.byref(a), ctypes.byref(b)), self.ctx)
        return a.value, b.value

    def launch_count(self) -> int:
        return int(self.lib.airpf_last_launch_count(self.ctx))

    @property
    def launch_mode(self) -> int:
        return int(self.lib.airpf_launch_mode(self.ctx))

    @property
    def tiling(self) -> dict:
        """The island-to-thread mapping: threads per island, particles per thread, islands
        per CTA (airpf_tiling)."""
        v = (ctypes.c_int32 * 3)()
        _binding.check(self.lib.airpf_tiling(self.ctx, ctypes.byref(v, 0), ctypes.byref(v, 4), ctypes.byref(v, 8)))
        return {"threads_per_island": v[0], "particles_per_thread": v[1], "islands_per_cta": v[2]}

    def sync(self):
        """Wait for the stream; raises AirpfError (AIRPF_ERR_TIMEOUT) if a bounded device wait ran out."""
        _binding.check(self.lib.airpf_sync(self.ctx), self.ctx)

    def inject(self, what: int):
        """Test hook of the failure path (see airpf_debug_inject)."""
        _binding.check(self.lib.airpf_debug_inject(self.ctx, what), self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.airpf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Chains of uneven (m, M): one ``AIRPF`` context per size class (its chains are that
    context's batch), run side by side through airpf_group_*.  Each member must have been
    created on a stream of its own; the group forks them from ``stream`` (default: torch's
    current stream) and joins them back."""

    def __init__(self, members, stream=None):
        import torch
        self._torch = torch
        self.lib = _binding.load()
        self.members = list(members)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (ctypes.c_void_p * len(self.members))(*[mb.ctx.value for mb in self.members])
        g = ctypes.c_void_p()
        _binding.check(self.lib.airpf_group_create(arr, len(self.members), ctypes.c_void_p(self.stream.cuda_stream),
                                                   ctypes.byref(g)))
        self.g = g

    @staticmethod
    def _ptrs(ts):
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])

    def run(self, thetas, y, chain0s, *, iter: int = 0):
        """thetas[i]: [B_i, d] float64 CUDA; returns the list of log Z tensors [B_i]."""
        torch = self._torch
        thetas = [t.to(device="cuda", dtype=torch.float64).contiguous() for t in thetas]
        y = y.reshape(-1).to(device="cuda", dtype=torch.float64).contiguous()
        out = [torch.empty(mb.B, dtype=torch.float64, device="cuda") for mb in self.members]
        c0 = (ctypes.c_uint32 * len(self.members))(*chain0s)
        self._keep = (thetas, y)
        _binding.check(self.lib.airpf_group_run(self.g, self._ptrs(thetas), _ptr(y), c0, iter, self._ptrs(out)))
        return out

    def pmmh(self, y, states_theta, states_logz, *, step, lo, hi, iters: int, chain0s, iter0: int = 0,
             n_accepts=None, record: bool = False):
        """airpf_pmmh for every member, one call; states are updated in place."""
        torch = self._torch
        n = len(self.members)
        y = y.reshape(-1).to(device="cuda", dtype=torch.float64).contiguous()
        d = self.members[0].theta_dim
        arrs = [np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(d)) for v in (step, lo, hi)]
        if n_accepts is None:
            n_accepts = [torch.zeros(mb.B, dtype=torch.int32, device="cuda") for mb in self.members]
        th_out = [torch.empty((iters, mb.B, d), dtype=torch.float64, device="cuda") for mb in self.members] \
            if record else None
        lz_out = [torch.empty((iters, mb.B), dtype=torch.float64, device="cuda") for mb in self.members] \
            if record else None
        c0 = (ctypes.c_uint32 * n)(*chain0s)
        self._keep = (y, arrs)
        _binding.check(self.lib.airpf_group_pmmh(
            self.g, _ptr(y), *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs], self._ptrs(states_theta),
            self._ptrs(states_logz), c0, iter0, iters, self._ptrs(th_out) if record else None,
            self._ptrs(lz_out) if record else None, self._ptrs(n_accepts)))
        return {"n_accept": n_accepts, "theta": th_out, "log_z": lz_out}

    def sync(self):
        _binding.check(self.lib.airpf_group_sync(self.g))

    def close(self):
        if getattr(self, "g", None):
            self.lib.airpf_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(model, theta, y, *, m: int, M: int, B: int = 1, dx: int = 1, dy: int = 1, mode="adaptive",
             tau: float = 0.3, precision="fp64", seed: int = 0, model_data=None, passes: int = 3, stream=None):
    """airpf_autotune: the fastest tiling for this configuration.  Returns
    ({"launch", "ppt", "islands_per_cta"}, ms per pass)."""
    import torch
    lib = _binding.load()
    mode = _MODES[mode] if isinstance(mode, str) else int(mode)
    precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    y = y.reshape(-1).to(device="cuda", dtype=torch.float64).contiguous()
    theta = theta.to(device="cuda", dtype=torch.float64).contiguous()
    cfg = AirpfConfig(model=model, dx=dx, dy=dy, m=m, M=M, T=y.numel() // dy, B=B, mode=mode, tau=tau,
                      precision=precision, record=0, seed=seed, launch=0, reserved=0)
    need = ctypes.c_size_t()
    _binding.check(lib.airpf_workspace_bytes(ctypes.byref(cfg), ctypes.byref(need)))
    ws = torch.empty(((need.value + 255) // 256) * 256 + 8 * B, dtype=torch.uint8, device="cuda")
    md = None
    if model_data is not None:
        md_np = np.ascontiguousarray(np.asarray(model_data, dtype=np.float64))
        md = md_np.ctypes.data_as(ctypes.c_void_p)
    stream = stream if stream is not None else torch.cuda.current_stream()
    best = AirpfConfig()
    ms = ctypes.c_float()
    _binding.check(lib.airpf_autotune(ctypes.byref(cfg), _ptr(ws), ws.numel(), md, _ptr(theta), _ptr(y), passes,
                                      ctypes.c_void_p(stream.cuda_stream), ctypes.byref(best), ctypes.byref(ms)))
    return {"launch": int(best.launch), "ppt": int(best.ppt), "islands_per_cta": int(best.islands_per_cta)}, \
        float(ms.value)


def run_static(model: int, theta, y, log_z, *, m: int, M: int, B: int = 1, dx: int = 1, dy: int = 1,
               mode="adaptive", tau: float = 0.3, precision="fp64", seed: int = 0, chain0: int = 0,
               iter: int = 0, model_data=None, launch="auto", stream=None, tau_int: float = 0.0,
               radix: int = 2):
    """One pass through airpf_run_static: no context and no device allocation (the library's
    static scratch serves as workspace).  theta [B, d], y [T*dy], log_z [B] (out) and the
    optional model_data are float64 CUDA tensors, used in place."""
    import torch
    lib = _binding.load()
    mode = _MODES[mode] if isinstance(mode, str) else int(mode)
    precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    launch = _LAUNCH[launch] if isinstance(launch, str) else int(launch)
    T = y.numel() // dy
    cfg = AirpfConfig(model=model, dx=dx, dy=dy, m=m, M=M, T=T, B=B, mode=mode, tau=tau, precision=precision,
                      record=0, seed=seed, launch=launch, reserved=0, tau_int=tau_int, radix=radix)
    # the kernels read theta[B*d], y[T*dy] and the model data and write log_z[B] through raw
    # pointers: every size is checked here, before the call
    d = int(lib.airpf_theta_dim(model, dx))
    if d <= 0:
        raise AirpfError(f"ARG: unknown model {model} (dx = {dx})")
    if theta.numel() != B * d:
        raise AirpfError(f"ARG: theta holds {theta.numel()} values, B * theta_dim = {B * d}")
    if log_z.numel() < B:
        raise AirpfError(f"ARG: log_z holds {log_z.numel()} values, fewer than B = {B}")
    if y.numel() == 0 or y.numel() % dy:
        raise AirpfError(f"ARG: y holds {y.numel()} values, not a positive multiple of dy = {dy}")
    if model == MODEL_LGSSM:
        if model_data is None or model_data.numel() != dx * dx + dy * dx:
            n = None if model_data is None else model_data.numel()
            raise AirpfError(f"ARG: the LGSSM needs model_data of dx*dx + dy*dx = {dx * dx + dy * dx} values, got {n}")
    for t in (theta, y, log_z) + ((model_data,) if model_data is not None else ()):
        if not (t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()):
            raise AirpfError("ARG: theta, y, log_z and model_data must be contiguous float64 CUDA tensors")
    stream = stream if stream is not None else torch.cuda.current_stream()
    _binding.check(lib.airpf_run_static(ctypes.byref(cfg), _ptr(theta), _ptr(y), _ptr(model_data), chain0, iter,
                                        _ptr(log_z), ctypes.c_void_p(stream.cuda_stream)))
    return log_z


_LOGZ_FUNCTION = None


def _logz_function():
    """The torch.autograd.Function behind log_z (defined on first use: torch is
    imported lazily)."""
    global _LOGZ_FUNCTION
    if _LOGZ_FUNCTION is None:
        import torch

        class AirpfLogZ(torch.autograd.Function):
            """log Z [B] of a context's filters as a function of theta [B, d]: the forward
            pass is airpf_grad (the filter with its lineage, island choices and s* recorded,
            then the adjoint with them held fixed), which keeps d log Z / d theta for the
            backward pass; y and the stream identity are not differentiated."""

            @staticmethod
            def forward(ctx, theta, y, f, chain0, iter):
                out = f.grad(theta, y, chain0=chain0, iter=iter)
                ctx.theta_shape = theta.shape
                ctx.theta_dtype = theta.dtype
                ctx.save_for_backward(out["grad"])
                return out["log_z"]

            @staticmethod
            def backward(ctx, g_logz):
                (grad,) = ctx.saved_tensors
                g = (g_logz.to(grad.dtype)[:, None] * grad).reshape(ctx.theta_shape).to(ctx.theta_dtype)
                return g, None, None, None, None

        _LOGZ_FUNCTION = AirpfLogZ
    return _LOGZ_FUNCTION


def log_z(f: AIRPF, theta, y, *, chain0: int = 0, iter: int = 0):
    """Differentiable log Z [B] of context ``f`` (created with ``record=RECORD_GRAD``) at
    theta [B, d] (or [d] for one filter): ``log_z(f, th, y).sum().backward()`` leaves the
    adjoint gradient of each filter's log Z in ``th.grad``."""
    return _logz_function().apply(theta, y, f, chain0, iter)


__all__ = ["AIRPF", "AirpfError", "Group", "autotune", "theta_dim", "run_static", "log_z", "MODEL_AR1", "MODEL_SV", "MODEL_NGM", "MODEL_LGSSM",
           "MODEL_TOY", "MODEL_CP", "NEVER", "ALWAYS", "ADAPTIVE", "FP64", "FP32_MIXED", "RECORD_LINEAGE",
           "RECORD_ENF", "RECORD_TRACE", "RECORD_TIMING", "RECORD_GRAD", "RECORD_MOMENTS", "LAUNCH_AUTO", "LAUNCH_STEPS", "LAUNCH_PERSISTENT_CTA",
           "LAUNCH_PERSISTENT_GRID", "LAUNCH_STEPS_SPLIT"]
