"""CPU oracle for the AIRPF hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline
leg (and ``bench.py --impl reference``) may import this package.  It shares no
code with the CUDA path (``paper_2312_06484_gb300``); both read their inputs
from ``synth``.

Contents:
  * ``philox``          Philox4x32-10 (Salmon et al., SC'11), C.
  * ``airpf``           Algorithm 1 of Heine (arXiv 2312.06484), literal, FP64, C.
  * ``bpf``             the bootstrap filter (the m = 1 case, Section 2), C.
  * ``pmmh``            particle marginal Metropolis-Hastings, C.
  * ``kalman``          Kalman-filter likelihoods (exact Z for linear-Gaussian models).
  * ``exact_variance``  exact E[Z^N] and E[(Z^N)^2] on finite HMMs (Theorem 3).
"""
from __future__ import annotations

import ctypes
import math
import numpy as np

from . import build as _build

MODE_NEVER, MODE_ALWAYS, MODE_ADAPTIVE = 0, 1, 2
TIE_NONE, TIE_RESAMPLE, TIE_ISLAND, TIE_ENF = 0, 1, 2, 3

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int32)
_U = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.oracle_philox.argtypes = [_U, _U, _U]
        _lib.oracle_airpf.argtypes = [ctypes.c_int] * 6 + [ctypes.c_int, ctypes.c_double,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      _D, _D, _D, _D, _D, _I, _I, _D, _I, _D, _I]
        _lib.oracle_bpf.argtypes = [ctypes.c_int] * 5 + [ctypes.c_uint64, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint32, _D, _D, _D, _D, _I, _I]
        _lib.oracle_pmmh.argtypes = [ctypes.c_int] * 6 + [ctypes.c_int, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_uint32, _D, _D, ctypes.c_int,
                                     _D, _D, _D, _D, _D, ctypes.c_uint32, ctypes.c_int,
                                     _D, _D, _I]
        _lib.oracle_model_logg.argtypes = [ctypes.c_int] * 3 + [_D, _D, _D, _D]
        _lib.oracle_model_logg.restype = ctypes.c_double
        _lib.oracle_model_prior.argtypes = [ctypes.c_int] * 3 + [_D, _D, ctypes.c_uint64,
                                            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _D]
        _lib.oracle_model_step.argtypes = [ctypes.c_int] * 3 + [_D, _D, ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, _D, _D]
        _lib.oracle_model_valid.argtypes = [ctypes.c_int, ctypes.c_int, _D]
        _lib.oracle_set_tie_rel.argtypes = [ctypes.c_double]
        _lib.oracle_set_tau_int.argtypes = [ctypes.c_double]
        _lib.oracle_set_radix.argtypes = [ctypes.c_int]
        _lib.oracle_set_tie_masks.argtypes = [ctypes.c_void_p] * 3
        _lib.oracle_airpf_batch.argtypes = [ctypes.c_int] * 6 + [ctypes.c_int, ctypes.c_double,
                                            ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_int, _D, _D, _D, _D]
        _lib.oracle_model_logf.argtypes = [ctypes.c_int] * 3 + [_D, _D, ctypes.c_uint32, _D, _D]
        _lib.oracle_model_logf.restype = ctypes.c_double
        _lib.oracle_model_logmu.argtypes = [ctypes.c_int] * 3 + [_D, _D, _D]
        _lib.oracle_model_logmu.restype = ctypes.c_double
        _lib.oracle_logz_fixed.argtypes = [ctypes.c_int] * 6 + [ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_uint32, _D, _D, _D, _I, _I, _D]
        _lib.oracle_fisher_score.argtypes = [ctypes.c_int] * 6 + [ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_uint32, _D, _D, _D, _I, _I, ctypes.c_int, _D]
        _lib.oracle_pmmh_langevin.argtypes = [ctypes.c_int] * 6 + [ctypes.c_int, ctypes.c_double,
                                              ctypes.c_uint64, ctypes.c_uint32, _D, _D, ctypes.c_int,
                                              _D, _D, _D, _D, _D, _D, ctypes.c_uint32, ctypes.c_int,
                                              _D, _D, _I]
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _ip(a):
    return None if a is None else a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def philox(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block for counter ctr[4] and key key[2]."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox(c.ctypes.data_as(_U), k.ctypes.data_as(_U), out.ctypes.data_as(_U))
    return out


def _model_data(model_data):
    return _f64(model_data if model_data is not None else np.zeros(1))


def airpf(model, theta, y, *, m, M, mode=MODE_ADAPTIVE, tau=0.3, dx=1, dy=1, seed=0, chain=0,
          iter=0, model_data=None, record=True, tie_rel=1e-12, moments=False, tau_int=0.0, radix=2,
          tie_masks=False):
    """Literal Algorithm 1 (FP64).  Returns a dict with log_z and, if record,
    logz_trace[T], anc[T, N], src[T, m], enf[T, S_r+1], sstar[T], xfinal[N, dx], tie, where
    S_r = log_radix(m) is the number of interaction stages and s* counts them.
    tie_rel: relative width of the band around a threshold in which a draw, an island
    choice or an ENF test is flagged as a tie (a diagnostic; the arithmetic is unchanged).
    moments: also return moments[T, 2, 2, dx], the output measures of the paper's output-
    measure equation at step t: [0] the prediction filter (the mutated particles weighted by
    W_{t,0}), [1] the filter after internal resampling (weighted by W_{t,1}); [., 0] E[x_d],
    [., 1] E[x_d^2].
    tau_int: adaptive internal resampling (an island resamples only when the ESS of its
    particle weights is below tau_int M); 0 resamples at every step.
    radix: interactions over groups of radix islands (a power of 2; m a power of it): each
    stage averages every group of r islands and each island draws one member of its group
    with probability proportional to the weights.
    tie_masks: also return tie_draw[T, N] (internal draw j of island k, index k*M+j, within
    the tie band), tie_src[T, m] (a tied island choice on the walk that gives island k its
    block) and tie_step[T] (a tied ENF test), as booleans."""
    lib().oracle_set_tie_rel(tie_rel)
    lib().oracle_set_tau_int(tau_int)
    lib().oracle_set_radix(radix)
    y = _f64(y)
    T = len(y) // dy
    mom = np.zeros((T, 2, 2, dx)) if moments else None
    lib().oracle_set_moments_out(_dp(mom))
    masks = None
    if tie_masks:
        masks = dict(tie_draw=np.zeros((T, m * M), np.uint8), tie_src=np.zeros((T, m), np.uint8),
                     tie_step=np.zeros(T, np.uint8))
        lib().oracle_set_tie_masks(masks["tie_draw"].ctypes.data, masks["tie_src"].ctypes.data,
                                   masks["tie_step"].ctypes.data)
    S = int(round(math.log2(m))) // max(1, int(round(math.log2(radix))))
    N = m * M
    th, md = _f64(theta), _model_data(model_data)
    lz = np.zeros(1)
    tie = np.zeros(2, dtype=np.int32)
    out = dict()
    if record:
        out = dict(logz_trace=np.zeros(T), anc=np.zeros((T, N), np.int32),
                   src=np.zeros((T, m), np.int32), enf=np.zeros((T, S + 1)),
                   sstar=np.zeros(T, np.int32), xfinal=np.zeros((N, dx)))
    rc = lib().oracle_airpf(model, dx, dy, m, M, T, mode, tau, seed, chain, iter,
                            _dp(th), _dp(md), _dp(y), _dp(lz), _dp(out.get("logz_trace")),
                            _ip(out.get("anc")), _ip(out.get("src")), _dp(out.get("enf")),
                            _ip(out.get("sstar")), _dp(out.get("xfinal")), _ip(tie))
    lib().oracle_set_tie_rel(1e-12)
    lib().oracle_set_moments_out(None)
    lib().oracle_set_tie_masks(None, None, None)
    lib().oracle_set_tau_int(0.0)
    lib().oracle_set_radix(2)
    if rc:
        raise ValueError("oracle_airpf rejected its arguments")
    if moments:
        out["moments"] = mom
    if masks:
        out.update({k: v.astype(bool) for k, v in masks.items()})
    out["log_z"] = float(lz[0])
    out["tie"] = (int(tie[0]), int(tie[1]))
    return out


def airpf_batch(model, theta, y, *, m, M, runs, mode=MODE_ADAPTIVE, tau=0.3, dx=1, dy=1,
                seed=0, chain0=0, iter=0, model_data=None, tau_int=0.0, radix=2) -> np.ndarray:
    """log Z of `runs` independent AIRPF runs keyed by chains chain0, chain0+1, ..."""
    y = _f64(y)
    T = len(y) // dy
    out = np.zeros(runs)
    lib().oracle_set_tau_int(tau_int)
    lib().oracle_set_radix(radix)
    rc = lib().oracle_airpf_batch(model, dx, dy, m, M, T, mode, tau, seed, chain0, iter, runs,
                                  _dp(_f64(theta)), _dp(_model_data(model_data)), _dp(y), _dp(out))
    lib().oracle_set_tau_int(0.0)
    lib().oracle_set_radix(2)
    if rc:
        raise ValueError("oracle_airpf_batch rejected its arguments")
    return out


def bpf(model, theta, y, *, M, dx=1, dy=1, seed=0, chain=0, iter=0, unit0=0, model_data=None):
    """Bootstrap particle filter (the m = 1 case).  Returns (log_z, anc[T, M], tie)."""
    y = _f64(y)
    T = len(y) // dy
    th, md = _f64(theta), _model_data(model_data)
    lz = np.zeros(1)
    anc = np.zeros((T, M), np.int32)
    tie = np.zeros(2, dtype=np.int32)
    rc = lib().oracle_bpf(model, dx, dy, M, T, seed, chain, iter, unit0, _dp(th), _dp(md),
                          _dp(y), _dp(lz), _ip(anc), _ip(tie))
    if rc:
        raise ValueError("oracle_bpf rejected its arguments")
    return float(lz[0]), anc, (int(tie[0]), int(tie[1]))


def pmmh(model, theta0, y, *, m, M, step, lo, hi, iters, mode=MODE_ADAPTIVE, tau=0.3, dx=1,
         dy=1, seed=0, chain=0, model_data=None, iter0=0, state_logz=float("nan")):
    """Random-walk PMMH with AIRPF likelihood estimates.  Returns dict with
    theta[iters, d], logz[iters], n_accept, final theta and log Z (for resume)."""
    y = _f64(y)
    T = len(y) // dy
    th = _f64(theta0).copy()
    d = len(th)
    md = _model_data(model_data)
    st = np.array([state_logz], dtype=np.float64)
    tr = np.zeros((iters, d))
    lz = np.zeros(iters)
    nacc = np.zeros(1, np.int32)
    rc = lib().oracle_pmmh(model, dx, dy, m, M, T, mode, tau, seed, chain, _dp(md), _dp(y), d,
                           _dp(_f64(step)), _dp(_f64(lo)), _dp(_f64(hi)), _dp(th), _dp(st),
                           iter0, iters, _dp(tr), _dp(lz), _ip(nacc))
    if rc:
        raise ValueError("oracle_pmmh rejected its arguments")
    return dict(theta=tr, logz=lz, n_accept=int(nacc[0]), theta_final=th,
                logz_final=float(st[0]))


def model_logg(model, theta, y, x, *, dx=1, dy=1, model_data=None) -> float:
    return lib().oracle_model_logg(model, dx, dy, _dp(_f64(theta)), _dp(_model_data(model_data)),
                                   _dp(_f64(y)), _dp(_f64(x)))


def model_prior(model, theta, *, unit, dx=1, dy=1, seed=0, chain=0, iter=0, model_data=None):
    x = np.zeros(dx)
    lib().oracle_model_prior(model, dx, dy, _dp(_f64(theta)), _dp(_model_data(model_data)), seed,
                             chain, iter, unit, _dp(x))
    return x


def model_step(model, theta, xp, *, unit, t, dx=1, dy=1, seed=0, chain=0, iter=0,
               model_data=None):
    x = np.zeros(dx)
    lib().oracle_model_step(model, dx, dy, _dp(_f64(theta)), _dp(_model_data(model_data)), seed,
                            chain, iter, unit, t, _dp(_f64(xp)), _dp(x))
    return x


def model_valid(model, theta, dx=1) -> bool:
    return bool(lib().oracle_model_valid(model, dx, _dp(_f64(theta))))


def model_logf(model, theta, xp, x, *, t=1, dx=1, dy=1, model_data=None) -> float:
    """log f_t(x | xp), the transition density."""
    return lib().oracle_model_logf(model, dx, dy, _dp(_f64(theta)), _dp(_model_data(model_data)), t,
                                   _dp(_f64(xp)), _dp(_f64(x)))


def model_logmu(model, theta, x, *, dx=1, dy=1, model_data=None) -> float:
    """log pi_0(x), the prior density of x_0."""
    return lib().oracle_model_logmu(model, dx, dy, _dp(_f64(theta)), _dp(_model_data(model_data)),
                                    _dp(_f64(x)))


def logz_fixed(model, theta, y, anc, sstar, *, m, M, dx=1, dy=1, seed=0, chain=0, iter=0,
               model_data=None, radix=2) -> float:
    """log Z of a run with its random numbers, lineage anc [T, N] and s* [T] held fixed,
    as a function of theta (FP64).  radix: the run's (s* counts stages of r islands)."""
    y = _f64(y)
    T = len(y) // dy
    anc = np.ascontiguousarray(np.asarray(anc, dtype=np.int32).reshape(T, m * M))
    sstar = np.ascontiguousarray(np.asarray(sstar, dtype=np.int32).reshape(T))
    out = np.zeros(1)
    lib().oracle_set_radix(radix)
    rc = lib().oracle_logz_fixed(model, dx, dy, m, M, T, seed, chain, iter, _dp(_f64(theta)),
                                 _dp(_model_data(model_data)), _dp(y), _ip(anc), _ip(sstar), _dp(out))
    lib().oracle_set_radix(2)
    if rc:
        raise ValueError("oracle_logz_fixed rejected its arguments")
    return float(out[0])


def logz_fixed_gradient(model, theta, y, anc, sstar, *, h=1e-5, **kw) -> np.ndarray:
    """Gradient of logz_fixed in every component of theta: central differences D(h) and
    D(h/2) (step h max(1, |theta_d|)) combined by one Richardson step, (4 D(h/2) - D(h)) / 3,
    which cancels the h^2 term of the central-difference error (Richardson, 1911).  A
    plain central difference at h = 1e-5 was off by 1e-4 relative on a nonlinear-growth
    path whose log Z bends sharply in q."""
    th = _f64(theta).copy()
    g = np.zeros(len(th))

    def central(d, hd):
        tp, tm = th.copy(), th.copy()
        tp[d] += hd
        tm[d] -= hd
        return (logz_fixed(model, tp, y, anc, sstar, **kw) - logz_fixed(model, tm, y, anc, sstar, **kw)) / (2 * hd)

    for d in range(len(th)):
        hd = h * max(1.0, abs(th[d]))
        g[d] = (4.0 * central(d, hd / 2) - central(d, hd)) / 3.0
    return g


def fisher_score(model, theta, y, anc, sstar, *, m, M, dx=1, dy=1, seed=0, chain=0, iter=0,
                 model_data=None, radix=2) -> np.ndarray:
    """Fisher-identity score along the lineages of a run (FP64); radix as for logz_fixed."""
    y = _f64(y)
    T = len(y) // dy
    th = _f64(theta)
    anc = np.ascontiguousarray(np.asarray(anc, dtype=np.int32).reshape(T, m * M))
    sstar = np.ascontiguousarray(np.asarray(sstar, dtype=np.int32).reshape(T))
    out = np.zeros(len(th))
    lib().oracle_set_radix(radix)
    rc = lib().oracle_fisher_score(model, dx, dy, m, M, T, seed, chain, iter, _dp(th),
                                   _dp(_model_data(model_data)), _dp(y), _ip(anc), _ip(sstar), len(th),
                                   _dp(out))
    lib().oracle_set_radix(2)
    if rc:
        raise ValueError("oracle_fisher_score rejected its arguments")
    return out


def pmmh_langevin(model, theta0, y, *, m, M, step, lo, hi, iters, mode=MODE_ADAPTIVE, tau=0.3, dx=1,
                  dy=1, seed=0, chain=0, model_data=None, iter0=0, state_logz=float("nan"), state_grad=None):
    """PMMH with the Langevin proposal driven by the Fisher score.  Returns dict with
    theta[iters, d], logz[iters], n_accept and the final theta, log Z and score (for resume)."""
    y = _f64(y)
    T = len(y) // dy
    th = _f64(theta0).copy()
    d = len(th)
    md = _model_data(model_data)
    st = np.array([state_logz], dtype=np.float64)
    g = np.zeros(d) if state_grad is None else _f64(state_grad).copy()
    tr = np.zeros((iters, d))
    lz = np.zeros(iters)
    nacc = np.zeros(1, np.int32)
    rc = lib().oracle_pmmh_langevin(model, dx, dy, m, M, T, mode, tau, seed, chain, _dp(md), _dp(y), d,
                                    _dp(_f64(step)), _dp(_f64(lo)), _dp(_f64(hi)), _dp(th), _dp(st), _dp(g),
                                    iter0, iters, _dp(tr), _dp(lz), _ip(nacc))
    if rc:
        raise ValueError("oracle_pmmh_langevin rejected its arguments")
    return dict(theta=tr, logz=lz, n_accept=int(nacc[0]), theta_final=th, logz_final=float(st[0]), grad_final=g)
