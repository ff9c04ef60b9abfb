// airpf_static.cu -- airpf_run_static: one filter pass with no context and no
// device allocation.  The pass runs the same kernels as airpf_run, on a scratch
// area of fixed size that this file holds as a device array of its own, and on
// the caller's buffers for theta, y, the model data and log Z.  The paper has no
// counterpart; this is a deployment entry point (see include/airpf.h).
//
// Scratch layout (256-byte aligned pieces, for the B filters of one call):
//   run parameters | X[0] X[1] particle stores | CTA records pe, pt, pq (x2) |
//   cascade summary csum, cup, nsrc | model constants | NGM drift table |
//   barrier and error words
// No piece has to start at zero: every word a pass reads it has written
// earlier in the same pass, and its first kernel clears the barrier and error
// words.
#include <cstring>
#include <mutex>

#include "../../include/airpf.h"
#include "airpf_internal.h"

using airpf::RunParams;
using airpf::StepParams;

namespace {

constexpr size_t kStaticScratchBytes = AIRPF_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[kMaxDevices];      // device address of the scratch, per device

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct StaticLayout {
    size_t run, X[2], pe[2], pt[2], pq[2], csum, cup, nsrc, mpar, drift, bar, total;
};

StaticLayout static_layout(const airpf_config* c)
{
    StaticLayout L;
    const size_t B = c->B, N = (size_t)c->m * c->M;
    const size_t rsz = c->precision == AIRPF_FP64 ? 8 : 4;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L.run = take(sizeof(RunParams));
    for (int i = 0; i < 2; ++i) L.X[i] = take(rsz * B * c->dx * N);
    for (int i = 0; i < 2; ++i) L.pe[i] = take(sizeof(int) * B * c->m);
    for (int i = 0; i < 2; ++i) L.pt[i] = take(sizeof(double) * B * 2 * c->m);
    for (int i = 0; i < 2; ++i) L.pq[i] = take(sizeof(double) * B * c->m * 8);
    L.csum = take(sizeof(int) * 4 * B);
    L.cup = take(sizeof(unsigned long long) * B * c->m);
    L.nsrc = take(sizeof(int) * B * c->m);
    L.mpar = take(airpf::model_par_bytes() * B);
    L.drift = take(sizeof(double) * (size_t)c->T);
    L.bar = take(sizeof(unsigned) * 4);
    L.total = o;
    return L;
}

// Device address of the scratch on the current device, looked up once per
// device (the lookup also loads this file's module, which holds the scratch).
airpf_status scratch_on_current_device(unsigned char** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        airpf::set_create_error("airpf_run_static: cudaGetDevice: %s", cudaGetErrorString(e));
        return AIRPF_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        airpf::set_create_error("airpf_run_static: device %d is beyond the %d devices it serves", dev, kMaxDevices);
        return AIRPF_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            airpf::set_create_error("airpf_run_static: cudaGetSymbolAddress of the scratch: %s",
                                    cudaGetErrorString(e));
            return AIRPF_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return AIRPF_OK;
}

airpf_status launch_failed(cudaError_t e, const char* what)
{
    airpf::set_create_error("airpf_run_static: %s: %s", what, cudaGetErrorString(e));
    return AIRPF_ERR_CUDA;
}

}  // namespace

extern "C" airpf_status airpf_run_static(const airpf_config* cfg, const double* d_theta, const double* d_y,
                                         const double* d_model_data, uint32_t chain0, uint32_t iter,
                                         double* d_log_z, void* stream)
{
    size_t ws = 0;
    airpf_status s = airpf_workspace_bytes(cfg, &ws);       // validates the configuration
    if (s != AIRPF_OK) return s;
    if (!d_theta || !d_y || !d_log_z) {
        airpf::set_create_error("airpf_run_static: theta, y and log_z are required");
        return AIRPF_ERR_ARG;
    }
    if (cfg->model == AIRPF_MODEL_LGSSM && !d_model_data) {
        airpf::set_create_error("airpf_run_static: LGSSM needs d_model_data (A and C)");
        return AIRPF_ERR_ARG;
    }
    if (cfg->record != 0) {
        airpf::set_create_error("airpf_run_static records nothing: record must be 0 (use a context)");
        return AIRPF_ERR_ARG;
    }
    if (cfg->launch == AIRPF_LAUNCH_PERSISTENT_GRID) {
        airpf::set_create_error("airpf_run_static runs AUTO, STEPS or PERSISTENT_CTA launches only");
        return AIRPF_ERR_UNSUPPORTED;
    }
    if (cfg->tau_int > 0.0) {
        airpf::set_create_error("airpf_run_static resamples every island at every step: tau_int must be 0");
        return AIRPF_ERR_UNSUPPORTED;
    }
    if (cfg->ppt != 0 || cfg->islands_per_cta != 0 || cfg->launch == AIRPF_LAUNCH_STEPS_SPLIT) {
        airpf::set_create_error("airpf_run_static takes the default tiling and launch forms: ppt and "
                                "islands_per_cta must be 0, launch not STEPS_SPLIT");
        return AIRPF_ERR_UNSUPPORTED;
    }
    if ((uint64_t)chain0 + (uint64_t)cfg->B > (1u << 24)) {
        airpf::set_create_error("airpf_run_static: chain0 + B must not exceed 2^24");
        return AIRPF_ERR_ARG;
    }
    const StaticLayout L = static_layout(cfg);
    if (L.total > kStaticScratchBytes) {
        airpf::set_create_error("airpf_run_static: this configuration needs %zu bytes of scratch, above the "
                                "%zu-byte static scratch; use airpf_create with a workspace of its own",
                                L.total, kStaticScratchBytes);
        return AIRPF_ERR_WORKSPACE;
    }
    unsigned char* base = nullptr;
    if ((s = scratch_on_current_device(&base)) != AIRPF_OK) return s;

    StepParams p;
    std::memset(&p, 0, sizeof(p));
    p.rb = 1;
    while (cfg->radix > 2 && (1 << p.rb) < cfg->radix) ++p.rb;
    p.B = cfg->B; p.m = cfg->m; p.M = cfg->M; p.N = cfg->m * cfg->M; p.dx = cfg->dx; p.dy = cfg->dy;
    p.T = cfg->T; p.mode = cfg->mode; p.model = cfg->model;
    while ((1 << p.S) < cfg->m) ++p.S;
    p.fp64 = cfg->precision == AIRPF_FP64;
    p.tau = cfg->tau;
    p.inv_M = 1.0 / (double)cfg->M;
    p.tau_f = (float)cfg->tau;
    {
        int lg = 0;
        while ((1 << lg) < cfg->M) ++lg;
        p.cdf_bits = 31 - lg;
        p.cdf_scale = ldexpf(1.0f, p.cdf_bits);
    }
    // one CTA per filter when a filter fits one, else one launch per step
    bool cta = false;
    if (cfg->launch == AIRPF_LAUNCH_AUTO || cfg->launch == AIRPF_LAUNCH_PERSISTENT_CTA) {
        airpf::choose_mapping(cfg->m, cfg->M, p.fp64, 0, cfg->m, &p.tpi, &p.ppt, &p.G);
        cta = p.G == cfg->m && p.G * p.tpi <= airpf::max_cta_threads();
        if (!cta && cfg->launch == AIRPF_LAUNCH_PERSISTENT_CTA) {
            airpf::set_create_error("airpf_run_static: a filter of m=%d x M=%d does not fit one CTA", cfg->m, cfg->M);
            return AIRPF_ERR_UNSUPPORTED;
        }
    }
    if (!cta) airpf::choose_mapping(cfg->m, cfg->M, p.fp64, 0, 0, &p.tpi, &p.ppt, &p.G);
    p.P = cfg->m / p.G;
    while ((1 << p.g) < p.G) ++p.g;
    while ((1 << p.lg_tpi) < p.tpi) ++p.lg_tpi;
    if (airpf::step_smem_bytes(p) > 227 * 1024) {
        airpf::set_create_error("airpf_run_static: a step needs %zu bytes of shared memory (%d CTAs per filter), "
                                "above 227 KB; use a context with AIRPF_LAUNCH_STEPS_SPLIT",
                                airpf::step_smem_bytes(p), p.P);
        return AIRPF_ERR_UNSUPPORTED;
    }
    p.theta_dim = airpf_theta_dim(cfg->model, cfg->dx);
    p.seed_lo = (uint32_t)(cfg->seed & 0xffffffffu);
    p.seed_hi = (uint32_t)(cfg->seed >> 32);
    p.run = reinterpret_cast<RunParams*>(base + L.run);
    p.theta = d_theta;
    p.mdata = d_model_data;
    p.y = d_y;
    p.active = nullptr;
    p.mpar = base + L.mpar;
    p.drift = base + L.drift;
    p.bar = reinterpret_cast<unsigned*>(base + L.bar);
    p.err = p.bar + 2;
    for (int i = 0; i < 2; ++i) {
        p.X[i] = base + L.X[i];
        p.pe[i] = reinterpret_cast<int*>(base + L.pe[i]);
        p.pt[i] = base + L.pt[i];
        p.pq[i] = base + L.pq[i];
        p.ires[i] = nullptr;
    }
    p.csum = reinterpret_cast<int*>(base + L.csum);
    p.cup = base + L.cup;
    p.nsrc = reinterpret_cast<int*>(base + L.nsrc);
    p.logz = d_log_z;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = airpf::prepare_step(p);
    if (e != cudaSuccess) return launch_failed(e, "kernel attribute setup");
    e = airpf::launch_set_run(reinterpret_cast<RunParams*>(base + L.run), iter, chain0, st);
    if (e != cudaSuccess) return launch_failed(e, "run parameter launch");
    if (cta) {
        e = airpf::launch_step(p, 0, st);
        if (e == cudaSuccess) e = airpf::launch_persistent(p, false, st);
        if (e != cudaSuccess) return launch_failed(e, "persistent launch");
        return AIRPF_OK;
    }
    for (int t = 0; t <= cfg->T + 1; ++t) {
        e = airpf::launch_step(p, t, st);
        if (e == cudaSuccess && t >= 1 && t <= cfg->T) e = airpf::launch_cascade(p, t, st);
        if (e != cudaSuccess) return launch_failed(e, "step launch");
    }
    return AIRPF_OK;
}
