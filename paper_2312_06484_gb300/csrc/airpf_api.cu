// airpf_api.cu -- C ABI of the AIRPF library (see include/airpf.h).
//
// Host runtime: checks arguments, carves the caller's device workspace into
// the particle stores and island-weight buffers, captures the T+1 step
// launches of one filter pass into a CUDA graph once per context, and replays
// it on the caller's stream.  The graph reads every per-call value (theta, y,
// iter, chain0) from fixed workspace addresses, so one capture serves all
// calls, including every PMMH iteration.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/airpf.h"
#include "airpf_internal.h"

using airpf::RunParams;
using airpf::StepParams;

namespace {

thread_local char g_create_error[512] = "";

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int ilog2_exact(int m)
{
    int s = 0;
    while ((1 << s) < m) ++s;
    return (1 << s) == m ? s : -1;
}

// Byte offsets of every buffer inside the workspace.
struct WsLayout {
    size_t tick, ge[2], gtr[2], gqs[2];
    size_t run, theta, mdata, y, X[2], pe[2], pt[2], pq[2], csum, cup, nsrc, utg, ires[2], logz, trace, enf,
        sstar, anc, active, mpar, drift, bar;
    size_t pm_prop, pm_logz_prop, pm_stats, pm_gprop, pm_lqf;
    size_t xck, xblk, logw, gpi[2], xh[3], dh[3], gout, sout, gacc;   // gradient pass
    size_t fw, fsum;                                             // output measures
    size_t lom[2];                                               // adaptive internal resampling
    int fm_nw;
    size_t total;
};

}  // namespace

struct airpf_ctx {
    airpf_config cfg;
    double md_host[airpf::kModelDataMax];   // LGSSM A and C (host copy, for the backward pass)
    int S, N, theta_dim;
    unsigned char* ws;
    size_t ws_bytes;
    WsLayout L;
    cudaStream_t stream;
    cudaStream_t cap_stream;
    cudaGraphExec_t graph;
    bool graph_ready;
    cudaGraphExec_t graph_pm;   // the same pass with per-filter active flags (PMMH)
    bool graph_pm_ready;
    cudaGraphExec_t graph_bwd;  // the backward pass of the gradient
    bool graph_bwd_ready;
    cudaStream_t bwd_aux;       // the backward pass's second capture stream (recomputation)
    cudaEvent_t bwd_ev[airpf::kGradEvents];
    bool bwd_aux_ready;
    int launch;               // resolved airpf_launch
    StepParams sp;
    StepParams sp_pm;
    cudaEvent_t* ev;          // AIRPF_RECORD_TIMING: 4 events per step (island kernel, cascade kernel)
    int n_ev;
    int64_t launches;
    char err[512];
};

namespace {

int theta_dim_of(int model, int dx)
{
    switch (model) {
    case AIRPF_MODEL_AR1: return 4;
    case AIRPF_MODEL_SV: return 3;
    case AIRPF_MODEL_NGM: return 3;
    case AIRPF_MODEL_LGSSM: return dx + 2;
    case AIRPF_MODEL_TOY: return 2;
    case AIRPF_MODEL_CP: return 3;
    }
    return 0;
}

const char* check_config(const airpf_config* c)
{
    if (!c) return "config is NULL";
    if (c->model < 0 || c->model > 5) return "unknown model";
    if (c->model == AIRPF_MODEL_LGSSM) {
        if (c->dx < 1 || c->dx > 8 || c->dy < 1 || c->dy > 8) return "LGSSM needs 1 <= dx, dy <= 8";
    } else if (c->model == AIRPF_MODEL_CP) {
        if (c->dx != 1 || c->dy != 2) return "the change-point model needs dx = 1, dy = 2 (y_t = (k_t, n_t))";
    } else if (c->dx != 1 || c->dy != 1) {
        return "scalar models need dx = dy = 1";
    }
    if (c->m < 1 || c->m > 65536 || ilog2_exact(c->m) < 0) return "m must be a power of 2 in [1, 65536]";
    if (c->M < 1 || c->M > 1024) return "M must be in [1, 1024]";
    if (c->T < 1 || c->T > (1 << 24)) return "T must be in [1, 2^24]";
    if (c->B < 1 || c->B > (1 << 24)) return "B must be in [1, 2^24]";
    if ((double)c->B * c->m * c->M > 2147483647.0) return "B * m * M must be below 2^31";
    if ((double)c->m * c->M > 4294967295.0) return "m * M must fit the 32-bit particle counter";
    if (c->mode < 0 || c->mode > 2) return "unknown interaction mode";
    if (!(c->tau > 0.0 && c->tau <= 1.0)) return "tau must be in (0, 1]";
    if (c->precision != AIRPF_FP64 && c->precision != AIRPF_FP32_MIXED) return "unknown precision";
    if (c->record < 0 || c->record > 63) return "unknown record bits";
    if (c->ckpt < 0 || c->ckpt > c->T) return "ckpt must be in [0, T]";
    if (!(c->tau_int >= 0.0 && c->tau_int <= 1.0)) return "tau_int must be in [0, 1]";
    if (c->radix != 0) {
        if (c->radix < 2 || (c->radix & (c->radix - 1))) return "radix must be 0 or a power of 2";
        int b = 0;
        while ((1 << b) < c->radix) ++b;
        if (ilog2_exact(c->m) % b != 0) return "m must be a power of the radix";
    }
    if (c->launch < 0 || c->launch > 4) return "unknown launch mode";
    if (c->reserved != 0) return "reserved must be 0";
    if (c->ppt != 0 && c->ppt != 2 && c->ppt != 4 && c->ppt != 8) return "ppt must be 0, 2, 4 or 8";
    if (c->ppt == 8 && !(c->precision == AIRPF_FP32_MIXED && (c->model == AIRPF_MODEL_SV || c->model == AIRPF_MODEL_NGM)))
        return "ppt = 8 is compiled for the FP32 SV and NGM filters only";
    if (c->islands_per_cta < 0 || c->islands_per_cta > 4096 || (c->islands_per_cta & (c->islands_per_cta - 1)))
        return "islands_per_cta must be 0 or a power of 2";
    return nullptr;
}

// binary stages per interaction stage: radix r = 2^b (0 and 2 both mean r = 2)
static int radix_bits(const airpf_config* c)
{
    int b = 1;
    while (c->radix > 2 && (1 << b) < c->radix) ++b;
    return b;
}

WsLayout make_ws_layout(const airpf_config* c)
{
    WsLayout L;
    const size_t B = c->B, N = (size_t)c->m * c->M, T = c->T;
    const size_t S = (size_t)ilog2_exact(c->m);
    const size_t rsz = c->precision == AIRPF_FP64 ? 8 : 4;
    const bool grad = c->record & AIRPF_RECORD_GRAD;
    const bool lin = (c->record & AIRPF_RECORD_LINEAGE) || grad;    // the gradient pass needs the
    const bool enf = (c->record & AIRPF_RECORD_ENF) || grad;        // lineage and s* of the run
    const bool tr = c->record & AIRPF_RECORD_TRACE;
    const size_t td = (size_t)theta_dim_of(c->model, c->dx);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L.run = take(sizeof(RunParams));
    L.theta = take(sizeof(double) * B * td);
    L.mdata = take(sizeof(double) * (size_t)(c->dx * c->dx + c->dy * c->dx));
    L.y = take(sizeof(double) * T * c->dy);
    for (int i = 0; i < 2; ++i) L.X[i] = take(rsz * B * c->dx * N);
    // CTA records: at most m of them (one island per CTA), each a subtree of 2G nodes
    for (int i = 0; i < 2; ++i) L.pe[i] = take(sizeof(int) * B * c->m);
    for (int i = 0; i < 2; ++i) L.pt[i] = take(sizeof(double) * B * 2 * c->m);
    for (int i = 0; i < 2; ++i) L.pq[i] = take(sizeof(double) * B * c->m * 8);
    L.csum = take(sizeof(int) * 4 * B);
    L.cup = take(sizeof(unsigned long long) * B * c->m);
    L.nsrc = take(sizeof(int) * B * c->m);
    L.utg = take(sizeof(double) * B * 2 * c->m);
    // split steps' group cascade: at most max(1, m / 2^7) groups of at most 2^7 CTA records
    {
        const size_t ngmax = c->m >> airpf::kTailGroupLog > 0 ? (size_t)(c->m >> airpf::kTailGroupLog) : 1;
        L.tick = take(sizeof(unsigned) * B);
        for (int i = 0; i < 2; ++i) {
            L.ge[i] = take(sizeof(int) * B * ngmax);
            L.gtr[i] = take(sizeof(double) * B * 2 * c->m);
            L.gqs[i] = take(sizeof(double) * B * ngmax * 16);
        }
    }
    for (int i = 0; i < 2; ++i) L.ires[i] = lin ? take(sizeof(int) * B * N) : 0;
    L.logz = take(sizeof(double) * B);
    L.trace = tr ? take(sizeof(double) * B * T) : 0;
    L.enf = enf ? take(sizeof(double) * B * T * (S / radix_bits(c) + 1)) : 0;
    L.sstar = enf ? take(sizeof(int) * B * T) : 0;
    L.anc = lin ? take(sizeof(int) * B * T * N) : 0;
    L.active = take(sizeof(int) * B);
    L.mpar = take(airpf::model_par_bytes() * B);
    L.drift = take(sizeof(double) * T);
    L.bar = take(sizeof(unsigned) * 4);
    L.pm_prop = take(sizeof(double) * B * td);
    L.pm_logz_prop = take(sizeof(double) * B);
    L.pm_stats = take(sizeof(int) * B);
    L.pm_gprop = take(sizeof(double) * B * td);
    L.pm_lqf = take(sizeof(double) * B);
    L.xck = L.xblk = L.logw = L.gout = L.sout = L.gacc = 0;
    for (int i = 0; i < 3; ++i) L.xh[i] = L.dh[i] = 0;
    L.gpi[0] = L.gpi[1] = 0;
    if (grad) {
        const size_t K = c->ckpt > 0 ? (size_t)c->ckpt : 1;
        const size_t nck = T / K + 1 + (T % K != 0 ? 1 : 0);
        const size_t dxs = c->model == AIRPF_MODEL_LGSSM ? 8 : (size_t)c->dx;   // states [N][dx padded]
        L.xck = take(rsz * B * nck * dxs * N);
        L.xblk = take(rsz * 2 * B * K * dxs * N);     // two blocks: one recomputed while the other is used
        L.logw = take(sizeof(double) * B * T * c->m);
        for (int i = 0; i < 2; ++i) L.gpi[i] = take(sizeof(double) * B * c->m);
        const size_t dxp = c->model == AIRPF_MODEL_LGSSM ? 8 : (size_t)c->dx;   // adjoints padded per particle
        for (int i = 0; i < 3; ++i) L.xh[i] = take(rsz * B * dxp * N);
        for (int i = 0; i < 3; ++i) L.dh[i] = take(rsz * B * N);
        L.gout = take(sizeof(double) * B * td);
        L.sout = take(sizeof(double) * B * td);
        L.gacc = take(sizeof(double) * B * c->m * 2 * 10);   // 2 x kMaxTheta (8 + 2) per island
    }
    L.lom[0] = L.lom[1] = 0;
    if (c->tau_int > 0.0)
        for (int i = 0; i < 2; ++i) L.lom[i] = take(rsz * B * N);
    L.fw = L.fsum = 0;
    L.fm_nw = 0;
    if (c->record & AIRPF_RECORD_MOMENTS) {
        // warps per island: the threads per island depend only on M and the particles per
        // thread (the requested count, or the default and the small-grid choice of two)
        int tpi = 0, pp = 0, G = 0, tpi2 = 0;
        airpf::choose_mapping(c->m, c->M, c->precision == AIRPF_FP64, c->ppt, 0, &tpi, &pp, &G);
        if (c->ppt == 0) airpf::choose_mapping(c->m, c->M, c->precision == AIRPF_FP64, 2, 1, &tpi2, &pp, &G);
        L.fm_nw = (tpi > tpi2 ? tpi : tpi2) / 32;
        L.fw = take(sizeof(double) * B * T * c->m * 2);
        L.fsum = take(sizeof(double) * B * T * c->m * L.fm_nw * 4 * c->dx);
    }
    L.total = o;
    return L;
}

void set_err(airpf_ctx* ctx, const char* fmt, ...)
{
    char* dst = ctx ? ctx->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
}

airpf_status cuda_fail(airpf_ctx* ctx, cudaError_t e, const char* what)
{
    set_err(ctx, "%s: %s", what, cudaGetErrorString(e));
    return AIRPF_ERR_CUDA;
}

bool is_steps(int launch) { return launch == AIRPF_LAUNCH_STEPS || launch == AIRPF_LAUNCH_STEPS_SPLIT; }

template <typename T> T* at(airpf_ctx* ctx, size_t off) { return reinterpret_cast<T*>(ctx->ws + off); }

airpf_status build_graph(airpf_ctx* ctx, const StepParams& p, cudaGraphExec_t* graph, bool* ready)
{
    if (*ready) return AIRPF_OK;
    cudaError_t e = airpf::prepare_step(p);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel attribute setup");
    e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    cudaError_t le = cudaSuccess;
    // timing: event-record nodes around each kernel of steps 1..T (plain graph
    // only), with plain stream-order edges between the kernels
    const bool timed = ctx->ev && graph == &ctx->graph;
    StepParams q = p;
    if (timed) q.pdl = 0;
    auto mark = [&](int t, int which) {
        if (timed && le == cudaSuccess && t >= 1 && t <= ctx->cfg.T)
            le = cudaEventRecordWithFlags(ctx->ev[4 * (t - 1) + which], ctx->cap_stream, cudaEventRecordExternal);
    };
    for (int t = 0; t <= ctx->cfg.T + 1 && le == cudaSuccess; ++t) {
        mark(t, 0);
        if (le == cudaSuccess) le = airpf::launch_step(q, t, ctx->cap_stream);
        mark(t, 1);
        mark(t, 2);
        if (le == cudaSuccess && !q.fused && t >= 1 && t <= ctx->cfg.T)
            le = airpf::launch_cascade(q, t, ctx->cap_stream);
        mark(t, 3);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, le, "step launch during capture");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    *ready = true;
    return AIRPF_OK;
}

// Enqueue one filter pass over the workspace inputs (theta, y, run params
// already set); pm selects the parameter block with per-filter active flags.
airpf_status enqueue_pass(airpf_ctx* ctx, bool pm = false)
{
    StepParams& p = pm ? ctx->sp_pm : ctx->sp;
    if (!is_steps(ctx->launch)) {
        cudaError_t e = airpf::launch_step(p, 0, ctx->stream);      // prologue
        if (e == cudaSuccess)
            e = airpf::launch_persistent(p, ctx->launch == AIRPF_LAUNCH_PERSISTENT_GRID, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "persistent launch");
        ctx->launches += 2;
        p.inject_stall = 0;
        return AIRPF_OK;
    }
    airpf_status s = pm ? build_graph(ctx, p, &ctx->graph_pm, &ctx->graph_pm_ready)
                        : build_graph(ctx, p, &ctx->graph, &ctx->graph_ready);
    if (s != AIRPF_OK) return s;
    cudaError_t e = cudaGraphLaunch(pm ? ctx->graph_pm : ctx->graph, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
    ctx->launches += (p.fused ? 1 : 2) * (int64_t)ctx->cfg.T + 2;
    return AIRPF_OK;
}

airpf_status copy_async(airpf_ctx* ctx, void* dst, const void* src, size_t bytes)
{
    if (bytes == 0) return AIRPF_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream);
    return e == cudaSuccess ? AIRPF_OK : cuda_fail(ctx, e, "cudaMemcpyAsync");
}

}  // namespace

namespace airpf {
cudaStream_t ctx_stream(const airpf_ctx* ctx) { return ctx->stream; }

void set_create_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_error, sizeof(g_create_error), fmt, ap);
    va_end(ap);
}
}  // namespace airpf

extern "C" {

airpf_status airpf_workspace_bytes(const airpf_config* cfg, size_t* bytes)
{
    const char* why = check_config(cfg);
    if (why || !bytes) {
        set_err(nullptr, "%s", why ? why : "bytes is NULL");
        return AIRPF_ERR_ARG;
    }
    *bytes = make_ws_layout(cfg).total;
    return AIRPF_OK;
}

int32_t airpf_theta_dim(int32_t model, int32_t dx) { return theta_dim_of(model, dx); }

airpf_status airpf_create(const airpf_config* cfg, void* d_workspace, size_t workspace_bytes,
                          const double* model_data, void* stream, airpf_ctx** out)
{
    if (!out) {
        set_err(nullptr, "out is NULL");
        return AIRPF_ERR_ARG;
    }
    *out = nullptr;
    const char* why = check_config(cfg);
    if (why) {
        set_err(nullptr, "%s", why);
        return AIRPF_ERR_ARG;
    }
    if (cfg->model == AIRPF_MODEL_LGSSM && !model_data) {
        set_err(nullptr, "LGSSM needs model_data (A and C)");
        return AIRPF_ERR_ARG;
    }
    if ((cfg->record & AIRPF_RECORD_GRAD) && !airpf::grad_supported(cfg->model)) {
        set_err(nullptr, "the gradient pass supports the AR1, SV, NGM and LGSSM models");
        return AIRPF_ERR_UNSUPPORTED;
    }
    if (cfg->tau_int > 0.0 && (cfg->record & (AIRPF_RECORD_GRAD | AIRPF_RECORD_MOMENTS))) {
        set_err(nullptr, "adaptive internal resampling (tau_int > 0) runs without the gradient and "
                         "output-measure records");
        return AIRPF_ERR_UNSUPPORTED;
    }
    const WsLayout L = make_ws_layout(cfg);
    if (!d_workspace || workspace_bytes < L.total || ((uintptr_t)d_workspace & 255u)) {
        set_err(nullptr, "workspace must be >= %zu bytes and 256-byte aligned", L.total);
        return AIRPF_ERR_WORKSPACE;
    }
    airpf_ctx* ctx = new (std::nothrow) airpf_ctx();
    if (!ctx) {
        set_err(nullptr, "host allocation failed");
        return AIRPF_ERR_ARG;
    }
    ctx->cfg = *cfg;
    ctx->S = ilog2_exact(cfg->m);
    ctx->N = cfg->m * cfg->M;
    ctx->theta_dim = theta_dim_of(cfg->model, cfg->dx);
    ctx->ws = static_cast<unsigned char*>(d_workspace);
    ctx->ws_bytes = workspace_bytes;
    ctx->L = L;
    ctx->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        set_err(nullptr, "cudaStreamCreate: %s", cudaGetErrorString(e));
        delete ctx;
        return AIRPF_ERR_CUDA;
    }

    StepParams& p = ctx->sp;
    std::memset(&p, 0, sizeof(p));
    p.B = cfg->B; p.m = cfg->m; p.M = cfg->M; p.N = ctx->N; p.dx = cfg->dx; p.dy = cfg->dy;
    p.T = cfg->T; p.S = ctx->S; p.mode = cfg->mode; p.model = cfg->model;
    p.fp64 = cfg->precision == AIRPF_FP64;
    p.tau = cfg->tau;
    p.inv_M = 1.0 / (double)cfg->M;
    p.tau_f = (float)cfg->tau;
    {
        int lg = 0;
        while ((1 << lg) < cfg->M) ++lg;
        p.cdf_bits = 31 - lg;                   // the CDF total stays below 2^31 + 1
        p.cdf_scale = ldexpf(1.0f, p.cdf_bits);
    }
    {
        // the island-to-thread mapping: requested particles per thread and
        // islands per CTA, or the defaults
        const int want_ppt = cfg->ppt;
        int want_g = cfg->islands_per_cta;
        int mode = cfg->launch;
        if (mode == AIRPF_LAUNCH_AUTO || mode == AIRPF_LAUNCH_PERSISTENT_CTA) {
            airpf::choose_mapping(cfg->m, cfg->M, p.fp64, want_ppt, cfg->m, &p.tpi, &p.ppt, &p.G);
            if (p.G == cfg->m && p.G * p.tpi <= airpf::max_cta_threads()) {
                mode = AIRPF_LAUNCH_PERSISTENT_CTA;
            } else if (mode == AIRPF_LAUNCH_PERSISTENT_CTA) {
                set_err(nullptr, "a filter of m=%d islands x M=%d does not fit one CTA", cfg->m, cfg->M);
                cudaStreamDestroy(ctx->cap_stream);
                delete ctx;
                return AIRPF_ERR_UNSUPPORTED;
            } else {
                mode = AIRPF_LAUNCH_AUTO;
            }
        }
        if (mode != AIRPF_LAUNCH_PERSISTENT_CTA) {
            airpf::choose_mapping(cfg->m, cfg->M, p.fp64, want_ppt, want_g, &p.tpi, &p.ppt, &p.G);
            if (p.G == cfg->m && cfg->m > 1 && p.G * p.tpi > 256) {
                want_g = cfg->m / 2;
                airpf::choose_mapping(cfg->m, cfg->M, p.fp64, want_ppt, want_g, &p.tpi, &p.ppt, &p.G);
            }
        }
        ctx->launch = mode;
        // per-step launches whose default tiling leaves SMs idle (fewer CTAs than SMs): two
        // particles per thread and one island per CTA spread the filters over more SMs
        // (measured 9-18% faster per pass for one filter of m = 64..256 islands).  Not for the
        // cooperative grid (every grid barrier would wait on m CTAs instead of m/G), and only
        // up to m = 512, where the island-per-CTA grid still takes fused steps.
        if ((mode == AIRPF_LAUNCH_AUTO || mode == AIRPF_LAUNCH_STEPS || mode == AIRPF_LAUNCH_STEPS_SPLIT) &&
            cfg->m <= 512 && cfg->ppt == 0 && cfg->islands_per_cta == 0) {
            int dev = 0, sms = 0;
            if (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                (long long)cfg->B * (cfg->m / p.G) < sms)
                airpf::choose_mapping(cfg->m, cfg->M, p.fp64, 2, 1, &p.tpi, &p.ppt, &p.G);
        }
    }
    p.P = cfg->m / p.G;
    p.g = ilog2_exact(p.G);
    p.lg_tpi = ilog2_exact(p.tpi);
    p.theta_dim = ctx->theta_dim;
    p.seed_lo = (uint32_t)(cfg->seed & 0xffffffffu);
    p.seed_hi = (uint32_t)(cfg->seed >> 32);
    p.run = at<RunParams>(ctx, L.run);
    p.theta = at<double>(ctx, L.theta);
    p.mdata = at<double>(ctx, L.mdata);
    p.y = at<double>(ctx, L.y);
    p.active = nullptr;
    p.mpar = at<void>(ctx, L.mpar);
    p.drift = at<void>(ctx, L.drift);
    p.bar = at<unsigned>(ctx, L.bar);
    p.err = at<unsigned>(ctx, L.bar) + 2;
    p.inject_stall = 0;
    // AUTO takes per-step launches for filters that span several CTAs: on GB300 a
    // kernel boundary (about 1 us in a graph) costs less than the device-scope
    // release/acquire pair of a grid barrier (about 3 us)
    // (and every CTA runs the cascade itself unless a filter spans more than
    // 512 CTAs, where reading all CTA records in every CTA would cost more)
    if (ctx->launch == AIRPF_LAUNCH_AUTO)
        ctx->launch = p.P <= 512 ? AIRPF_LAUNCH_STEPS : AIRPF_LAUNCH_STEPS_SPLIT;
    // split steps of the FP32 SV and NGM filters with islands of 256 to 1024 particles: eight
    // particles a thread (one warp an island of 256, two of 512, four of 1024), four islands
    // a CTA up to 512 particles -- fewer island-level barriers and shared-memory carries, and a
    // thread's fixed costs spread over twice the particles.  Measured on the m = 65536 NGM
    // workload: M = 256 155.6 -> 118.2 ms a pass (CTAs of 4 islands; 8 islands 128.0, 16
    // 147.6), M = 512 290.2 -> 224.0 (4 islands; 2 islands 303.6), M = 1024 576.8 -> 438.0
    // (the default 2 islands).  Fused steps keep four particles a thread (the m = 1024 SV
    // workload: 4.6 against 5.8-6.0 ms).
    if (ctx->launch == AIRPF_LAUNCH_STEPS_SPLIT && !p.fp64 && cfg->ppt == 0 && cfg->islands_per_cta == 0 &&
        (cfg->M == 256 || cfg->M == 512 || cfg->M == 1024) &&
        (cfg->model == AIRPF_MODEL_SV || cfg->model == AIRPF_MODEL_NGM)) {
        airpf::choose_mapping(cfg->m, cfg->M, p.fp64, 8, cfg->M <= 512 ? 4 : 0, &p.tpi, &p.ppt, &p.G);
        p.P = cfg->m / p.G;
        p.g = ilog2_exact(p.G);
        p.lg_tpi = ilog2_exact(p.tpi);
    }
    // (split steps keep the default 256-thread CTAs: on the m = 65536 workload they beat
    // 512-thread CTAs by 5-6% at M = 256 and 512 -- the block barriers of 16 warps cost more
    // than the cascade kernel's twice as many records -- and lose 1% at M = 64)
    // per-step launches overlap each kernel's start with the previous one
    // (programmatic dependent launch); fused steps have no cascade kernel
    p.pdl = is_steps(ctx->launch) ? 1 : 0;
    p.fused = ctx->launch == AIRPF_LAUNCH_STEPS ? 1 : 0;
    p.split = ctx->launch == AIRPF_LAUNCH_STEPS_SPLIT ? 1 : 0;
    p.gs = p.g + airpf::kTailGroupLog <= p.S ? airpf::kTailGroupLog : p.S - p.g;   // 2^gs records a group
    p.NG = p.P >> p.gs;
    if (airpf::step_smem_bytes(p) > 227 * 1024) {
        set_err(nullptr, "the step kernel would need %zu bytes of shared memory (m/G = %d CTA records per filter); "
                "use AIRPF_LAUNCH_STEPS_SPLIT or more islands per CTA", airpf::step_smem_bytes(p), p.P);
        cudaStreamDestroy(ctx->cap_stream);
        delete ctx;
        return AIRPF_ERR_UNSUPPORTED;
    }
    if (ctx->launch == AIRPF_LAUNCH_PERSISTENT_GRID) {
        e = airpf::prepare_step(p);
        const bool fits = (e == cudaSuccess) && airpf::persistent_grid_fits(p);
        if (fits) {
            ctx->launch = AIRPF_LAUNCH_PERSISTENT_GRID;
        } else if (ctx->launch == AIRPF_LAUNCH_PERSISTENT_GRID) {
            set_err(nullptr, "the grid of %d CTAs cannot be resident at once", p.B * (p.m / p.G));
            cudaStreamDestroy(ctx->cap_stream);
            delete ctx;
            return AIRPF_ERR_UNSUPPORTED;
        } else {
            ctx->launch = AIRPF_LAUNCH_STEPS;
        }
    }
    e = airpf::prepare_step(p);
    if (e != cudaSuccess) {
        set_err(nullptr, "kernel attribute setup: %s", cudaGetErrorString(e));
        cudaStreamDestroy(ctx->cap_stream);
        delete ctx;
        return AIRPF_ERR_CUDA;
    }
    // fused steps: the 128-register instantiation when the grid is one wave at its
    // occupancy (measured faster there; on larger grids the halved occupancy costs more)
    p.wide = (p.fused && airpf::wide_fused_fits(p)) ? 1 : 0;
    {
        unsigned zero[4] = {0, 0, 0, 0};
        e = cudaMemcpy(p.bar, zero, sizeof(zero), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            set_err(nullptr, "workspace init: %s", cudaGetErrorString(e));
            cudaStreamDestroy(ctx->cap_stream);
            delete ctx;
            return AIRPF_ERR_CUDA;
        }
    }
    for (int i = 0; i < 2; ++i) {
        p.X[i] = at<void>(ctx, L.X[i]);
        p.pe[i] = at<int>(ctx, L.pe[i]);
        p.pt[i] = at<void>(ctx, L.pt[i]);
        p.pq[i] = at<void>(ctx, L.pq[i]);
        p.ires[i] = L.ires[i] ? at<int>(ctx, L.ires[i]) : nullptr;
    }
    p.csum = at<int>(ctx, L.csum);
    p.cup = at<void>(ctx, L.cup);
    p.nsrc = at<int>(ctx, L.nsrc);
    p.utg = at<void>(ctx, L.utg);
    p.tick = at<unsigned>(ctx, L.tick);
    for (int i = 0; i < 2; ++i) {
        p.ge[i] = at<int>(ctx, L.ge[i]);
        p.gtr[i] = at<void>(ctx, L.gtr[i]);
        p.gqs[i] = at<void>(ctx, L.gqs[i]);
    }
    p.logz = at<double>(ctx, L.logz);
    p.trace = (cfg->record & AIRPF_RECORD_TRACE) ? at<double>(ctx, L.trace) : nullptr;
    p.enf = L.enf ? at<double>(ctx, L.enf) : nullptr;
    p.sstar = L.sstar ? at<int>(ctx, L.sstar) : nullptr;
    p.anc = L.anc ? at<int>(ctx, L.anc) : nullptr;
    if (cfg->record & AIRPF_RECORD_GRAD) {
        p.grad = 1;
        p.ckpt = cfg->ckpt > 0 ? cfg->ckpt : 1;
        p.nck = cfg->T / p.ckpt + 1 + (cfg->T % p.ckpt != 0 ? 1 : 0);
        p.xck = at<void>(ctx, L.xck);
        p.xblk = at<void>(ctx, L.xblk);
        p.logw = at<double>(ctx, L.logw);
        for (int i = 0; i < 2; ++i) p.gpi[i] = at<double>(ctx, L.gpi[i]);
        for (int i = 0; i < 3; ++i) {
            p.xh[i] = at<void>(ctx, L.xh[i]);
            p.dh[i] = at<void>(ctx, L.dh[i]);
        }
        p.gout = at<double>(ctx, L.gout);
        p.gacc = at<double>(ctx, L.gacc);
        p.sout = at<double>(ctx, L.sout);
    }
    p.rb = radix_bits(cfg);
    p.air = cfg->tau_int > 0.0 ? 1 : 0;
    p.tau_int = cfg->tau_int;
    for (int i = 0; i < 2; ++i) p.lom[i] = L.lom[i] ? at<void>(ctx, L.lom[i]) : nullptr;
    p.fmom = 0;
    p.fm_nw = 0;
    p.fw = p.fsum = nullptr;
    if (cfg->record & AIRPF_RECORD_MOMENTS) {
        if (p.tpi / 32 > L.fm_nw) {
            set_err(nullptr, "internal: warps per island %d, workspace sized for %d", p.tpi / 32, L.fm_nw);
            cudaStreamDestroy(ctx->cap_stream);
            delete ctx;
            return AIRPF_ERR_UNSUPPORTED;
        }
        p.fmom = 1;
        p.fm_nw = p.tpi / 32;
        p.fw = at<double>(ctx, L.fw);
        p.fsum = at<double>(ctx, L.fsum);
    }
    ctx->sp_pm = p;
    ctx->sp_pm.active = at<int>(ctx, L.active);

    if (cfg->model == AIRPF_MODEL_LGSSM) {
        const size_t n = sizeof(double) * (size_t)(cfg->dx * cfg->dx + cfg->dy * cfg->dx);
        std::memcpy(ctx->md_host, model_data, n);
        e = cudaMemcpyAsync(at<void>(ctx, L.mdata), model_data, n, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            set_err(nullptr, "model data copy: %s", cudaGetErrorString(e));
            cudaStreamDestroy(ctx->cap_stream);
            delete ctx;
            return AIRPF_ERR_CUDA;
        }
    }
    if (cfg->record & AIRPF_RECORD_TIMING) {
        if (!is_steps(ctx->launch) || cfg->T > (1 << 16)) {
            set_err(nullptr, "AIRPF_RECORD_TIMING needs a per-step launch and T <= 65536");
            cudaStreamDestroy(ctx->cap_stream);
            delete ctx;
            return AIRPF_ERR_UNSUPPORTED;
        }
        ctx->n_ev = 4 * cfg->T;
        ctx->ev = new (std::nothrow) cudaEvent_t[ctx->n_ev];
        int made = 0;
        e = ctx->ev ? cudaSuccess : cudaErrorMemoryAllocation;
        for (; made < ctx->n_ev && e == cudaSuccess; ++made) e = cudaEventCreate(&ctx->ev[made]);
        if (e != cudaSuccess) {
            set_err(nullptr, "timing events: %s", cudaGetErrorString(e));
            for (int i = 0; i + 1 < made; ++i) cudaEventDestroy(ctx->ev[i]);
            delete[] ctx->ev;
            cudaStreamDestroy(ctx->cap_stream);
            delete ctx;
            return AIRPF_ERR_CUDA;
        }
    }
    *out = ctx;
    return AIRPF_OK;
}

airpf_status airpf_destroy(airpf_ctx* ctx)
{
    if (!ctx) return AIRPF_ERR_ARG;
    if (ctx->graph_ready) cudaGraphExecDestroy(ctx->graph);
    if (ctx->graph_pm_ready) cudaGraphExecDestroy(ctx->graph_pm);
    if (ctx->graph_bwd_ready) cudaGraphExecDestroy(ctx->graph_bwd);
    if (ctx->bwd_aux_ready) {
        for (int i = 0; i < airpf::kGradEvents; ++i) cudaEventDestroy(ctx->bwd_ev[i]);
        cudaStreamDestroy(ctx->bwd_aux);
    }
    if (ctx->ev) {
        for (int i = 0; i < ctx->n_ev; ++i) cudaEventDestroy(ctx->ev[i]);
        delete[] ctx->ev;
    }
    cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return AIRPF_OK;
}

airpf_status airpf_run(airpf_ctx* ctx, const double* d_theta, const double* d_y, uint32_t chain0,
                       uint32_t iter, double* d_log_z, int32_t* d_anc, double* d_enf, int32_t* d_sstar,
                       double* d_trace)
{
    if (!ctx) return AIRPF_ERR_ARG;
    const airpf_config& c = ctx->cfg;
    if (!d_theta || !d_y || !d_log_z) {
        set_err(ctx, "theta, y and log_z are required");
        return AIRPF_ERR_ARG;
    }
    if ((uint64_t)chain0 + (uint64_t)c.B > (1u << 24)) {
        set_err(ctx, "chain0 + B must not exceed 2^24");
        return AIRPF_ERR_ARG;
    }
    if ((d_anc && !(c.record & AIRPF_RECORD_LINEAGE)) || ((d_enf || d_sstar) && !(c.record & AIRPF_RECORD_ENF))
        || (d_trace && !(c.record & AIRPF_RECORD_TRACE))) {
        set_err(ctx, "an output was requested that the context does not record");
        return AIRPF_ERR_ARG;
    }
    ctx->launches = 0;
    const size_t B = c.B, T = c.T, N = ctx->N;
    airpf_status s;
    if ((s = copy_async(ctx, at<void>(ctx, ctx->L.theta), d_theta, sizeof(double) * B * ctx->theta_dim))) return s;
    if ((s = copy_async(ctx, at<void>(ctx, ctx->L.y), d_y, sizeof(double) * T * c.dy))) return s;
    cudaError_t e = airpf::launch_set_run(at<RunParams>(ctx, ctx->L.run), iter, chain0, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_run launch");
    ctx->launches += 1;
    if ((s = enqueue_pass(ctx))) return s;
    if ((s = copy_async(ctx, d_log_z, at<void>(ctx, ctx->L.logz), sizeof(double) * B))) return s;
    if (d_anc && (s = copy_async(ctx, d_anc, at<void>(ctx, ctx->L.anc), sizeof(int) * B * T * N))) return s;
    if (d_enf && (s = copy_async(ctx, d_enf, at<void>(ctx, ctx->L.enf),
                                 sizeof(double) * B * T * (ctx->S / radix_bits(&c) + 1))))
        return s;
    if (d_sstar && (s = copy_async(ctx, d_sstar, at<void>(ctx, ctx->L.sstar), sizeof(int) * B * T))) return s;
    if (d_trace && (s = copy_async(ctx, d_trace, at<void>(ctx, ctx->L.trace), sizeof(double) * B * T))) return s;
    return AIRPF_OK;
}

airpf_status airpf_run_host(airpf_ctx* ctx, const double* theta, const double* y, uint32_t chain0,
                            uint32_t iter, double* log_z)
{
    if (!ctx) return AIRPF_ERR_ARG;
    if (!theta || !y || !log_z) {
        set_err(ctx, "theta, y and log_z are required");
        return AIRPF_ERR_ARG;
    }
    airpf_status s = airpf_run(ctx, theta, y, chain0, iter, log_z, nullptr, nullptr, nullptr, nullptr);
    if (s != AIRPF_OK) return s;
    return airpf_sync(ctx);
}

// ---------------------------------------------------------------------------
// Stepwise passes: the caller drives the steps, so that the islands of one filter
// can be split over several processes (one GPU each) with an exchange of the step's
// CTA records and particle rows between the island launch and the cascade.
// ---------------------------------------------------------------------------
static airpf_status step_check(airpf_ctx* ctx)
{
    if (!ctx) return AIRPF_ERR_ARG;
    if (!is_steps(ctx->launch)) {
        set_err(ctx, "stepwise passes need per-step launches (AIRPF_LAUNCH_STEPS or AIRPF_LAUNCH_STEPS_SPLIT)");
        return AIRPF_ERR_UNSUPPORTED;
    }
    if (ctx->cfg.record != 0 || ctx->cfg.B != 1 || ctx->cfg.tau_int > 0.0) {
        set_err(ctx, "stepwise passes run one filter (B = 1) without records or adaptive internal resampling");
        return AIRPF_ERR_UNSUPPORTED;
    }
    return AIRPF_OK;
}

airpf_status airpf_step_begin(airpf_ctx* ctx, const double* d_theta, const double* d_y, uint32_t chain0, uint32_t iter)
{
    airpf_status s = step_check(ctx);
    if (s != AIRPF_OK) return s;
    if (!d_theta || !d_y) {
        set_err(ctx, "theta and y are required");
        return AIRPF_ERR_ARG;
    }
    if ((uint64_t)chain0 + 1u > (1u << 24)) {
        set_err(ctx, "chain0 must be below 2^24");
        return AIRPF_ERR_ARG;
    }
    const airpf_config& c = ctx->cfg;
    if ((s = copy_async(ctx, at<void>(ctx, ctx->L.theta), d_theta, sizeof(double) * ctx->theta_dim))) return s;
    if ((s = copy_async(ctx, at<void>(ctx, ctx->L.y), d_y, sizeof(double) * (size_t)c.T * c.dy))) return s;
    cudaError_t e = airpf::launch_set_run(at<RunParams>(ctx, ctx->L.run), iter, chain0, ctx->stream);
    if (e == cudaSuccess) e = airpf::prepare_step(ctx->sp);
    StepParams q = ctx->sp;
    q.pdl = 0;
    if (e == cudaSuccess) e = airpf::launch_step(q, 0, ctx->stream);      // the prologue
    return e == cudaSuccess ? AIRPF_OK : cuda_fail(ctx, e, "airpf_step_begin");
}

airpf_status airpf_step_islands(airpf_ctx* ctx, int32_t t, int32_t cta0, int32_t ncta)
{
    airpf_status s = step_check(ctx);
    if (s != AIRPF_OK) return s;
    const int P = ctx->sp.P;
    if (t < 1 || t > ctx->cfg.T) {
        set_err(ctx, "step %d outside 1 .. T = %d", t, ctx->cfg.T);
        return AIRPF_ERR_ARG;
    }
    if (ncta == 0) ncta = P;
    if (cta0 < 0 || ncta < 1 || (ncta & (ncta - 1)) || cta0 % ncta != 0 || cta0 + ncta > P) {
        set_err(ctx, "CTA range [%d, %d) must be an aligned power-of-2 range within the %d CTAs", cta0, cta0 + ncta, P);
        return AIRPF_ERR_ARG;
    }
    StepParams q = ctx->sp;
    q.pdl = 0;
    q.cta0 = cta0;
    q.ncta = ncta;
    q.lg_ncta = ilog2_exact(ncta);
    cudaError_t e = airpf::launch_step(q, t, ctx->stream);
    return e == cudaSuccess ? AIRPF_OK : cuda_fail(ctx, e, "airpf_step_islands");
}

airpf_status airpf_step_cascade(airpf_ctx* ctx, int32_t t)
{
    airpf_status s = step_check(ctx);
    if (s != AIRPF_OK) return s;
    if (t < 1 || t > ctx->cfg.T) {
        set_err(ctx, "step %d outside 1 .. T = %d", t, ctx->cfg.T);
        return AIRPF_ERR_ARG;
    }
    if (ctx->sp.fused && t < ctx->cfg.T) return AIRPF_OK;     // the next island launch runs it in every CTA
    StepParams q = ctx->sp;
    q.pdl = 0;
    cudaError_t e;
    if (ctx->sp.fused) {
        // the last step's cascade (log Z): the lineage launch of step T+1 runs it
        e = airpf::launch_step(q, t + 1, ctx->stream);
    } else {
        e = airpf::launch_cascade(q, t, ctx->stream);
    }
    return e == cudaSuccess ? AIRPF_OK : cuda_fail(ctx, e, "airpf_step_cascade");
}

airpf_status airpf_step_end(airpf_ctx* ctx, double* d_log_z)
{
    airpf_status s = step_check(ctx);
    if (s != AIRPF_OK) return s;
    if (!d_log_z) {
        set_err(ctx, "log_z is required");
        return AIRPF_ERR_ARG;
    }
    return copy_async(ctx, d_log_z, at<void>(ctx, ctx->L.logz), sizeof(double));
}

airpf_status airpf_step_regions(airpf_ctx* ctx, int32_t t, size_t* offsets, size_t* bytes, int32_t* count)
{
    airpf_status s = step_check(ctx);
    if (s != AIRPF_OK) return s;
    if (!offsets || !bytes || !count || t < 0) return AIRPF_ERR_ARG;
    const airpf_config& c = ctx->cfg;
    const size_t P = (size_t)ctx->sp.P, G = (size_t)ctx->sp.G, N = (size_t)ctx->N;
    const size_t rsz = c.precision == AIRPF_FP64 ? 8 : 4;
    const int par = t & 1;
    int n = 0;
    offsets[n] = ctx->L.pe[par];
    bytes[n++] = sizeof(int) * P;
    offsets[n] = ctx->L.pt[par];
    bytes[n++] = sizeof(double) * 2 * G * P;
    offsets[n] = ctx->L.pq[par];
    bytes[n++] = rsz * 8 * P;
    for (int d = 0; d < c.dx; ++d) {
        offsets[n] = ctx->L.X[par] + rsz * (size_t)d * N;
        bytes[n++] = rsz * N;
    }
    *count = n;
    return AIRPF_OK;
}

airpf_status airpf_step_levels(airpf_ctx* ctx, int32_t* levels)
{
    airpf_status s = step_check(ctx);
    if (s != AIRPF_OK) return s;
    if (!levels) return AIRPF_ERR_ARG;
    if (ctx->sp.fused) {
        set_err(ctx, "fused steps run a step's cascade inside the next island launch");
        return AIRPF_ERR_UNSUPPORTED;
    }
    int ss = 0;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&ss, ctx->sp.csum, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "airpf_step_levels");
    *levels = ss - 1;                 // binary levels below the first quiet one
    return AIRPF_OK;
}

airpf_status airpf_sync(airpf_ctx* ctx)
{
    if (!ctx) return AIRPF_ERR_ARG;
    unsigned flag = 0;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&flag, ctx->sp.err, sizeof(flag), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "airpf_sync");
    if (flag) {
        set_err(ctx, "a grid-barrier wait timed out; the pass's results are invalid");
        return AIRPF_ERR_TIMEOUT;
    }
    return AIRPF_OK;
}

airpf_status airpf_grad(airpf_ctx* ctx, const double* d_theta, const double* d_y, uint32_t chain0, uint32_t iter,
                        double* d_log_z, double* d_grad, double* d_score)
{
    if (!ctx) return AIRPF_ERR_ARG;
    if (!ctx->sp.grad) {
        set_err(ctx, "the context was created without AIRPF_RECORD_GRAD");
        return AIRPF_ERR_UNSUPPORTED;
    }
    if (!d_grad && !d_score) {
        set_err(ctx, "grad or score is required");
        return AIRPF_ERR_ARG;
    }
    airpf_status s = airpf_run(ctx, d_theta, d_y, chain0, iter, d_log_z, nullptr, nullptr, nullptr, nullptr);
    if (s != AIRPF_OK) return s;
    const int64_t fwd = ctx->launches;
    if (!ctx->graph_bwd_ready) {
        if (!ctx->bwd_aux_ready) {
            cudaError_t e = cudaStreamCreateWithFlags(&ctx->bwd_aux, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "backward-pass stream");
            int made = 0;
            while (made < airpf::kGradEvents && e == cudaSuccess) {
                e = cudaEventCreateWithFlags(&ctx->bwd_ev[made], cudaEventDisableTiming);
                if (e == cudaSuccess) ++made;
            }
            if (e != cudaSuccess) {
                for (int i = 0; i < made; ++i) cudaEventDestroy(ctx->bwd_ev[i]);
                cudaStreamDestroy(ctx->bwd_aux);
                return cuda_fail(ctx, e, "backward-pass events");
            }
            ctx->bwd_aux_ready = true;
        }
        cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
        cudaError_t le = airpf::launch_grad_backward(ctx->sp, ctx->md_host, ctx->cap_stream, ctx->bwd_aux,
                                                     ctx->bwd_ev);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(ctx, le, "gradient launch during capture");
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ctx->graph_bwd, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
        ctx->graph_bwd_ready = true;
    }
    cudaError_t e = cudaGraphLaunch(ctx->graph_bwd, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
    {
        const int T = ctx->cfg.T, K = ctx->sp.ckpt;
        int rec = 0;
        for (int t = 1; t <= T; ++t) rec += (t % K != 0 && t != T);
        ctx->launches = fwd + 1 + T + (T - 1) + rec;
    }
    const size_t n = sizeof(double) * (size_t)ctx->cfg.B * ctx->theta_dim;
    if (d_grad && (s = copy_async(ctx, d_grad, ctx->sp.gout, n))) return s;
    if (d_score && (s = copy_async(ctx, d_score, ctx->sp.sout, n))) return s;
    return AIRPF_OK;
}

airpf_status airpf_kernel_times(airpf_ctx* ctx, double* step_ms, double* cascade_ms)
{
    if (!ctx || !step_ms || !cascade_ms) return AIRPF_ERR_ARG;
    if (!ctx->ev) {
        set_err(ctx, "the context was created without AIRPF_RECORD_TIMING");
        return AIRPF_ERR_UNSUPPORTED;
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "airpf_kernel_times");
    double a = 0.0, b = 0.0;
    for (int t = 0; t < ctx->cfg.T; ++t) {
        float x = 0.f, y = 0.f;
        e = cudaEventElapsedTime(&x, ctx->ev[4 * t], ctx->ev[4 * t + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&y, ctx->ev[4 * t + 2], ctx->ev[4 * t + 3]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventElapsedTime");
        a += x;
        b += y;
    }
    *step_ms = a;
    *cascade_ms = b;
    return AIRPF_OK;
}

airpf_status airpf_moments(airpf_ctx* ctx, double* d_moments)
{
    if (!ctx || !d_moments) return AIRPF_ERR_ARG;
    if (!(ctx->cfg.record & AIRPF_RECORD_MOMENTS)) {
        set_err(ctx, "the context was created without AIRPF_RECORD_MOMENTS");
        return AIRPF_ERR_UNSUPPORTED;
    }
    const cudaError_t e = airpf::launch_moments(ctx->sp, d_moments, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "moments kernel launch");
    return AIRPF_OK;
}

int32_t airpf_launch_mode(const airpf_ctx* ctx) { return ctx ? ctx->launch : 0; }

airpf_status airpf_tiling(const airpf_ctx* ctx, int32_t* threads_per_island, int32_t* particles_per_thread,
                          int32_t* islands_per_cta)
{
    if (!ctx || !threads_per_island || !particles_per_thread || !islands_per_cta) return AIRPF_ERR_ARG;
    *threads_per_island = ctx->sp.tpi;
    *particles_per_thread = ctx->sp.ppt;
    *islands_per_cta = ctx->sp.G;
    return AIRPF_OK;
}

airpf_status airpf_debug_inject(airpf_ctx* ctx, int32_t what)
{
    if (!ctx) return AIRPF_ERR_ARG;
    if (ctx->launch != AIRPF_LAUNCH_PERSISTENT_GRID) {
        set_err(ctx, "fault injection needs the grid-persistent launch");
        return AIRPF_ERR_UNSUPPORTED;
    }
    ctx->sp.inject_stall = what == 1 ? 1 : 0;
    return AIRPF_OK;
}

airpf_status airpf_pmmh(airpf_ctx* ctx, const double* d_y, const double* step, const double* lo,
                        const double* hi, double* d_state_theta, double* d_state_logz, uint32_t chain0,
                        uint32_t iter0, int32_t iters, double* d_theta_out, double* d_logz_out,
                        int32_t* d_n_accept)
{
    if (!ctx) return AIRPF_ERR_ARG;
    const airpf_config& c = ctx->cfg;
    if (!d_y || !step || !lo || !hi || !d_state_theta || !d_state_logz || !d_n_accept) {
        set_err(ctx, "y, step, lo, hi, state_theta, state_logz and n_accept are required");
        return AIRPF_ERR_ARG;
    }
    if (iters < 0) {
        set_err(ctx, "iters must be >= 0");
        return AIRPF_ERR_ARG;
    }
    if ((uint64_t)chain0 + (uint64_t)c.B > (1u << 24)) {
        set_err(ctx, "chain0 + B must not exceed 2^24");
        return AIRPF_ERR_ARG;
    }
    if ((uint64_t)iter0 + (uint64_t)iters > 0xffffffffull) {
        set_err(ctx, "iter0 + iters must stay below 2^32 - 1 (reserved for the initial estimate)");
        return AIRPF_ERR_ARG;
    }
    const int td = ctx->theta_dim;
    airpf::PmmhParams q;
    std::memset(&q, 0, sizeof(q));
    q.B = c.B;
    q.theta_dim = td;
    q.model = c.model;
    q.dx = c.dx;
    q.seed_lo = (uint32_t)(c.seed & 0xffffffffu);
    q.seed_hi = (uint32_t)(c.seed >> 32);
    q.chain0 = chain0;
    for (int d = 0; d < td; ++d) {
        if (!(step[d] >= 0.0) || (step[d] > 0.0 && !(lo[d] <= hi[d]))) {
            set_err(ctx, "component %d: step must be >= 0 and lo <= hi", d);
            return AIRPF_ERR_ARG;
        }
        q.step[d] = step[d];
        q.lo[d] = lo[d];
        q.hi[d] = hi[d];
    }
    q.run = at<RunParams>(ctx, ctx->L.run);
    q.theta = at<double>(ctx, ctx->L.theta);
    q.logz = at<double>(ctx, ctx->L.logz);
    q.active = at<int>(ctx, ctx->L.active);
    q.state_theta = d_state_theta;
    q.state_logz = d_state_logz;
    q.n_accept = d_n_accept;
    q.theta_out = d_theta_out;
    q.logz_out = d_logz_out;

    ctx->launches = 0;
    airpf_status s;
    if ((s = copy_async(ctx, at<void>(ctx, ctx->L.y), d_y, sizeof(double) * (size_t)c.T * c.dy))) return s;
    // the initial estimate of the chains whose log Z is NaN (a pass with no
    // active filter when there is none), then one pass per iteration
    for (int64_t j = -1; j < iters; ++j) {
        const int initial = j < 0;
        const uint32_t it = initial ? 0xffffffffu : iter0 + (uint32_t)j;
        cudaError_t e = airpf::launch_pmmh_propose(q, it, initial, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "PMMH proposal launch");
        if ((s = enqueue_pass(ctx, true))) return s;
        e = airpf::launch_pmmh_accept(q, it, initial ? 0 : (int)j, initial, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "PMMH acceptance launch");
        ctx->launches += 2;
    }
    return AIRPF_OK;
}

airpf_status airpf_pmmh_langevin(airpf_ctx* ctx, const double* d_y, const double* step, const double* lo,
                                 const double* hi, double* d_state_theta, double* d_state_logz,
                                 double* d_state_grad, uint32_t chain0, uint32_t iter0, int32_t iters,
                                 double* d_theta_out, double* d_logz_out, int32_t* d_n_accept)
{
    if (!ctx) return AIRPF_ERR_ARG;
    const airpf_config& c = ctx->cfg;
    if (!ctx->sp.grad) {
        set_err(ctx, "the Langevin proposal needs a context created with AIRPF_RECORD_GRAD");
        return AIRPF_ERR_UNSUPPORTED;
    }
    if (!d_y || !step || !lo || !hi || !d_state_theta || !d_state_logz || !d_state_grad || !d_n_accept) {
        set_err(ctx, "y, step, lo, hi, state_theta, state_logz, state_grad and n_accept are required");
        return AIRPF_ERR_ARG;
    }
    if (iters < 0 || (uint64_t)chain0 + (uint64_t)c.B > (1u << 24) ||
        (uint64_t)iter0 + (uint64_t)iters > 0xffffffffull) {
        set_err(ctx, "iters >= 0, chain0 + B <= 2^24 and iter0 + iters < 2^32 - 1 are required");
        return AIRPF_ERR_ARG;
    }
    const int td = ctx->theta_dim;
    airpf::PmmhParams q;
    std::memset(&q, 0, sizeof(q));
    q.B = c.B;
    q.theta_dim = td;
    q.model = c.model;
    q.dx = c.dx;
    q.seed_lo = (uint32_t)(c.seed & 0xffffffffu);
    q.seed_hi = (uint32_t)(c.seed >> 32);
    q.chain0 = chain0;
    for (int d = 0; d < td; ++d) {
        if (!(step[d] >= 0.0) || (step[d] > 0.0 && !(lo[d] <= hi[d]))) {
            set_err(ctx, "component %d: step must be >= 0 and lo <= hi", d);
            return AIRPF_ERR_ARG;
        }
        q.step[d] = step[d];
        q.lo[d] = lo[d];
        q.hi[d] = hi[d];
    }
    q.theta = at<double>(ctx, ctx->L.pm_prop);          // the proposals, input of each gradient pass
    q.logz = at<double>(ctx, ctx->L.pm_logz_prop);
    q.active = at<int>(ctx, ctx->L.active);
    q.state_theta = d_state_theta;
    q.state_logz = d_state_logz;
    q.n_accept = d_n_accept;
    q.theta_out = d_theta_out;
    q.logz_out = d_logz_out;
    q.state_grad = d_state_grad;
    q.gprop = at<double>(ctx, ctx->L.pm_gprop);
    q.lqf = at<double>(ctx, ctx->L.pm_lqf);
    int64_t launches = 0;
    for (int64_t j = -1; j < iters; ++j) {
        const int initial = j < 0;
        const uint32_t it = initial ? 0xffffffffu : iter0 + (uint32_t)j;
        cudaError_t e = airpf::launch_lmh_propose(q, it, initial, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "Langevin proposal launch");
        airpf_status s = airpf_grad(ctx, q.theta, d_y, chain0, it, at<double>(ctx, ctx->L.pm_logz_prop), nullptr,
                                    at<double>(ctx, ctx->L.pm_gprop));
        if (s != AIRPF_OK) return s;
        launches += ctx->launches + 2;
        e = airpf::launch_lmh_accept(q, it, initial ? 0 : (int)j, initial, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "Langevin acceptance launch");
    }
    ctx->launches = launches;
    return AIRPF_OK;
}

int64_t airpf_last_launch_count(const airpf_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* airpf_last_error(const airpf_ctx* ctx) { return ctx ? ctx->err : g_create_error; }

const char* airpf_status_string(airpf_status s)
{
    switch (s) {
    case AIRPF_OK: return "AIRPF_OK";
    case AIRPF_ERR_ARG: return "AIRPF_ERR_ARG";
    case AIRPF_ERR_CUDA: return "AIRPF_ERR_CUDA";
    case AIRPF_ERR_WORKSPACE: return "AIRPF_ERR_WORKSPACE";
    case AIRPF_ERR_TIMEOUT: return "AIRPF_ERR_TIMEOUT";
    case AIRPF_ERR_UNSUPPORTED: return "AIRPF_ERR_UNSUPPORTED";
    }
    return "unknown status";
}

}  // extern "C"
