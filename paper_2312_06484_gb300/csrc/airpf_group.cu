// airpf_group.cu -- host runtime for batches of filters with uneven sizes and
// the tiling autotuner (see include/airpf.h).
//
// A batch of chains with different (m, M) is a set of contexts, one per size
// class, each holding the chains of its class as the filters of one batch.
// The group runs every context's pass (or PMMH iterations) on the context's
// own stream, forked from and joined back to the group's stream by events, so
// the classes' per-step kernels run side by side on the GPU and the caller sees
// one asynchronous operation on one stream.
//
// The autotuner times candidate tilings (particles per thread, islands per CTA,
// one or two kernels per step, one CTA per filter when a filter fits) on the
// caller's workspace and returns the fastest as a configuration.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/airpf.h"
#include "airpf_internal.h"

struct airpf_group {
    std::vector<airpf_ctx*> ctxs;
    cudaStream_t stream;
    cudaEvent_t fork;
    std::vector<cudaEvent_t> join;
};

namespace {

airpf_status group_fail(cudaError_t e, const char* what)
{
    airpf::set_create_error("%s: %s", what, cudaGetErrorString(e));
    return AIRPF_ERR_CUDA;
}

// Make every member stream wait for the group stream's work so far.
airpf_status fork_members(airpf_group* g)
{
    cudaError_t e = cudaEventRecord(g->fork, g->stream);
    if (e != cudaSuccess) return group_fail(e, "group fork");
    for (airpf_ctx* c : g->ctxs) {
        e = cudaStreamWaitEvent(airpf::ctx_stream(c), g->fork, 0);
        if (e != cudaSuccess) return group_fail(e, "group fork wait");
    }
    return AIRPF_OK;
}

// Make the group stream wait for every member's work so far.
airpf_status join_members(airpf_group* g)
{
    for (size_t i = 0; i < g->ctxs.size(); ++i) {
        cudaError_t e = cudaEventRecord(g->join[i], airpf::ctx_stream(g->ctxs[i]));
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->join[i], 0);
        if (e != cudaSuccess) return group_fail(e, "group join");
    }
    return AIRPF_OK;
}

airpf_status member_fail(airpf_status s, int i, airpf_ctx* c)
{
    airpf::set_create_error("group member %d: %s", i, airpf_last_error(c));
    return s;
}

}  // namespace

extern "C" {

airpf_status airpf_group_create(airpf_ctx* const* ctxs, int32_t n, void* stream, airpf_group** out)
{
    if (!out) {
        airpf::set_create_error("out is NULL");
        return AIRPF_ERR_ARG;
    }
    *out = nullptr;
    if (!ctxs || n < 1) {
        airpf::set_create_error("a group needs at least one context");
        return AIRPF_ERR_ARG;
    }
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) {
            airpf::set_create_error("context %d is NULL", i);
            return AIRPF_ERR_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) {
                airpf::set_create_error("context %d appears twice", i);
                return AIRPF_ERR_ARG;
            }
    }
    airpf_group* g = new (std::nothrow) airpf_group();
    if (!g) {
        airpf::set_create_error("host allocation failed");
        return AIRPF_ERR_ARG;
    }
    g->ctxs.assign(ctxs, ctxs + n);
    g->stream = static_cast<cudaStream_t>(stream);
    g->join.assign(n, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
    int made = 0;
    for (; e == cudaSuccess && made < n; ++made) e = cudaEventCreateWithFlags(&g->join[made], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        airpf::set_create_error("group events: %s", cudaGetErrorString(e));
        for (int i = 0; i + 1 < made; ++i) cudaEventDestroy(g->join[i]);
        if (made > 0) cudaEventDestroy(g->fork);
        delete g;
        return AIRPF_ERR_CUDA;
    }
    *out = g;
    return AIRPF_OK;
}

airpf_status airpf_group_destroy(airpf_group* g)
{
    if (!g) return AIRPF_ERR_ARG;
    cudaEventDestroy(g->fork);
    for (cudaEvent_t e : g->join) cudaEventDestroy(e);
    delete g;
    return AIRPF_OK;
}

airpf_status airpf_group_run(airpf_group* g, const double* const* d_theta, const double* d_y,
                             const uint32_t* chain0, uint32_t iter, double* const* d_log_z)
{
    if (!g || !d_theta || !d_y || !chain0 || !d_log_z) {
        airpf::set_create_error("group, theta, y, chain0 and log_z are required");
        return AIRPF_ERR_ARG;
    }
    airpf_status s = fork_members(g);
    if (s != AIRPF_OK) return s;
    for (size_t i = 0; i < g->ctxs.size(); ++i) {
        s = airpf_run(g->ctxs[i], d_theta[i], d_y, chain0[i], iter, d_log_z[i], nullptr, nullptr, nullptr, nullptr);
        if (s != AIRPF_OK) return member_fail(s, (int)i, g->ctxs[i]);
    }
    return join_members(g);
}

airpf_status airpf_group_pmmh(airpf_group* g, const double* d_y, const double* step, const double* lo,
                              const double* hi, double* const* d_state_theta, double* const* d_state_logz,
                              const uint32_t* chain0, uint32_t iter0, int32_t iters, double* const* d_theta_out,
                              double* const* d_logz_out, int32_t* const* d_n_accept)
{
    if (!g || !d_y || !step || !lo || !hi || !d_state_theta || !d_state_logz || !chain0 || !d_n_accept) {
        airpf::set_create_error("group, y, step, lo, hi, state_theta, state_logz, chain0 and n_accept are required");
        return AIRPF_ERR_ARG;
    }
    airpf_status s = fork_members(g);
    if (s != AIRPF_OK) return s;
    for (size_t i = 0; i < g->ctxs.size(); ++i) {
        s = airpf_pmmh(g->ctxs[i], d_y, step, lo, hi, d_state_theta[i], d_state_logz[i], chain0[i], iter0, iters,
                       d_theta_out ? d_theta_out[i] : nullptr, d_logz_out ? d_logz_out[i] : nullptr,
                       d_n_accept[i]);
        if (s != AIRPF_OK) return member_fail(s, (int)i, g->ctxs[i]);
    }
    return join_members(g);
}

airpf_status airpf_group_sync(airpf_group* g)
{
    if (!g) return AIRPF_ERR_ARG;
    for (size_t i = 0; i < g->ctxs.size(); ++i) {
        airpf_status s = airpf_sync(g->ctxs[i]);
        if (s != AIRPF_OK) return member_fail(s, (int)i, g->ctxs[i]);
    }
    cudaError_t e = cudaStreamSynchronize(g->stream);
    return e == cudaSuccess ? AIRPF_OK : group_fail(e, "airpf_group_sync");
}

airpf_status airpf_autotune(const airpf_config* cfg, void* d_workspace, size_t workspace_bytes,
                            const double* model_data, const double* d_theta, const double* d_y, int32_t passes,
                            void* stream, airpf_config* best, float* best_ms)
{
    size_t need = 0;
    airpf_status s = airpf_workspace_bytes(cfg, &need);
    if (s != AIRPF_OK) return s;
    if (!best || !best_ms || !d_theta || !d_y || passes < 1) {
        airpf::set_create_error("autotune needs theta, y, best, best_ms and passes >= 1");
        return AIRPF_ERR_ARG;
    }
    if (cfg->record != 0) {
        airpf::set_create_error("autotune times passes that record nothing: record must be 0");
        return AIRPF_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return group_fail(ce, "autotune events");
    }
    // candidate tilings, each distinct in its actual (launch, tpi, ppt, G)
    struct Cand { int launch, ppt, g; };
    std::vector<Cand> cands;
    std::vector<int> seen;                    // actual (tpi, ppt, G) of each candidate, packed
    const int fp64 = cfg->precision == AIRPF_FP64;
    auto add = [&](int launch, int ppt, int want_g) {
        int tpi = 0, pp = 0, G = 0;
        airpf::choose_mapping(cfg->m, cfg->M, fp64, ppt, want_g, &tpi, &pp, &G);
        if (launch == AIRPF_LAUNCH_PERSISTENT_CTA && !(G == cfg->m && G * tpi <= airpf::max_cta_threads())) return;
        const int key = (launch << 24) | (tpi << 12) | (pp << 8) | G;
        for (int k : seen)
            if (k == key) return;
        seen.push_back(key);
        cands.push_back({launch, ppt, want_g});
    };
    // eight particles a thread: compiled for the FP32 SV and NGM filters, islands of 256 or more
    const bool ppt8 = !fp64 && cfg->M >= 256 && (cfg->model == AIRPF_MODEL_SV || cfg->model == AIRPF_MODEL_NGM);
    for (int ppt : {2, 4, 8}) {
        if (ppt == 8 && !ppt8) continue;
        add(AIRPF_LAUNCH_PERSISTENT_CTA, ppt, cfg->m);
        for (int want_g = 1; want_g <= 16 && want_g <= cfg->m; want_g *= 2) {
            add(AIRPF_LAUNCH_STEPS, ppt, want_g);
            add(AIRPF_LAUNCH_STEPS_SPLIT, ppt, want_g);
        }
    }
    float best_t = -1.0f;
    airpf_config best_cfg = *cfg;
    double* d_out = nullptr;          // log Z of the timed passes: the last bytes of the workspace
    if (workspace_bytes < ((need + 255) & ~size_t(255)) + sizeof(double) * (size_t)cfg->B) {
        airpf::set_create_error("autotune needs airpf_workspace_bytes(cfg) rounded up to 256, plus 8 B bytes");
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return AIRPF_ERR_WORKSPACE;
    }
    d_out = reinterpret_cast<double*>(static_cast<unsigned char*>(d_workspace) + ((need + 255) & ~size_t(255)));
    for (const Cand& c : cands) {
        airpf_config k = *cfg;
        k.launch = c.launch;
        k.ppt = c.ppt;
        k.islands_per_cta = c.g;
        airpf_ctx* ctx = nullptr;
        if (airpf_create(&k, d_workspace, need, model_data, stream, &ctx) != AIRPF_OK) continue;
        s = airpf_run(ctx, d_theta, d_y, 0, 0xfffffff0u, d_out, nullptr, nullptr, nullptr, nullptr);   // warm-up
        if (s == AIRPF_OK) ce = cudaEventRecord(e0, st);
        for (int j = 0; s == AIRPF_OK && ce == cudaSuccess && j < passes; ++j)
            s = airpf_run(ctx, d_theta, d_y, 0, (uint32_t)j, d_out, nullptr, nullptr, nullptr, nullptr);
        if (s == AIRPF_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, st);
        if (s == AIRPF_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        if (s == AIRPF_OK && ce == cudaSuccess) s = airpf_sync(ctx);
        float ms = 0.0f;
        if (s == AIRPF_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        airpf_destroy(ctx);
        if (s != AIRPF_OK || ce != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (ce != cudaSuccess) return group_fail(ce, "autotune pass");
            return s;
        }
        ms /= (float)passes;
        if (best_t < 0.0f || ms < best_t) {
            best_t = ms;
            best_cfg = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_t < 0.0f) {
        airpf::set_create_error("autotune: no candidate tiling could be created");
        return AIRPF_ERR_UNSUPPORTED;
    }
    *best = best_cfg;
    *best_ms = best_t;
    return AIRPF_OK;
}

}  // extern "C"
