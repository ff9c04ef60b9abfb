// airpf_step.cu -- host-side entry points of the AIRPF step kernels: launch
// geometry, shared-memory sizing, and dispatch to the per-precision
// instantiations (airpf_launch_f32.cu, airpf_launch_f64.cu) of the templates in
// airpf_step_impl.cuh.
#include "airpf_step_impl.cuh"

namespace airpf {

cudaError_t dispatch_f32(const StepParams& p, int t, cudaStream_t stream, int op, int* fits);
cudaError_t dispatch_f64(const StepParams& p, int t, cudaStream_t stream, int op, int* fits);

// ---------------------------------------------------------------------------
size_t step_smem_bytes(const StepParams& p) { return make_layout(p).total; }

size_t model_par_bytes() { return sizeof(ModelPar<double>); }

void choose_mapping(int m, int M, int fp64, int want_ppt, int want_g, int* tpi, int* ppt, int* G)
{
    (void)fp64;
    // particles per thread: requested (2 or 4), else 2 up to M = 64 (one warp per
    // island) and 4 above (measured fastest at M = 256: fewer threads per island)
    // (the kernels are compiled for these two); threads per island a multiple of
    // 32 covering M; islands per CTA: the requested count (up to 512 threads; a
    // whole filter when want_g >= m and it fits) or 256 threads' worth
    int pp = (want_ppt == 2 || want_ppt == 4) ? want_ppt : (M <= 64 ? 2 : 4);
    int t = 32;
    while (t * pp < M && t < kDefaultThreads) t *= 2;
    if (t * pp < M) {
        pp = 4;
        while (t * pp < M && t < kDefaultThreads) t *= 2;
    }
    *tpi = t;
    *ppt = pp;
    int g = kDefaultThreads / t;
    if (g < 1) g = 1;
    if (want_g >= m && m * t <= kMaxCtaThreads) g = m;
    else if (want_g > 0) g = want_g * t <= kMaxThreads ? want_g : kMaxThreads / t;
    while (g > 1 && (g & (g - 1))) --g;      // a power of 2 dividing m
    if (g > m) g = m;
    *G = g < 1 ? 1 : g;
}

int max_cta_threads() { return kMaxCtaThreads; }

template <typename R, int MODEL, int DX>
static cudaError_t launch_typed(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    const size_t smem = step_smem_bytes(p);
    const int block = p.G * p.tpi;
    const int grid = p.B * (p.m / p.G);
    const int want = smem > 48 * 1024 ? (int)smem : 48 * 1024;
    if (op == OP_PREPARE) {
        // opt in to more than 48 KB of dynamic shared memory (outside any capture)
        cudaError_t e = cudaFuncSetAttribute(airpf_step_kernel<R, MODEL, DX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(airpf_persistent_kernel<R, MODEL, DX, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(airpf_persistent_kernel<R, MODEL, DX, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        return e;
    }
    if (op == OP_FITS) {
        // can every CTA of the grid-persistent kernel be resident at once?
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, airpf_persistent_kernel<R, MODEL, DX, true>,
                                                              block, smem);
        *fits = (e == cudaSuccess && block <= kMaxThreads && (long long)per_sm * sms >= grid) ? 1 : 0;
        return e;
    }
    if (op == OP_PERSIST_GRID) {
        StepParams q = p;
        void* args[] = {&q};
        return cudaLaunchCooperativeKernel((const void*)airpf_persistent_kernel<R, MODEL, DX, true>, dim3(grid),
                                           dim3(block), args, smem, stream);
    }
    if (op == OP_PERSIST_CTA) {
        airpf_persistent_kernel<R, MODEL, DX, false><<<grid, block, smem, stream>>>(p);
        return cudaGetLastError();
    }
    if (t == 0) {
        const int n = p.B > p.T ? p.B : p.T;
        airpf_prologue_kernel<R, MODEL><<<(n + 127) / 128, 128, 0, stream>>>(p);
        return cudaGetLastError();
    }
    airpf_step_kernel<R, MODEL, DX><<<grid, block, smem, stream>>>(p, t);
    return cudaGetLastError();
}

static cudaError_t dispatch(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    return p.fp64 ? dispatch_f64(p, t, stream, op, fits) : dispatch_f32(p, t, stream, op, fits);
}

cudaError_t prepare_step(const StepParams& p) { return dispatch(p, 0, nullptr, OP_PREPARE, nullptr); }

cudaError_t launch_step(const StepParams& p, int t, cudaStream_t stream)
{
    return dispatch(p, t, stream, OP_STEP, nullptr);
}

cudaError_t launch_cascade(const StepParams& p, int t, cudaStream_t stream)
{
    return dispatch(p, t, stream, OP_CASCADE, nullptr);
}

cudaError_t launch_persistent(const StepParams& p, bool grid, cudaStream_t stream)
{
    return dispatch(p, 0, stream, grid ? OP_PERSIST_GRID : OP_PERSIST_CTA, nullptr);
}

bool persistent_grid_fits(const StepParams& p)
{
    int fits = 0;
    return dispatch(p, 0, nullptr, OP_FITS, &fits) == cudaSuccess && fits;
}

__global__ void set_run_kernel(RunParams* r, uint32_t iter, uint32_t chain0)
{
    r->iter = iter;
    r->chain0 = chain0;
}

cudaError_t launch_set_run(RunParams* d_run, uint32_t iter, uint32_t chain0, cudaStream_t stream)
{
    set_run_kernel<<<1, 1, 0, stream>>>(d_run, iter, chain0);
    return cudaGetLastError();
}

}  // namespace airpf
