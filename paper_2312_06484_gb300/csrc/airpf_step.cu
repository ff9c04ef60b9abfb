// airpf_step.cu -- host-side entry points of the AIRPF step kernels: launch
// geometry, shared-memory sizing, and dispatch to the instantiations
// (airpf_launch_inst.cu) of the templates in airpf_step_impl.cuh.
#include "airpf_step_impl.cuh"

namespace airpf {

// the instantiations compiled in airpf_launch_inst.cu, one object per triple
#define AIRPF_EXTERN_DISPATCH(R, MODEL, PPT) \
    extern template cudaError_t dispatch_inst<R, MODEL, PPT>(const StepParams&, int, cudaStream_t, int, int*);
AIRPF_EXTERN_DISPATCH(float, AR1, 2)
AIRPF_EXTERN_DISPATCH(float, AR1, 4)
AIRPF_EXTERN_DISPATCH(float, SV, 2)
AIRPF_EXTERN_DISPATCH(float, SV, 4)
AIRPF_EXTERN_DISPATCH(float, NGM, 2)
AIRPF_EXTERN_DISPATCH(float, NGM, 4)
AIRPF_EXTERN_DISPATCH(float, LGSSM, 2)
AIRPF_EXTERN_DISPATCH(float, LGSSM, 4)
AIRPF_EXTERN_DISPATCH(float, TOY, 2)
AIRPF_EXTERN_DISPATCH(float, TOY, 4)
AIRPF_EXTERN_DISPATCH(float, CP, 2)
AIRPF_EXTERN_DISPATCH(float, CP, 4)
AIRPF_EXTERN_DISPATCH(double, AR1, 2)
AIRPF_EXTERN_DISPATCH(double, AR1, 4)
AIRPF_EXTERN_DISPATCH(double, SV, 2)
AIRPF_EXTERN_DISPATCH(double, SV, 4)
AIRPF_EXTERN_DISPATCH(double, NGM, 2)
AIRPF_EXTERN_DISPATCH(double, NGM, 4)
AIRPF_EXTERN_DISPATCH(double, LGSSM, 2)
AIRPF_EXTERN_DISPATCH(double, LGSSM, 4)
AIRPF_EXTERN_DISPATCH(double, TOY, 2)
AIRPF_EXTERN_DISPATCH(double, TOY, 4)
AIRPF_EXTERN_DISPATCH(double, CP, 2)
AIRPF_EXTERN_DISPATCH(double, CP, 4)
#undef AIRPF_EXTERN_DISPATCH

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

template <typename R, int MODEL>
static cudaError_t dispatch_model(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    if (p.ppt == 2) return dispatch_inst<R, MODEL, 2>(p, t, stream, op, fits);
    if (p.ppt == 4) return dispatch_inst<R, MODEL, 4>(p, t, stream, op, fits);
    return cudaErrorInvalidValue;
}

template <typename R>
static cudaError_t dispatch_typed(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    switch (p.model) {
    case AR1: return dispatch_model<R, AR1>(p, t, stream, op, fits);
    case SV: return dispatch_model<R, SV>(p, t, stream, op, fits);
    case NGM: return dispatch_model<R, NGM>(p, t, stream, op, fits);
    case LGSSM: return dispatch_model<R, LGSSM>(p, t, stream, op, fits);
    case TOY: return dispatch_model<R, TOY>(p, t, stream, op, fits);
    case CP: return dispatch_model<R, CP>(p, t, stream, op, fits);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t dispatch(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    return p.fp64 ? dispatch_typed<double>(p, t, stream, op, fits) : dispatch_typed<float>(p, t, stream, op, fits);
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

bool wide_fused_fits(const StepParams& p)
{
    int fits = 0;
    return dispatch(p, 0, nullptr, OP_WIDE_FITS, &fits) == cudaSuccess && fits;
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
