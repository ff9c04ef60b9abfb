// airpf_step.cu -- host-side entry points of the AIRPF step kernels: launch
// geometry, shared-memory sizing, and dispatch to the instantiations
// (airpf_launch_inst.cu) of the templates in airpf_step_impl.cuh.
#include "airpf.h"
#include "airpf_step_impl.cuh"

namespace airpf {

// the instantiations compiled in airpf_launch_inst.cu, one object per triple
#define AIRPF_EXTERN_DISPATCH(R, MODEL, PPT) \
    extern template cudaError_t dispatch_inst<R, MODEL, PPT>(const StepParams&, int, cudaStream_t, int, int*);
AIRPF_EXTERN_DISPATCH(float, AR1, 2)
AIRPF_EXTERN_DISPATCH(float, AR1, 4)
AIRPF_EXTERN_DISPATCH(float, SV, 2)
AIRPF_EXTERN_DISPATCH(float, SV, 4)
AIRPF_EXTERN_DISPATCH(float, SV, 8)
AIRPF_EXTERN_DISPATCH(float, NGM, 2)
AIRPF_EXTERN_DISPATCH(float, NGM, 4)
AIRPF_EXTERN_DISPATCH(float, NGM, 8)
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
    // particles per thread: requested (2, 4, or 8, compiled for the FP32 SV and NGM
    // filters only; airpf_create asks for 8 on their split steps), else 2 up to M = 64
    // (one warp per island) and 4 above (measured fastest for fused steps at M = 256);
    // threads per island a multiple of 32 covering M; islands per CTA: the requested count
    // (up to 512 threads; a whole filter when want_g >= m and it fits) or 256 threads' worth
    int pp = (want_ppt == 2 || want_ppt == 4 || want_ppt == 8) ? want_ppt : (M <= 64 ? 2 : 4);
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
    if constexpr (sizeof(R) == 4 && (MODEL == SV || MODEL == NGM))
        if (p.ppt == 8) return dispatch_inst<R, MODEL, 8>(p, t, stream, op, fits);
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

// The output measures' moments of step t + 1 for filter c (grid T x min(B, 65535),
// 256 threads): out[c][t][s][0..dx) = E[x_d], out[c][t][s][dx..2dx) = E[x_d^2] under
// pi^N_{t,s} = sum_k W^k_{t,s} M^-1 sum_i delta(xi^{k,i}_{t,s}) / sum_k W^k_{t,s}, with
// s = 0 the mutated particles and W_{t,0}, s = 1 the internally resampled particles and
// W_{t,1}.  Every sum runs in a fixed order (deterministic); NaN when every W is 0.
constexpr int kMomThreads = 256;

__global__ void __launch_bounds__(kMomThreads) moments_kernel(StepParams p, double* out)
{
    __shared__ double part[kMomThreads / 32][2 * kMaxDx + 1];
    __shared__ double wmax[kMomThreads / 32];
    const int t = blockIdx.x, dx = p.dx, m = p.m, nw = p.fm_nw, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int c = blockIdx.y; c < p.B; c += gridDim.y) {
        const double* fw = p.fw + ((size_t)c * p.T + t) * m * 2;
        const double* fs = p.fsum + ((size_t)c * p.T + t) * m * nw * 4 * dx;
        for (int s = 0; s < 2; ++s) {
            double mx = -INFINITY;
            for (int k = tid; k < m; k += blockDim.x) mx = fmax(mx, fw[k * 2 + s]);
            mx = warp_max(mx);
            if (lane == 0) wmax[warp] = mx;
            __syncthreads();
            mx = -INFINITY;
            for (int w = 0; w < nwarps; ++w) mx = fmax(mx, wmax[w]);
            double acc[2 * kMaxDx + 1];
#pragma unroll
            for (int j = 0; j <= 2 * kMaxDx; ++j) acc[j] = 0.0;
            if (mx > -INFINITY) {
                for (int k = tid; k < m; k += blockDim.x) {
                    const double wk = exp(fw[k * 2 + s] - mx);
                    acc[2 * kMaxDx] += wk;
#pragma unroll
                    for (int j = 0; j < 2 * kMaxDx; ++j) {
                        if (j < 2 * dx) {
                            double sj = 0.0;
                            for (int v = 0; v < nw; ++v) sj += fs[((size_t)k * nw + v) * 4 * dx + s * 2 * dx + j];
                            acc[j] += wk * sj;
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j <= 2 * kMaxDx; ++j) {
                const double v = warp_sum(acc[j]);
                if (lane == 0) part[warp][j] = v;
            }
            __syncthreads();
            if (tid < 2 * dx) {
                double num = 0.0, den = 0.0;
                for (int w = 0; w < nwarps; ++w) {
                    num += part[w][tid];
                    den += part[w][2 * kMaxDx];
                }
                out[(((size_t)c * p.T + t) * 2 + s) * 2 * dx + tid] = mx > -INFINITY ? num / (den * (double)p.M) : NAN;
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_moments(const StepParams& p, double* out, cudaStream_t stream)
{
    if (p.fmom == 0 || p.fw == nullptr || p.fsum == nullptr) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)p.T, (unsigned)(p.B < 65535 ? p.B : 65535));
    moments_kernel<<<grid, kMomThreads, 0, stream>>>(p, out);
    return cudaGetLastError();
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

// the FP64 path's double functions over an array (a test hook): 0 exp, 1 log,
// 2 sin(2 pi x), 3 cos(2 pi x)
__global__ void math_tab_kernel(int fn, const double* x, double* y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    {
        if (fn == 0) y[i] = exp_tab(x[i]);
        else if (fn == 1) y[i] = log_tab(x[i]);
        else if (fn == 2 || fn == 3) {
            double sv, cv;
            sincos2pi_tab(x[i], &sv, &cv);
            y[i] = fn == 2 ? sv : cv;
        } else {                       // functions of a 32-bit word w (given as a double)
            const uint32_t w = (uint32_t)x[i];
            if (fn == 4) y[i] = unif_f64(w);
            else if (fn == 5) y[i] = log_unif(w);
            else {
                double sv, cv;
                sincos2pi_unif(w, &sv, &cv);
                y[i] = fn == 6 ? sv : cv;
            }
        }
    }
}

}  // namespace airpf

extern "C" airpf_status airpf_debug_math(int32_t fn, const double* d_x, double* d_y, int64_t n, void* stream)
{
    if (fn < 0 || fn > 7 || n < 0 || (n > 0 && (!d_x || !d_y))) return AIRPF_ERR_ARG;
    if (n == 0) return AIRPF_OK;
    const int64_t blocks64 = (n + 255) / 256;
    const int blocks = (int)(blocks64 < 4096 ? blocks64 : 4096);
    airpf::math_tab_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(fn, d_x, d_y, n);
    return cudaGetLastError() == cudaSuccess ? AIRPF_OK : AIRPF_ERR_CUDA;
}
