// airpf_grad.cu -- gradient of log Z^N_T with respect to theta, after a forward
// pass that recorded the lineage, s*, the island log-weights and checkpointed
// states (record AIRPF_RECORD_GRAD).
//
// Adjoint with the lineage held fixed.  With the random numbers, the
// ancestors, the island choices and s* fixed, log Z = log sum_k W^k_{T,1} is a
// smooth function of theta through the particles x_t = f(parent, z_t) and the
// observation densities.  Reverse mode gives
//   d log Z / d l_t(k,i) = pi_t(k) w_t(k,i),
// where w_t(k,i) is particle i's normalised weight within island k and pi_t(k)
// the island's smoothing weight: pi_T(k) = W^k_{T,1} / sum_j W^j_{T,1}, and,
// going back, each block of 2^(s*_{t-1} - 1) islands hands its total pi_t mass
// to its members in proportion to W^j_{t-1,1} (the block averaging of the
// interaction stages, eq. (3), is linear and symmetric).  Particle adjoints
// x^_t = x^ from the children + l^ dl/dx flow to the parents through
// (df/dparent)^T by atomic scatter-add along the lineage; theta^ collects
// l^ dl/dtheta + x^ df/dtheta (and the prior's dependence at t = 1).
//
// Fisher-identity score along the lineages: every time-t particle carries the
// final weight delta_t of its descendants (delta_T = pi_T w_T, scattered back
// along the lineage), and score = sum_t sum_q delta_t(q) grad_theta
// [log f(x_t^q | parent) + log g(y_t | x_t^q)] + the prior's term.
//
// States between checkpoints are recomputed from the previous state, the
// lineage and the regenerated transition noise.  Particle arithmetic and the
// per-thread and per-warp sums, the particle adjoints and the descendant weights in
// the pass's precision R; smoothing weights and the CTA and island sums of the
// theta terms in double.
#include <climits>

#include "airpf_device.cuh"
#include "airpf_internal.h"

namespace airpf {
namespace {

constexpr int kGradThreads = 128;

// time-t particles [N][DX] of filter c (a particle's DX components together):
// a checkpoint slot, or the recomputed states of block t / ckpt (two block buffers,
// by the block's parity: one is recomputed while the adjoint steps use the other)
template <typename R, int DX>
__device__ __forceinline__ R* xstate(const StepParams& p, int c, int t)
{
    const size_t per = (size_t)DX * p.N;
    int slot = -1;
    if (t == 0) slot = 0;
    else if (t % p.ckpt == 0) slot = t / p.ckpt;
    else if (t == p.T) slot = p.nck - 1;
    if (slot >= 0) return reinterpret_cast<R*>(p.xck) + ((size_t)c * p.nck + slot) * per;
    const size_t buf = (size_t)((t / p.ckpt) & 1);
    return reinterpret_cast<R*>(p.xblk) + ((buf * p.B + c) * p.ckpt + (t % p.ckpt)) * per;
}

// a particle's DX components from/to the [N][DX] layout (two 16-byte accesses for 8 floats)
template <typename R, int DX>
__device__ __forceinline__ void load_state(const R* base, size_t g, int dx, R* x)
{
    if constexpr (DX == 8 && sizeof(R) == 4) {
        const float4 a = __ldcg(reinterpret_cast<const float4*>(base + g * 8));
        const float4 b = __ldcg(reinterpret_cast<const float4*>(base + g * 8) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
        for (int d = 0; d < DX; ++d) x[d] = (d < dx) ? base[g * DX + d] : (R)0;
    }
}

template <typename R, int DX>
__device__ __forceinline__ void store_state(R* base, size_t g, int dx, const R* x)
{
    if constexpr (DX == 8 && sizeof(R) == 4) {
        reinterpret_cast<float4*>(base + g * 8)[0] = make_float4(x[0], x[1], x[2], x[3]);
        reinterpret_cast<float4*>(base + g * 8)[1] = make_float4(x[4], x[5], x[6], x[7]);
    } else {
#pragma unroll
        for (int d = 0; d < DX; ++d)
            if (d < dx) base[g * DX + d] = x[d];
    }
}

// index among the time-(t-1) particles of the parent of time-t particle g
__device__ __forceinline__ int parent_of(const StepParams& p, int c, int t, int g)
{
    return t == 1 ? g : __ldcg(&p.anc[((size_t)c * p.T + (t - 2)) * p.N + g]);
}

// The LGSSM's A and C as a kernel parameter, rows padded to kMaxDx: with the
// loops over rows and columns unrolled, every element is a constant operand
// of its instruction (no load).
template <typename R>
struct ModelMat {
    R A[kMaxDx * kMaxDx];
    R C[kMaxDy * kMaxDx];
};

// transition x = A parent + sqrt(q) z in the order of the forward pass's
// model_transition (diagonal of A from theta), so recomputed states equal the
// recorded ones
template <typename R, int MODEL, int DX>
__device__ __forceinline__ void transition_mm(const ModelPar<R>& mp, int dx, const R* xp, R* x, const ModelMat<R>& mm,
                                              const R* z)
{
    if (MODEL != LGSSM) {
        model_transition<R, MODEL, DX>(mp, dx, xp, x, nullptr, z, 0u);
    } else {
#pragma unroll
        for (int r = 0; r < DX; ++r) {
            if (r < dx) {
                R acc = 0;
#pragma unroll
                for (int cc = 0; cc < DX; ++cc)
                    if (cc < dx) acc += ((r == cc) ? mp.th[r] : mm.A[r * kMaxDx + cc]) * xp[cc];
                x[r] = acc + mp.c0 * z[r];
            }
        }
    }
}

// log g(y | x) in the order of the forward pass's model_logg
template <typename R, int MODEL, int DX>
__device__ __forceinline__ R logg_mm(const ModelPar<R>& mp, const R* y, int dx, int dy, const R* x,
                                     const ModelMat<R>& mm)
{
    if (MODEL != LGSSM) return model_logg<R, MODEL, DX>(mp, y, dx, dy, x, nullptr);
    R l;
    {
        R ss = 0;
#pragma unroll
        for (int o = 0; o < kMaxDy; ++o) {
            if (o < dy) {
                R e = y[o];
#pragma unroll
                for (int cc = 0; cc < DX; ++cc)
                    if (cc < dx) e -= mm.C[o * kMaxDx + cc] * x[cc];
                ss += e * e;
            }
        }
        l = mp.c2 - ss * mp.c1;
    }
    return (l > -INFINITY) ? l : (R)(-INFINITY);
}

// x_t of the particles between checkpoints: x_t(g) = f(x_{t-1}(parent), z_t(g))
// Launched dependently on the kernel before it (the previous step's recompute): the
// noise is drawn before the wait, the parent states (that kernel's output) read after.
template <typename R, int MODEL, int DX>
__global__ void __launch_bounds__(256) grad_recompute_kernel(StepParams p, const __grid_constant__ ModelMat<R> mm,
                                                              int t)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int c = blockIdx.y;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    ModelPar<R> mp = reinterpret_cast<const ModelPar<R>*>(p.mpar)[c];
    if (MODEL == NGM) mp.drift = reinterpret_cast<const R*>(p.drift)[t - 1];
    const RunParams run = *p.run;
    const Stream st{p.seed_lo, p.seed_hi, run.iter, (run.chain0 + (uint32_t)c) << 8};
    const int dx = p.dx;
    const bool has = g < p.N;
    R xp[DX], x[DX], z[DX > 1 ? DX : 1];
    uint32_t w0 = 0, w2 = 0;
    int par = 0;
    if (has) {
        model_step_noise<R, MODEL, DX>(mp, st, (uint32_t)g, (uint32_t)t, dx, z, w0, w2);
        par = parent_of(p, c, t, g);                 // the forward pass's lineage
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (!has) return;
    const R* xprev = xstate<R, DX>(p, c, t - 1);
    R* xt = xstate<R, DX>(p, c, t);
    load_state<R, DX>(xprev, (size_t)par, dx, xp);
    transition_mm<R, MODEL, DX>(mp, dx, xp, x, mm, z);
    store_state<R, DX>(xt, (size_t)g, dx, x);
}

// pi_T(k) = W^k_{T,1} / sum_j W^j_{T,1}: one CTA per filter
__global__ void __launch_bounds__(256) grad_pi_final_kernel(StepParams p)
{
    __shared__ double red[32];
    const int c = blockIdx.x, m = p.m;
    const double* lw = p.logw + ((size_t)c * p.T + (p.T - 1)) * m;
    double mx = -INFINITY;
    for (int k = threadIdx.x; k < m; k += blockDim.x) mx = fmax(mx, lw[k]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    __syncthreads();
    double sum = 0.0;
    if (mx > -INFINITY)
        for (int k = threadIdx.x; k < m; k += blockDim.x) sum += exp(lw[k] - mx);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    double* pi = p.gpi[p.T & 1] + (size_t)c * m;
    for (int k = threadIdx.x; k < m; k += blockDim.x)
        pi[k] = (sum > 0.0 && lw[k] > -INFINITY) ? exp(lw[k] - mx) / sum : 0.0;
}

// mean of the transition from the parent, and its scale (z = (x - mean) / scale)
template <typename R, int MODEL, int DX>
__device__ __forceinline__ void transition_mean(const ModelPar<R>& mp, int dx, const R* xp, const ModelMat<R>& mm,
                                                R* mu, R& s)
{
    if (MODEL == AR1) {
        mu[0] = mp.th[0] * xp[0];
        s = mp.th[1];
    } else if (MODEL == SV) {
        mu[0] = mp.th[0] + mp.th[1] * (xp[0] - mp.th[0]);
        s = mp.th[2];
    } else if (MODEL == NGM) {
        const R v = xp[0];
        mu[0] = (R)0.5 * v + fdiv<R>((R)25 * v, (R)1 + v * v) + mp.drift;   // as the forward transition
        s = mp.c0;                       // sqrt(q)
    } else {
#pragma unroll
        for (int r = 0; r < DX; ++r) {
            if (r < dx) {
                R acc = 0;
#pragma unroll
                for (int cc = 0; cc < DX; ++cc)
                    if (cc < dx) acc += ((r == cc) ? mp.th[r] : mm.A[r * kMaxDx + cc]) * xp[cc];
                mu[r] = acc;
            }
        }
        s = mp.c0;                       // sqrt(q)
    }
}

// Step t of the backward pass: one CTA per island.  Resident CTAs a SM: 7 in FP32 (at
// most 72 registers; m = 2048 islands then take two waves of the 152 SMs instead of
// 2.25), 6 in FP64 (which would spill heavily at 72).
template <typename R>
constexpr int grad_island_min_ctas() { return sizeof(R) == 4 ? 7 : 6; }

template <typename R, int MODEL, int DX>
__global__ void __launch_bounds__(kGradThreads, grad_island_min_ctas<R>()) grad_island_kernel(StepParams p, const __grid_constant__ ModelMat<R> mm,
                                                                   int t, int dep)
{
    // launched dependently on step t+1's kernel (programmatic dependent launch): the
    // next kernel may start once every CTA of this one has, and this one reads step
    // t+1's outputs (adjoints, descendant weights, pi_{t+1}) only after the wait below
    if (dep) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char gsm[];
    __shared__ R yv[kMaxDy];
    __shared__ R tsum[2 * kMaxTheta][kGradThreads + 1];   // the threads' theta terms, a row per term
    __shared__ R tpart[kGradThreads];
    __shared__ double pred[2][kGradThreads / 32];
    __shared__ R rmx[kGradThreads / 32];
    __shared__ R rsum[kGradThreads / 32];
    R* lsm = reinterpret_cast<R*>(gsm);                  // [M] log-weights of the island
    const int c = blockIdx.y, k = blockIdx.x;
    const int M = p.M, N = p.N, dx = p.dx, dy = p.dy, td = p.theta_dim;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const R* xt = xstate<R, DX>(p, c, t);
    const R* xprev = xstate<R, DX>(p, c, t - 1);
    // particle adjoints x^ [N][DX] (a particle's components together: vector atomics
    // to its parent) and descendant weights [N], in the pass's precision; buffer t % 3
    // holds step t's inputs and is cleared as it is read (it is step t-3's output buffer)
    const size_t xo = (size_t)c * N * DX;
    R* xh_in = reinterpret_cast<R*>(p.xh[t % 3]) + xo;
    R* xh_out = reinterpret_cast<R*>(p.xh[(t + 2) % 3]) + xo;
    R* dh_in = reinterpret_cast<R*>(p.dh[t % 3]) + (size_t)c * N;
    R* dh_out = reinterpret_cast<R*>(p.dh[(t + 2) % 3]) + (size_t)c * N;
    // the thread's first particle (the only one when M <= blockDim): its state, parent,
    // parent state, adjoint and descendant weight are loaded first, so that these loads
    // (two dependent rounds) are in flight during the island's softmax
    const bool pre = tid < M;
    const int g0 = k * M + tid;
    int par0 = 0;
    R x0[DX], xp0[DX], xh0[DX], dh0 = (R)0;
#pragma unroll
    for (int d = 0; d < DX; ++d) x0[d] = xp0[d] = xh0[d] = (R)0;
    // (the states, the lineage, y and the forward pass's records are earlier kernels' outputs)
    if (pre) {
        par0 = parent_of(p, c, t, g0);
        load_state<R, DX>(xt, (size_t)g0, dx, x0);
        load_state<R, DX>(xprev, (size_t)par0, dx, xp0);
    }
    for (int o = tid; o < dy; o += blockDim.x) yv[o] = (R)p.y[(size_t)(t - 1) * dy + o];
    __syncthreads();
    ModelPar<R> mp = reinterpret_cast<const ModelPar<R>*>(p.mpar)[c];
    if (MODEL == NGM) mp.drift = reinterpret_cast<const R*>(p.drift)[t - 1];

    // island softmax of the log-weights
    R mx = (R)(-INFINITY);
    for (int i = tid; i < M; i += blockDim.x) {
        const int g = k * M + i;
        R x[DX];
        if (i == tid) {
#pragma unroll
            for (int d = 0; d < DX; ++d) x[d] = x0[d];
        } else {
            load_state<R, DX>(xt, (size_t)g, dx, x);
        }
        const R l = logg_mm<R, MODEL, DX>(mp, yv, dx, dy, x, mm);
        lsm[i] = l;
        mx = l > mx ? l : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const R v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    if (lane == 0) rmx[warp] = mx;
    __syncthreads();
    mx = rmx[0];
    for (int w = 1; w < nw; ++w) mx = rmx[w] > mx ? rmx[w] : mx;
    R sum = 0;
    if (mx > (R)(-INFINITY))
        for (int i = tid; i < M; i += blockDim.x) sum += exp(lsm[i] - mx);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) rsum[warp] = sum;
    __syncthreads();
    sum = 0;
    for (int w = 0; w < nw; ++w) sum += rsum[w];
    const R inv_sum = sum > (R)0 ? (R)1 / sum : (R)0;

    // step t+1's outputs from here on
    if (dep) asm volatile("griddepcontrol.wait;" ::: "memory");
    if (pre) {
        load_state<R, DX>(xh_in, (size_t)g0, dx, xh0);
        if (t < p.T) dh0 = dh_in[g0];
    }
    // pi_t(k): at t = T from grad_pi_final_kernel; before, from pi_{t+1} of the block of
    // r^(s*_t - 1) = 2^lvl islands holding k (r = 2^rb the radix), whose pi_{t+1} mass
    // the block hands to its members in proportion to W_{t,1} (the averaging of the
    // interaction stages is linear and symmetric); computed by the island's own CTA and
    // written for step t-1's CTAs
    double pik = 0.0;
    if (t == p.T) {
        pik = p.gpi[t & 1][(size_t)c * p.m + k];
    } else {
        const int lvl = (p.sstar[(size_t)c * p.T + (t - 1)] - 1) * p.rb;
        const double* pin = p.gpi[(t + 1) & 1] + (size_t)c * p.m;
        if (lvl == 0) {
            pik = pin[k];
        } else {
            const int n = 1 << lvl, j0 = (k >> lvl) << lvl;
            const double* lw = p.logw + ((size_t)c * p.T + (t - 1)) * p.m;
            double lmx = -INFINITY, mass = 0.0;
            for (int j = j0 + tid; j < j0 + n; j += blockDim.x) {
                lmx = fmax(lmx, lw[j]);
                mass += pin[j];
            }
            for (int o = 16; o > 0; o >>= 1) {
                lmx = fmax(lmx, __shfl_xor_sync(0xffffffffu, lmx, o));
                mass += __shfl_xor_sync(0xffffffffu, mass, o);
            }
            if (lane == 0) {
                pred[0][warp] = lmx;
                pred[1][warp] = mass;
            }
            __syncthreads();
            lmx = pred[0][0];
            mass = pred[1][0];
            for (int w = 1; w < nw; ++w) {
                lmx = fmax(lmx, pred[0][w]);
                mass += pred[1][w];
            }
            double sw = 0.0;
            if (lmx > -INFINITY)
                for (int j = j0 + tid; j < j0 + n; j += blockDim.x) sw += exp(lw[j] - lmx);
            for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(0xffffffffu, sw, o);
            __syncthreads();                              // pred read above
            if (lane == 0) pred[0][warp] = sw;
            __syncthreads();
            sw = 0.0;
            for (int w = 0; w < nw; ++w) sw += pred[0][w];
            pik = (sw > 0.0 && lw[k] > -INFINITY) ? exp(lw[k] - lmx) / sw * mass : 0.0;
        }
        if (tid == 0) p.gpi[t & 1][(size_t)c * p.m + k] = pik;
    }
    const R pik_r = (R)pik;

    // per-thread sums in the pass's precision (a thread holds few particles),
    // the CTA and grid reductions in double
    // the thread's theta terms accumulate in its column of tsum (rows 0..td-1 the adjoint
    // terms, td..2td-1 the score terms): registers stay free for the particle arithmetic
    for (int d = 0; d < 2 * td; ++d) tsum[d][tid] = (R)0;
    auto ga = [&](int d) -> R& { return tsum[d][tid]; };
    auto gs = [&](int d) -> R& { return tsum[td + d][tid]; };
    for (int i = tid; i < M; i += blockDim.x) {
        const int g = k * M + i;
        const R wi = (lsm[i] > (R)(-INFINITY)) ? exp(lsm[i] - mx) * inv_sum : (R)0;
        const R lhat = pik_r * wi;                                   // d log Z / d l_t(k,i)
        const bool first = (i == tid);
        const R delta = (t == p.T) ? lhat : (first ? dh0 : dh_in[g]);   // descendant weight
        const int par = first ? par0 : parent_of(p, c, t, g);
        R x[DX], xp[DX], mu[DX];
        R s;
        R xhat[DX], v[DX];
        if (first) {
#pragma unroll
            for (int d = 0; d < DX; ++d) {
                x[d] = x0[d];
                xp[d] = xp0[d];
                xhat[d] = xh0[d];
            }
        } else {
            load_state<R, DX>(xt, (size_t)g, dx, x);
            load_state<R, DX>(xprev, (size_t)par, dx, xp);
            load_state<R, DX>(xh_in, (size_t)g, dx, xhat);
        }
        transition_mean<R, MODEL, DX>(mp, dx, xp, mm, mu, s);
        if (MODEL == AR1) {
            const R a = mp.th[0], sv = mp.th[1], sw = mp.th[2], s0 = mp.th[3];
            const R e = yv[0] - x[0];
            const R zz = (x[0] - mu[0]) / sv;
            const R dsw = (R)(-1) / sw + e * e / (sw * sw * sw);
            xhat[0] += lhat * e / (sw * sw);
            ga(0) += xhat[0] * xp[0];
            ga(1) += xhat[0] * zz;
            ga(2) += lhat * dsw;
            v[0] = a * xhat[0];
            gs(0) += delta * zz * xp[0] / sv;
            gs(1) += delta * (zz * zz - (R)1) / sv;
            gs(2) += delta * dsw;
            if (t == 1) {                          // x_0 = sigma_0 z_0
                const R x0 = xp[0];
                ga(3) += v[0] * x0 / s0;
                gs(3) += delta * (x0 * x0 / (s0 * s0) - (R)1) / s0;
            }
        } else if (MODEL == SV) {
            // x = mu + phi (parent - mu) + sigma z;  l = -x/2 - y^2 e^-x / 2 + const
            const R mu_ = mp.th[0], phi = mp.th[1], sg = mp.th[2];
            const R zz = (x[0] - mu[0]) / sg;
            xhat[0] += lhat * ((R)(-0.5) + (R)0.5 * yv[0] * yv[0] * exp(-x[0]));
            ga(0) += xhat[0] * ((R)1 - phi);
            ga(1) += xhat[0] * (xp[0] - mu_);
            ga(2) += xhat[0] * zz;
            v[0] = phi * xhat[0];
            gs(0) += delta * zz * ((R)1 - phi) / sg;
            gs(1) += delta * zz * (xp[0] - mu_) / sg;
            gs(2) += delta * (zz * zz - (R)1) / sg;
            if (t == 1) {                          // x_0 = mu + sigma (1 - phi^2)^-1/2 z_0
                const R om = (R)1 - phi * phi;
                const R sd0 = sg / sqrt(om);
                const R z0 = (xp[0] - mu_) / sd0;
                ga(0) += v[0];
                ga(1) += v[0] * z0 * sd0 * phi / om;
                ga(2) += v[0] * z0 * sd0 / sg;
                gs(0) += delta * z0 / sd0;
                gs(1) += delta * (z0 * z0 - (R)1) * phi / om;
                gs(2) += delta * (z0 * z0 - (R)1) / sg;
            }
        } else if (MODEL == NGM) {
            // x = p/2 + 25 p / (1 + p^2) + drift + sqrt(q) z;  l = -log(2 pi r)/2 - (y - x^2/20)^2 / (2 r)
            const R q = mp.th[0], r = mp.th[1], p0 = mp.th[2];
            const R sq = mp.c0;
            const R zz = (x[0] - mu[0]) / sq;
            const R e = yv[0] - ngm_obs_mean<R>(x[0]);
            const R dlr = (R)(-0.5) / r + e * e / ((R)2 * r * r);
            xhat[0] += lhat * e * (x[0] / (R)10) / r;
            ga(0) += xhat[0] * zz / ((R)2 * sq);
            ga(1) += lhat * dlr;
            const R pv = xp[0], den = (R)1 + pv * pv;
            v[0] = xhat[0] * ((R)0.5 + (R)25 * ((R)1 - pv * pv) / (den * den));
            gs(0) += delta * (zz * zz - (R)1) / ((R)2 * q);
            gs(1) += delta * dlr;
            if (t == 1) {                          // x_0 = sqrt(p0) z_0
                const R sp0 = sqrt(p0);
                const R z0 = pv / sp0;
                ga(2) += v[0] * z0 / ((R)2 * sp0);
                gs(2) += delta * (z0 * z0 - (R)1) / ((R)2 * p0);
            }
        } else {
            const R inv_r = (R)2 * mp.c1;          // c1 = 1/(2r)
            R ee[kMaxDy], ss = 0;
#pragma unroll
            for (int o = 0; o < kMaxDy; ++o) {
                ee[o] = 0;
                if (o < dy) {
                    R e = yv[o];
#pragma unroll
                    for (int cc = 0; cc < DX; ++cc)
                        if (cc < dx) e -= mm.C[o * kMaxDx + cc] * x[cc];
                    ee[o] = e;
                    ss += e * e;
                }
            }
            const R dlr = (R)(-0.5) * (R)dy + ss * mp.c1;
            const R inv_s = (R)1 / s;
            R zn = 0, qsum = 0;
#pragma unroll
            for (int d = 0; d < DX; ++d) {
                if (d < dx) {
                    R dl = 0;
#pragma unroll
                    for (int o = 0; o < kMaxDy; ++o)
                        if (o < dy) dl += mm.C[o * kMaxDx + d] * ee[o];
                    xhat[d] += lhat * dl * inv_r;
                    const R zd = (x[d] - mu[d]) * inv_s;
                    ga(d) += xhat[d] * xp[d];                   // A_dd
                    qsum += xhat[d] * (R)0.5 * s * zd;           // log q
                    gs(d) += delta * zd * xp[d] * inv_s;
                    zn += zd * zd;
                }
            }
            // slots dx (log q) and dx + 1 (log r), with static indices (registers, not a stack array)
#pragma unroll
            for (int d = 0; d < kMaxTheta; ++d) {
                if (d == dx) {
                    ga(d) += qsum;
                    gs(d) += delta * (R)0.5 * (zn - (R)dx);
                }
                if (d == dx + 1) {
                    ga(d) += lhat * dlr;
                    gs(d) += delta * dlr;
                }
            }
#pragma unroll
            for (int cc = 0; cc < DX; ++cc) {
                v[cc] = 0;
                if (cc < dx) {
#pragma unroll
                    for (int rr = 0; rr < DX; ++rr)
                        if (rr < dx) v[cc] += ((rr == cc) ? mp.th[rr] : mm.A[rr * kMaxDx + cc]) * xhat[rr];
                }
            }
        }
        if (t >= 2) {                      // to the parent, along the lineage
            if constexpr (DX == 8 && sizeof(R) == 4) {
                // two 16-byte vector atomics (sm_90 and later) for the 8 components
                float4* o = reinterpret_cast<float4*>(&xh_out[(size_t)par * DX]);
                atomicAdd(o, make_float4(v[0], v[1], v[2], v[3]));
                atomicAdd(o + 1, make_float4(v[4], v[5], v[6], v[7]));
            } else {
#pragma unroll
                for (int d = 0; d < DX; ++d)
                    if (d < dx) atomicAdd(&xh_out[(size_t)par * DX + d], v[d]);
            }
            atomicAdd(&dh_out[par], delta);
        }
#pragma unroll
        for (int d = 0; d < DX; ++d)
            if (d < dx) xh_in[(size_t)g * DX + d] = (R)0;
        dh_in[g] = (R)0;
    }
    // the CTA's theta sums, in the pass's precision and a fixed order: every thread's
    // 2 td values into shared memory (a row per term), segments of each row summed by
    // the threads, then the segments; the island's running sums over the steps in double
    // (this CTA alone updates row k of gacc: no atomics; the final sum over the islands
    // runs in island order)
    const int nt = 2 * td;
    __syncthreads();
    const int nseg = blockDim.x / nt;              // segments per term (at least 1: nt <= 20 < 128)
    const int seglen = (blockDim.x + nseg - 1) / nseg;
    if (tid < nt * nseg) {
        const int r = tid % nt, sg = tid / nt;
        const int a0 = sg * seglen, a1 = a0 + seglen < (int)blockDim.x ? a0 + seglen : (int)blockDim.x;
        R acc = (R)0;
        for (int q = a0; q < a1; ++q) acc += tsum[r][q];
        tpart[tid] = acc;
    }
    __syncthreads();
    if (tid < nt) {
        R acc = (R)0;
        for (int sg = 0; sg < nseg; ++sg) acc += tpart[sg * nt + tid];
        double* gacc = p.gacc + ((size_t)c * p.m + k) * 2 * kMaxTheta;
        const int slot = tid < td ? tid : kMaxTheta + tid - td;
        gacc[slot] += (double)acc;
    }
    (void)lane;
    (void)warp;
}

// gout, sout: the islands' running sums of the theta terms, added in island order
__global__ void __launch_bounds__(256) grad_sum_kernel(StepParams p)
{
    __shared__ double red[2 * kMaxTheta][8];
    const int c = blockIdx.x, td = p.theta_dim, m = p.m;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double a[2 * kMaxTheta];
#pragma unroll
    for (int d = 0; d < 2 * kMaxTheta; ++d) a[d] = 0.0;
    for (int k = tid; k < m; k += blockDim.x) {
        const double* acc = p.gacc + ((size_t)c * m + k) * 2 * kMaxTheta;
#pragma unroll
        for (int d = 0; d < 2 * kMaxTheta; ++d) a[d] += acc[d];
    }
#pragma unroll
    for (int d = 0; d < 2 * kMaxTheta; ++d) {
        double v = a[d];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[d][warp] = v;
    }
    __syncthreads();
    if (tid < td) {
        double g = 0.0, sc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            g += red[tid][w];
            sc += red[kMaxTheta + tid][w];
        }
        p.gout[(size_t)c * td + tid] = g;
        p.sout[(size_t)c * td + tid] = sc;
    }
}

template <typename R, int MODEL, int DX>
cudaError_t backward_typed(const StepParams& p, const double* host_md, cudaStream_t stream, cudaStream_t aux,
                           cudaEvent_t* ev)
{
    ModelMat<R> mm;
    for (int i = 0; i < kMaxDx * kMaxDx; ++i) mm.A[i] = (R)0;
    for (int i = 0; i < kMaxDy * kMaxDx; ++i) mm.C[i] = (R)0;
    if (MODEL == LGSSM && host_md) {
        for (int r = 0; r < p.dx; ++r)
            for (int cc = 0; cc < p.dx; ++cc) mm.A[r * kMaxDx + cc] = (R)host_md[r * p.dx + cc];
        for (int o = 0; o < p.dy; ++o)
            for (int cc = 0; cc < p.dx; ++cc) mm.C[o * kMaxDx + cc] = (R)host_md[p.dx * p.dx + o * p.dx + cc];
    }
    const size_t xbytes = (size_t)p.B * DX * p.N * sizeof(R);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMemsetAsync(p.xh[i], 0, xbytes, stream);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMemsetAsync(p.dh[i], 0, sizeof(R) * (size_t)p.B * p.N, stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(p.gacc, 0, sizeof(double) * (size_t)p.B * p.m * 2 * kMaxTheta, stream);
    if (e != cudaSuccess) return e;
    grad_pi_final_kernel<<<p.B, 256, 0, stream>>>(p);
    const size_t smem = sizeof(R) * (size_t)p.M;
    const dim3 pgrid((p.N + 255) / 256, p.B), igrid(p.m, p.B);
    const int K = p.ckpt;
    const int nb = (p.T + K - 1) / K;
    auto steps = [&](int b, int* lo, int* hi) {
        *lo = b * K + 1;
        *hi = (b + 1) * K < p.T ? (b + 1) * K : p.T;
    };
    // the states of block b's steps that are not checkpoints, on the second stream
    // (each recompute launched dependently on the one before it in the block)
    auto recompute = [&](int b) -> cudaError_t {
        int lo, hi;
        steps(b, &lo, &hi);
        cudaError_t r = cudaSuccess;
        bool first = true;
        for (int t = lo; t <= hi && r == cudaSuccess; ++t) {
            if (t % K == 0 || t == p.T) continue;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = pgrid;
            cfg.blockDim = dim3(256);
            cfg.stream = aux;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = first ? 0 : 1;
            r = cudaLaunchKernelEx(&cfg, grad_recompute_kernel<R, MODEL, DX>, p, mm, t);
            first = false;
        }
        return r == cudaSuccess ? cudaEventRecord(ev[1 + (b & 1)], aux) : r;
    };
    // block b's adjoint steps, last step first, once its states are recomputed
    auto adjoint = [&](int b) -> cudaError_t {
        int lo, hi;
        steps(b, &lo, &hi);
        cudaError_t r = cudaStreamWaitEvent(stream, ev[1 + (b & 1)], 0);
        for (int t = hi; t >= lo && r == cudaSuccess; --t) {
            // the first step of a block follows the recomputation in plain stream order;
            // the others start while the step before them finishes
            const int dep = t < hi ? 1 : 0;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = igrid;
            cfg.blockDim = dim3(kGradThreads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = dep;
            r = cudaLaunchKernelEx(&cfg, grad_island_kernel<R, MODEL, DX>, p, mm, t, dep);
        }
        return r == cudaSuccess ? cudaEventRecord(ev[3 + (b & 1)], stream) : r;
    };
    // fork: block b-1 is recomputed while block b's adjoint steps run; its buffer was
    // last read by block b+1's adjoint steps
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev[0], 0);
    if (e == cudaSuccess) e = recompute(nb - 1);
    for (int b = nb - 1; b >= 0 && e == cudaSuccess; --b) {
        if (b >= 1) {
            if (b + 1 <= nb - 1) e = cudaStreamWaitEvent(aux, ev[3 + ((b + 1) & 1)], 0);
            if (e == cudaSuccess) e = recompute(b - 1);
        }
        if (e == cudaSuccess) e = adjoint(b);      // joins the second stream back (block 0 last)
    }
    if (e == cudaSuccess) grad_sum_kernel<<<p.B, 256, 0, stream>>>(p);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

template <typename R>
cudaError_t backward_r(const StepParams& p, const double* host_md, cudaStream_t stream, cudaStream_t aux,
                       cudaEvent_t* ev)
{
    if (p.model == AR1) return backward_typed<R, AR1, 1>(p, host_md, stream, aux, ev);
    if (p.model == SV) return backward_typed<R, SV, 1>(p, host_md, stream, aux, ev);
    if (p.model == NGM) return backward_typed<R, NGM, 1>(p, host_md, stream, aux, ev);
    if (p.model == LGSSM) return backward_typed<R, LGSSM, kMaxDx>(p, host_md, stream, aux, ev);
    return cudaErrorInvalidValue;
}

}  // namespace

bool grad_supported(int model) { return model == AR1 || model == SV || model == NGM || model == LGSSM; }

cudaError_t launch_grad_backward(const StepParams& p, const double* host_md, cudaStream_t stream, cudaStream_t aux,
                                 cudaEvent_t* ev)
{
    if (p.M * (p.fp64 ? 8 : 4) > 48 * 1024) return cudaErrorInvalidValue;
    return p.fp64 ? backward_r<double>(p, host_md, stream, aux, ev) : backward_r<float>(p, host_md, stream, aux, ev);
}

}  // namespace airpf
