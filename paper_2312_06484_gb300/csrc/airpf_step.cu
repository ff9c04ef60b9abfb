// airpf_step.cu -- the AIRPF time step on sm_103a.
//
// One launch per time step t (Algorithm 1 of Heine, arXiv 2312.06484, main
// loop), captured in a CUDA graph by the runtime.  Each CTA owns G islands of
// one filter.  Launch t does, in order:
//
//  1. the interaction cascade of step t-1 (Algorithm 1, stages s = 1..S),
//     recomputed by every CTA of the filter from the m island weights of step
//     t-1 so that no second launch or grid-wide barrier is needed:
//       - island weights W^k_{t-1,1} (extended-range doubles) are rescaled by
//         one common power of two and summed in a binary tree in shared
//         memory; level l holds the sums over aligned blocks of 2^l islands;
//       - after s-1 interacting butterfly stages (eq. (3)) every island weight
//         is the mean of its aligned block of 2^(s-1) islands, so
//         ENF_{t,s} = Tot^2 2^(s-1) / (m sum_b B_{s-1,b}^2) for every stage
//         from the one tree; the interacting stages form a prefix (a stage
//         with alpha = I leaves the weights, hence the ENF, unchanged), so
//         s* = min{s : ENF_s >= tau} (adaptation line of Algorithm 1);
//       - island k's new weight is its block mean at level s*-1 (normalised
//         so that the weights average to 1; log Z accumulates the log of the
//         pre-normalisation mean), and the block it inherits is
//         src(k) = c_1(c_2(...c_{s*-1}(k))) where c_s(j) picks the lower
//         island of {j, j xor 2^(s-1)} iff u_{t,s,j} (W_lo + W_hi) < W_lo;
//  2. the island work of step t for the CTA's islands: mutate the inherited
//     internally-resampled block of island src(k) through K_t (Algorithm 1,
//     last stage), weight by g_t, reduce the island maximum, build the
//     inclusive CDF (FP64, or an exact 2^-31 fixed-point integer prefix sum in
//     FP32 mode), draw M multinomial ancestors by binary search (internal
//     resample), gather, store, and publish W^k_{t,1} = W^k_{t,0} M^-1 sum g.
//
// Launch T+1 runs the final cascade only (it sets log Z and the lineage of
// step T).
#include <climits>
#include <cstdio>

#include "airpf_device.cuh"
#include "airpf_internal.h"

namespace airpf {

namespace {

constexpr int kMaxThreads = 256;
constexpr int kPptMax = 4;
constexpr int kMaxStages = 16;

template <typename R> struct CdfType;
template <> struct CdfType<double> { using T = double; };
template <> struct CdfType<float> { using T = unsigned long long; };

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// offset (in doubles) of tree level l for m leaves: levels 0..S stored back to back
__device__ __forceinline__ int tree_off(int m, int l) { return 2 * m - 2 * (m >> l); }

struct Layout {
    size_t tree, island, small, total;   // byte offsets
    size_t cdf, xs, red, mxr;            // island sub-offsets (per island strides below)
    size_t cdf_stride, xs_stride, red_stride;
};

__host__ __device__ inline Layout make_layout(const StepParams& p)
{
    Layout L;
    const size_t rsz = p.fp64 ? 8 : 4;
    const size_t nwi = (size_t)((p.tpi + 31) / 32);           // warps per island
    const size_t treeb = align16(sizeof(double) * (2 * (size_t)p.m + 2 * kMaxStages + 8));
    L.cdf_stride = sizeof(double) * (size_t)p.M;              // double or u64
    L.xs_stride = align16(rsz * (size_t)p.M * p.dx);
    L.red_stride = sizeof(double) * nwi;
    L.cdf = 0;
    L.xs = L.cdf + align16(L.cdf_stride * p.G);
    L.red = L.xs + L.xs_stride * p.G;
    L.mxr = L.red + align16(L.red_stride * p.G);
    const size_t islandb = L.mxr + align16(L.red_stride * p.G);
    L.tree = 0;
    L.island = 0;                                             // overlaps the tree
    L.small = align16(treeb > islandb ? treeb : islandb);
    const size_t smallb = align16(sizeof(double) * (size_t)p.G) + align16(2 * sizeof(int) * (size_t)p.G)
                          + align16(sizeof(double) * 16)
                          + align16(rsz * (size_t)(p.dx * p.dx + p.dy * p.dx + kMaxDy))
                          + align16(sizeof(ModelPar<double>));
    L.total = L.small + smallb;
    return L;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename V>
__device__ __forceinline__ V warp_max(V v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const V w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v) ? w : v;
    }
    return v;
}

template <typename V>
__device__ __forceinline__ V warp_incl_scan(V v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V w = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += w;
    }
    return v;
}

// Island weight of the cascade: double r in [0.5,1) (or 0) times 2^e.
struct XW {
    double r;
    int e;
};

// v = r 2^e with r in [0.5, 1), by exponent-field manipulation (v > 0 normal);
// falls back to frexp for subnormal inputs.
__device__ __forceinline__ XW xw_from_bits(double v, int e_add)
{
    XW w;
    if (!(v > 0.0)) {
        w.r = 0.0;
        w.e = 0;
        return w;
    }
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) {
        int e2;
        w.r = frexp(v, &e2);
        w.e = e2 + e_add;
        return w;
    }
    w.r = __longlong_as_double((b & ~(0x7ffLL << 52)) | (1022LL << 52));
    w.e = ex - 1022 + e_add;
    return w;
}

__device__ __forceinline__ XW xw_from(double v, int e_add)
{
    XW w;
    if (!(v > 0.0)) {
        w.r = 0.0;
        w.e = 0;
        return w;
    }
    int ex;
    w.r = frexp(v, &ex);
    w.e = ex + e_add;
    return w;
}

// ---------------------------------------------------------------------------
// Cascade of step tp for filter c (see file comment).  Every thread of the CTA
// calls it.  Outputs in shared memory: own_wr/own_we/own_src for the CTA's
// islands; records written by the filter's designated CTA.
// ---------------------------------------------------------------------------
__device__ void cascade(const StepParams& p, int c, int tp, int k0, const Stream& st, double* tree,
                        double* scal, double* own_wr, int* own_we, int* own_src, bool designated)
{
    const int m = p.m, S = p.S, tid = threadIdx.x, nthr = blockDim.x;
    const double* wr = p.wr[tp & 1] + (size_t)c * m;
    const int* we = p.we[tp & 1] + (size_t)c * m;
    double* Q = tree + 2 * m;                 // [kMaxStages]
    int* iscal = reinterpret_cast<int*>(Q + kMaxStages);   // [4]: emax, sstar

    // 1. largest binary exponent among nonzero weights
    int emax = INT_MIN;
    for (int k = tid; k < m; k += nthr) {
        const double r = wr[k];
        if (r > 0.0 && we[k] > emax) emax = we[k];
    }
    emax = warp_max(emax);
    if (tid == 0) iscal[0] = INT_MIN;
    __syncthreads();
    if ((tid & 31) == 0) atomicMax(&iscal[0], emax);
    __syncthreads();
    emax = iscal[0];
    const bool dead = (emax == INT_MIN);

    // 2. leaves rescaled by 2^-emax (exact), then the block-sum tree
    for (int k = tid; k < m; k += nthr) {
        const double r = wr[k];
        tree[k] = (dead || !(r > 0.0)) ? 0.0 : ldexp(r, we[k] - emax);
    }
    __syncthreads();
    for (int l = 1; l <= S; ++l) {
        const int n = m >> l;
        double* dst = tree + tree_off(m, l);
        const double* src = tree + tree_off(m, l - 1);
        for (int b = tid; b < n; b += nthr) dst[b] = src[2 * b] + src[2 * b + 1];
        __syncthreads();
    }
    // 3. per-level sums of squares, one warp per level
    {
        const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
        for (int l = warp; l < S; l += nw) {
            const int n = m >> l;
            const double* v = tree + tree_off(m, l);
            double acc = 0.0;
            for (int b = lane; b < n; b += 32) acc = fma(v[b], v[b], acc);
            acc = warp_sum(acc);
            if (lane == 0) Q[l] = acc;
        }
    }
    __syncthreads();
    // 4. s*: stage s interacts iff ENF_s < tau, i.e. Tot^2 2^(s-1) < tau m Q_{s-1};
    //    tested for all stages at once by the first warp (no division)
    if (tid < 32) {
        const double tot = tree[tree_off(m, S)];
        bool quiet = false;
        if (tid < S) {
            const int s = tid + 1;
            quiet = (tot > 0.0) && !(tot * tot * ldexp(1.0, s - 1) < p.tau * (double)m * Q[s - 1]);
        }
        const unsigned qm = __ballot_sync(0xffffffffu, quiet);
        if (tid == 0) {
            int ss;
            if (p.mode == 0) ss = 1;
            else if (p.mode == 1) ss = S + 1;
            else ss = qm ? (__ffs(qm)) : S + 1;       // first quiet stage
            iscal[1] = ss;
            scal[0] = tot;
            if (designated) {
                const double L = (tot > 0.0) ? log(tot) - log((double)m) + (double)emax * 0.6931471805599453
                                             : -INFINITY;
                const double lz = p.logz[c] + L;
                p.logz[c] = lz;
                if (p.trace) p.trace[(size_t)c * p.T + (tp - 1)] = lz;
                if (p.sstar) p.sstar[(size_t)c * p.T + (tp - 1)] = ss;
                if (p.enf) {
                    double* e = p.enf + ((size_t)c * p.T + (tp - 1)) * (S + 1);
                    double last = 1.0;
                    for (int s = 1; s <= S; ++s) {
                        const int sr = s <= ss ? s : ss;
                        const double v = (tot > 0.0) ? tot * tot * ldexp(1.0, sr - 1) / ((double)m * Q[sr - 1]) : 0.0;
                        e[s] = v;
                        if (s == ss) last = v;
                    }
                    if (tp < p.T) {
                        const double nxt = (tot > 0.0) ? (ss <= S ? last : 1.0) : 0.0;
                        p.enf[((size_t)c * p.T + tp) * (S + 1)] = nxt;
                    }
                }
            }
        }
    }
    __syncthreads();
    // 5. the CTA's islands: new weight and inherited block
    const int ss = iscal[1];
    const double tot = scal[0];
    const int lvl = ss - 1;
    for (int g = tid; g < p.G; g += nthr) {
        const int k = k0 + g;
        if (dead) {
            own_wr[g] = 0.0;
            own_we[g] = 0;
        } else {
            const double bsum = tree[tree_off(m, lvl) + (k >> lvl)];
            const XW w = xw_from(bsum * (double)m / (tot * ldexp(1.0, lvl)), 0);
            own_wr[g] = w.r;
            own_we[g] = w.e;
        }
        int j = k;
        for (int s = lvl; s >= 1; --s) {
            const int l = s - 1, b = 1 << l, pi = j >> l;
            const double lo = tree[tree_off(m, l) + (pi & ~1)];
            const double hi = tree[tree_off(m, l) + (pi | 1)];
            const double u = unif_f64(st.draw((uint32_t)j, (uint32_t)tp, KIND_ISLAND, (uint32_t)s).x);
            j = (u * (lo + hi) < lo) ? (j & ~b) : (j | b);
        }
        own_src[g] = j;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Cascade of step tp in the FP32-mixed path: the same steps as cascade(), with
// the island weights turned into 64-bit fixed-point leaves relative to the
// largest island (50 fractional bits for the largest weight), so that the block
// sums are exact integers, identical in every CTA and cheap; the ENF test uses
// float, the island choice u (W_lo + W_hi) < W_lo is decided exactly in 128-bit
// integers, and log Z and the normalisation use the exact total in double.
// ---------------------------------------------------------------------------
__device__ void cascade_fx(const StepParams& p, int c, int tp, int k0, const Stream& st, double* tree_d,
                           double* scal, double* own_wr, int* own_we, int* own_src, bool designated)
{
    using u64 = unsigned long long;
    const int m = p.m, S = p.S, tid = threadIdx.x, nthr = blockDim.x;
    const double* wr = p.wr[tp & 1] + (size_t)c * m;
    const int* we = p.we[tp & 1] + (size_t)c * m;
    u64* tree = reinterpret_cast<u64*>(tree_d);
    float* Q = reinterpret_cast<float*>(tree_d + 2 * m);          // [kMaxStages]
    int* iscal = reinterpret_cast<int*>(tree_d + 2 * m + kMaxStages);

    int emax = INT_MIN;
    for (int k = tid; k < m; k += nthr) {
        if (wr[k] > 0.0 && we[k] > emax) emax = we[k];
    }
    emax = warp_max(emax);
    if (tid == 0) iscal[0] = INT_MIN;
    __syncthreads();
    if ((tid & 31) == 0) atomicMax(&iscal[0], emax);
    __syncthreads();
    emax = iscal[0];
    const bool dead = (emax == INT_MIN);

    // leaves: r in [0.5,1) has a 53-bit significand; shift it to the common scale
    for (int k = tid; k < m; k += nthr) {
        const double r = wr[k];
        u64 leaf = 0;
        if (!dead && r > 0.0) {
            const int sh = emax - we[k] + 3;
            const u64 mant = ((u64)__double_as_longlong(r) & ((1ull << 52) - 1)) | (1ull << 52);
            leaf = (sh < 64) ? (mant >> sh) : 0ull;
        }
        tree[k] = leaf;
    }
    __syncthreads();
    for (int l = 1; l <= S; ++l) {
        const int n = m >> l;
        u64* dst = tree + tree_off(m, l);
        const u64* src = tree + tree_off(m, l - 1);
        for (int b = tid; b < n; b += nthr) dst[b] = src[2 * b] + src[2 * b + 1];
        __syncthreads();
    }
    {
        const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
        for (int l = warp; l < S; l += nw) {
            const int n = m >> l;
            const u64* v = tree + tree_off(m, l);
            float acc = 0.0f;
            for (int b = lane; b < n; b += 32) {
                const float x = __ull2float_rn(v[b]) * 0x1p-62f;
                acc = fmaf(x, x, acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) Q[l] = acc;
        }
    }
    __syncthreads();
    if (tid < 32) {
        const u64 tot = tree[tree_off(m, S)];
        const float totf = __ull2float_rn(tot) * 0x1p-62f;
        bool quiet = false;
        if (tid < S) {
            const int s = tid + 1;
            quiet = (tot > 0) && !(totf * totf * ldexpf(1.0f, s - 1) < (float)p.tau * (float)m * Q[s - 1]);
        }
        const unsigned qm = __ballot_sync(0xffffffffu, quiet);
        if (tid == 0) {
            int ss;
            if (p.mode == 0) ss = 1;
            else if (p.mode == 1) ss = S + 1;
            else ss = qm ? __ffs(qm) : S + 1;
            iscal[1] = ss;
            scal[0] = (double)tot;
            if (designated) {
                // sum_k W'_k = tot 2^(emax - 50)
                const double L = (tot > 0) ? log((double)tot) - log((double)m) + (double)(emax - 50) * 0.6931471805599453
                                           : -INFINITY;
                const double lz = p.logz[c] + L;
                p.logz[c] = lz;
                if (p.trace) p.trace[(size_t)c * p.T + (tp - 1)] = lz;
                if (p.sstar) p.sstar[(size_t)c * p.T + (tp - 1)] = ss;
                if (p.enf) {
                    double* e = p.enf + ((size_t)c * p.T + (tp - 1)) * (S + 1);
                    double last = 1.0;
                    for (int s = 1; s <= S; ++s) {
                        const int sr = s <= ss ? s : ss;
                        const double v = (tot > 0) ? (double)totf * totf * ldexp(1.0, sr - 1) / ((double)m * Q[sr - 1]) : 0.0;
                        e[s] = v;
                        if (s == ss) last = v;
                    }
                    if (tp < p.T) p.enf[((size_t)c * p.T + tp) * (S + 1)] = (tot > 0) ? (ss <= S ? last : 1.0) : 0.0;
                }
            }
        }
    }
    __syncthreads();
    const int ss = iscal[1];
    const double totd = scal[0];
    const int lvl = ss - 1;
    for (int g = tid; g < p.G; g += nthr) {
        const int k = k0 + g;
        if (dead) {
            own_wr[g] = 0.0;
            own_we[g] = 0;
        } else {
            const double bsum = (double)tree[tree_off(m, lvl) + (k >> lvl)];
            const XW w = xw_from_bits(bsum * (double)m / (totd * ldexp(1.0, lvl)), 0);
            own_wr[g] = w.r;
            own_we[g] = w.e;
        }
        int j = k;
        for (int s = lvl; s >= 1; --s) {
            const int l = s - 1, b = 1 << l, pi = j >> l;
            const u64 lo = tree[tree_off(m, l) + (pi & ~1)];
            const u64 hi = tree[tree_off(m, l) + (pi | 1)];
            const u64 w2 = 2ull * (u64)st.draw((uint32_t)j, (uint32_t)tp, KIND_ISLAND, (uint32_t)s).x + 1ull;
            // (2w+1)(lo+hi) < 2^33 lo, in 128 bits
            const u64 sum = lo + hi;
            const u64 p_lo = w2 * sum, p_hi = __umul64hi(w2, sum);
            const u64 r_lo = lo << 33, r_hi = lo >> 31;
            const bool pick_lo = (p_hi < r_hi) || (p_hi == r_hi && p_lo < r_lo);
            j = pick_lo ? (j & ~b) : (j | b);
        }
        own_src[g] = j;
    }
    __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------
template <typename R, int MODEL, int DX>
__global__ void __launch_bounds__(kMaxThreads) airpf_step_kernel(StepParams p, int t)
{
    using Cdf = typename CdfType<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int cpf = p.m / p.G;                 // CTAs per filter
    const int c = blockIdx.x / cpf;
    const int k0 = (blockIdx.x - c * cpf) * p.G;
    if (p.active != nullptr && p.active[c] == 0) return;   // uniform over the CTA
    const int tid = threadIdx.x;
    const int N = p.N, M = p.M, dx = p.dx;
    const Layout L = make_layout(p);
    double* tree = reinterpret_cast<double*>(smem + L.tree);
    double* own_wr = reinterpret_cast<double*>(smem + L.small);
    int* own_we = reinterpret_cast<int*>(smem + L.small + align16(sizeof(double) * p.G));
    int* own_src = own_we + p.G;
    double* scal = reinterpret_cast<double*>(smem + L.small + align16(sizeof(double) * p.G)
                                             + align16(2 * sizeof(int) * p.G));
    R* mshared = reinterpret_cast<R*>(reinterpret_cast<unsigned char*>(scal) + align16(sizeof(double) * 16));
    const RunParams run = *p.run;
    const Stream st{p.seed_lo, p.seed_hi, run.iter, (run.chain0 + (uint32_t)c) << 8};
    const bool designated = (k0 == 0);

    // ---- cascade of step t-1 ----
    if (t == 1) {
        for (int g = tid; g < p.G; g += blockDim.x) {
            own_wr[g] = 0.5;          // W = 1 = 0.5 * 2^1
            own_we[g] = 1;
            own_src[g] = k0 + g;
        }
        if (designated && tid == 0) {
            p.logz[c] = 0.0;
            if (p.enf) p.enf[(size_t)c * p.T * (p.S + 1)] = 1.0;
        }
        __syncthreads();
    } else {
        if constexpr (sizeof(R) == 8) cascade(p, c, t - 1, k0, st, tree, scal, own_wr, own_we, own_src, designated);
        else cascade_fx(p, c, t - 1, k0, st, tree, scal, own_wr, own_we, own_src, designated);
    }

    // ---- lineage of step t-1: parent of particle (k, i) among time-(t-1) particles ----
    if (p.anc != nullptr && t >= 2) {
        const int* ires = p.ires[(t - 1) & 1] + (size_t)c * N;
        int* anc = p.anc + ((size_t)c * p.T + (t - 2)) * N;
        for (int q = tid; q < p.G * M; q += blockDim.x) {
            const int g = q / M, i = q - g * M;
            const int par = own_src[g];
            anc[(k0 + g) * M + i] = par * M + ires[par * M + i];
        }
    }
    if (t == p.T + 1) return;

    // ---- island work of step t ----
    Cdf* cdf_all = reinterpret_cast<Cdf*>(smem + L.island + L.cdf);
    R* xs_all = reinterpret_cast<R*>(smem + L.island + L.xs);
    double* red_all = reinterpret_cast<double*>(smem + L.island + L.red);
    double* mxr_all = reinterpret_cast<double*>(smem + L.island + L.mxr);
    const int nwi = (p.tpi + 31) >> 5;

    ModelPar<R>* mps = reinterpret_cast<ModelPar<R>*>(
        reinterpret_cast<unsigned char*>(mshared) + align16(sizeof(R) * (size_t)(dx * dx + p.dy * dx + kMaxDy)));
    if (tid == 0) {
        model_setup<R, MODEL>(*mps, p.theta + (size_t)c * p.theta_dim, dx, p.dy);
        model_step_setup<R, MODEL>(*mps, t);
    }
    R* Am = mshared;
    R* Cm = mshared + dx * dx;
    R* yv = Cm + p.dy * dx;
    if (MODEL == LGSSM) {
        for (int q = tid; q < dx * dx + p.dy * dx; q += blockDim.x) mshared[q] = (R)p.mdata[q];
    }
    for (int q = tid; q < p.dy; q += blockDim.x) yv[q] = (R)p.y[(size_t)(t - 1) * p.dy + q];
    __syncthreads();     // also orders the cascade's smem reads before the island work reuses it
    const ModelPar<R> mp = *mps;

    const int g = tid / p.tpi, li = tid - g * p.tpi;
    const int lane = tid & 31, wi = li >> 5;   // warp index within the island
    const int k = k0 + g;
    const int par = own_src[g];
    Cdf* cdf = cdf_all + (size_t)g * M;
    R* xs = reinterpret_cast<R*>(reinterpret_cast<unsigned char*>(xs_all) + L.xs_stride * g);
    double* red = red_all + (size_t)g * nwi;
    double* mxr = mxr_all + (size_t)g * nwi;
    const R* Xp = reinterpret_cast<const R*>(p.X[(t - 1) & 1]);
    R* Xc = reinterpret_cast<R*>(p.X[t & 1]);

    R xv[kPptMax][DX];
    R lv[kPptMax];
    uint32_t wres[kPptMax];
#pragma unroll
    for (int r = 0; r < kPptMax; ++r) {
        lv[r] = (R)(-INFINITY);
        wres[r] = 0;
        const int i = li * p.ppt + r;
        if (r < p.ppt && i < M) {
            const uint32_t unit = (uint32_t)(k * M + i);
            R xp[DX];
            if (t == 1) {
                model_prior<R, MODEL, DX>(mp, st, unit, dx, xp);
            } else {
#pragma unroll
                for (int d = 0; d < DX; ++d)
                    if (d < dx) xp[d] = Xp[((size_t)c * dx + d) * N + (size_t)par * M + i];
            }
            wres[r] = model_step<R, MODEL, DX>(mp, st, unit, (uint32_t)t, dx, xp, xv[r], Am);
            lv[r] = model_logg<R, MODEL, DX>(mp, yv, dx, p.dy, xv[r], Cm);
        }
    }

    // island maximum of the log-weights
    R mx = lv[0];
#pragma unroll
    for (int r = 1; r < kPptMax; ++r) mx = (lv[r] > mx) ? lv[r] : mx;
    mx = warp_max(mx);
    if (nwi > 1) {
        if (lane == 0) mxr[wi] = (double)mx;
        __syncthreads();
        double v = mxr[0];
        for (int w = 1; w < nwi; ++w) v = (mxr[w] > v) ? mxr[w] : v;
        mx = (R)v;
    }
    const bool alive = (mx > (R)(-INFINITY));

    // weights and the thread-local inclusive prefix
    Cdf part[kPptMax];
    Cdf run_sum = 0;
#pragma unroll
    for (int r = 0; r < kPptMax; ++r) {
        Cdf w = 0;
        if (alive && r < p.ppt && lv[r] > (R)(-INFINITY)) {
            if constexpr (sizeof(R) == 8) {
                w = exp(lv[r] - mx);
            } else {
                w = (Cdf)__float2ull_rn(__expf(lv[r] - mx) * 2147483648.0f);
            }
        }
        run_sum += w;
        part[r] = run_sum;
    }
    // island-wide exclusive offset of this thread
    Cdf incl = warp_incl_scan(run_sum, lane);
    Cdf excl = incl - run_sum;
    if (nwi > 1) {
        if (lane == 31) {
            if constexpr (sizeof(R) == 8) red[wi] = (double)incl;
            else reinterpret_cast<Cdf*>(red)[wi] = incl;
        }
        __syncthreads();
        Cdf off = 0;
        for (int w = 0; w < wi; ++w) {
            if constexpr (sizeof(R) == 8) off += red[w];
            else off += reinterpret_cast<Cdf*>(red)[w];
        }
        excl += off;
    }
#pragma unroll
    for (int r = 0; r < kPptMax; ++r) {
        const int i = li * p.ppt + r;
        if (r < p.ppt && i < M) {
            cdf[i] = excl + part[r];
#pragma unroll
            for (int d = 0; d < DX; ++d)
                if (d < dx) xs[(size_t)d * M + i] = xv[r][d];
        }
    }
    __syncthreads();
    const Cdf total = cdf[M - 1];

    // multinomial draws: ancestor of draw j = first i with C_i > u_j C_{M-1}.
    // Fixed-depth branchless lower bound, the thread's draws advanced together.
    int* ires_out = (p.ires[t & 1] != nullptr) ? p.ires[t & 1] + (size_t)c * N + (size_t)k * M : nullptr;
    Cdf target[kPptMax];
    int base[kPptMax];
#pragma unroll
    for (int r = 0; r < kPptMax; ++r) {
        base[r] = 0;
        if constexpr (sizeof(R) == 8) {
            target[r] = unif_f64(wres[r]) * total;
        } else {
            const unsigned long long hi = total >> 32;
            const uint32_t lo = (uint32_t)(total & 0xffffffffull);
            target[r] = (unsigned long long)wres[r] * hi + (unsigned long long)__umulhi(wres[r], lo);
        }
    }
    for (int n = M; n > 1;) {
        const int half = n >> 1;
#pragma unroll
        for (int r = 0; r < kPptMax; ++r) {
            const Cdf v = cdf[base[r] + half - 1];
            base[r] = (v > target[r]) ? base[r] : base[r] + half;
        }
        n -= half;
    }
#pragma unroll
    for (int r = 0; r < kPptMax; ++r) {
        const int j = li * p.ppt + r;
        if (r < p.ppt && j < M) {
            const int a = alive ? base[r] : j;
#pragma unroll
            for (int d = 0; d < DX; ++d)
                if (d < dx) Xc[((size_t)c * dx + d) * N + (size_t)k * M + j] = xs[(size_t)d * M + a];
            if (ires_out) ires_out[j] = a;
        }
    }

    // island weight W^k_{t,1} = W^k_{t,0} exp(max) (sum_i w_i) / M, extended range
    if (li == 0) {
        XW w{0.0, 0};
        const double wr0 = own_wr[g];
        if (alive && wr0 > 0.0) {
            if constexpr (sizeof(R) == 8) {
                double mxd = fmin(fmax((double)mx, -1.0e7), 1.0e7);
                const double n = floor(mxd * 1.4426950408889634);
                // two-constant reduction of mxd - n ln 2 (Cody and Waite, 1980)
                double f = fma(-n, 0.6931471805599453, mxd);
                f = fma(-n, 2.3190468138462996e-17, f);
                w = xw_from_bits(exp(f) * ((double)total / (double)M) * wr0, own_we[g] + (int)n);
            } else {
                // float log-weights: exp of the reduced argument in float, the
                // product and the exponent bookkeeping in double / integers
                const float mxf = fminf(fmaxf((float)mx, -1.0e7f), 1.0e7f);
                const float n = floorf(mxf * 1.44269504f);
                float f = fmaf(-n, 0.693145752f, mxf);
                f = fmaf(-n, 1.42860677e-06f, f);
                const double ef = (double)__expf(f);
                w = xw_from_bits(ef * ((double)total * (0x1p-31 / (double)M)) * wr0, own_we[g] + (int)n);
            }
        }
        p.wr[t & 1][(size_t)c * p.m + k] = w.r;
        p.we[t & 1][(size_t)c * p.m + k] = w.e;
    }
}

__global__ void set_run_kernel(RunParams* r, uint32_t iter, uint32_t chain0)
{
    r->iter = iter;
    r->chain0 = chain0;
}

// ---------------------------------------------------------------------------
size_t step_smem_bytes(const StepParams& p) { return make_layout(p).total; }

void choose_mapping(int m, int M, int fp64, int want_ppt, int want_g, int* tpi, int* ppt, int* G)
{
    (void)fp64;
    // particles per thread: requested (1, 2 or 4) or 4; threads per island a
    // multiple of 32 covering M; islands per CTA up to 256 threads (or requested)
    int pp = (want_ppt == 1 || want_ppt == 2 || want_ppt == 4) ? want_ppt : kPptMax;
    int t = 32;
    while (t * pp < M && t < kMaxThreads) t *= 2;
    if (t * pp < M) pp = (M + t - 1) / t;
    *tpi = t;
    *ppt = (M + t - 1) / t;
    int g = kMaxThreads / t;
    if (want_g > 0 && want_g < g) g = want_g;
    while (g > 1 && (g & (g - 1))) --g;      // a power of 2 dividing m
    if (g > m) g = m;
    *G = g < 1 ? 1 : g;
}

template <typename R, int MODEL, int DX>
static cudaError_t launch_typed(const StepParams& p, int t, cudaStream_t stream, bool prepare_only)
{
    const size_t smem = step_smem_bytes(p);
    auto fn = airpf_step_kernel<R, MODEL, DX>;
    if (prepare_only) {
        // opt in to more than 48 KB of dynamic shared memory (outside any capture)
        const int want = smem > 48 * 1024 ? (int)smem : 48 * 1024;
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    }
    const int grid = p.B * (p.m / p.G);
    fn<<<grid, p.G * p.tpi, smem, stream>>>(p, t);
    return cudaGetLastError();
}

static cudaError_t dispatch(const StepParams& p, int t, cudaStream_t stream, bool prep)
{
    if (p.fp64) {
        switch (p.model) {
        case AR1: return launch_typed<double, AR1, 1>(p, t, stream, prep);
        case SV: return launch_typed<double, SV, 1>(p, t, stream, prep);
        case NGM: return launch_typed<double, NGM, 1>(p, t, stream, prep);
        case TOY: return launch_typed<double, TOY, 1>(p, t, stream, prep);
        case LGSSM: return launch_typed<double, LGSSM, kMaxDx>(p, t, stream, prep);
        }
    } else {
        switch (p.model) {
        case AR1: return launch_typed<float, AR1, 1>(p, t, stream, prep);
        case SV: return launch_typed<float, SV, 1>(p, t, stream, prep);
        case NGM: return launch_typed<float, NGM, 1>(p, t, stream, prep);
        case TOY: return launch_typed<float, TOY, 1>(p, t, stream, prep);
        case LGSSM: return launch_typed<float, LGSSM, kMaxDx>(p, t, stream, prep);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t prepare_step(const StepParams& p) { return dispatch(p, 0, nullptr, true); }

cudaError_t launch_step(const StepParams& p, int t, cudaStream_t stream) { return dispatch(p, t, stream, false); }

cudaError_t launch_set_run(RunParams* d_run, uint32_t iter, uint32_t chain0, cudaStream_t stream)
{
    set_run_kernel<<<1, 1, 0, stream>>>(d_run, iter, chain0);
    return cudaGetLastError();
}

}  // namespace airpf
