// airpf_step.cu -- the AIRPF time step on sm_103a.
//
// One launch per time step t (Algorithm 1 of Heine, arXiv 2312.06484, main
// loop), captured in a CUDA graph by the runtime after one prologue launch
// that derives the model constants of every filter.  Each CTA owns G islands
// of one filter.  Launch t does, in order:
//
//  1. the interaction cascade of step t-1 (Algorithm 1, stages s = 1..S),
//     recomputed by every CTA of the filter from the m island weights of step
//     t-1 so that no second launch or grid-wide barrier is needed:
//       - island weights W^k_{t-1,1}, kept unnormalised as in Algorithm 1 in an
//         extended range (double mantissa, integer binary exponent), are
//         rescaled by the largest exponent and summed in a binary tree in
//         shared memory; level l holds the sums over aligned blocks of 2^l
//         islands.  The lower five levels are built with warp shuffles;
//       - after s-1 interacting butterfly stages (eq. (3)) every island weight
//         is the mean of its aligned block of 2^(s-1) islands, so
//         ENF_{t,s} = Tot^2 2^(s-1) / (m sum_b B_{s-1,b}^2) for every stage
//         from the one tree; the interacting stages form a prefix (a stage
//         with alpha = I leaves the weights, hence the ENF, unchanged), so
//         s* = min{s : ENF_s >= tau} (adaptation line of Algorithm 1);
//       - island k's new weight W^k_{t,0} is its block mean at level s*-1, and
//         the block it inherits is src(k) = c_1(c_2(...c_{s*-1}(k))) where
//         c_s(j) picks the lower island of {j, j xor 2^(s-1)} iff
//         u_{t,s,j} (W_lo + W_hi) < W_lo;
//       - log Z^N_{t-1} = log(m^-1 sum_k W^k) (Section 2) is read off the
//         tree total when it is recorded.
//     FP64 path: leaves, sums and sums of squares in double (decisions agree
//     with an FP64 reference to rounding).  FP32-mixed path: leaves are
//     64-bit fixed point relative to the largest island, so block sums are
//     exact integers; the ENF test uses float; the island choice is decided
//     exactly in 128-bit integers.
//  2. the island work of step t for the CTA's islands: mutate the inherited
//     internally-resampled block of island src(k) through K_t (Algorithm 1,
//     last stage), weight by g_t, reduce the island maximum, build the
//     inclusive CDF (FP64, or an exact 2^-31 fixed-point integer prefix sum in
//     FP32 mode), draw M multinomial ancestors by binary search (internal
//     resample), gather, store, and publish W^k_{t,1} = W^k_{t,0} M^-1 sum g.
//
// Launch T+1 runs the final cascade only (it yields log Z and the lineage of
// step T).
#include <climits>
#include <cstdio>

#include "airpf_device.cuh"
#include "airpf_internal.h"

namespace airpf {

namespace {

constexpr int kMaxThreads = 256;      // per-step and grid-persistent CTAs
constexpr int kMaxCtaThreads = 512;   // a whole filter in one CTA
constexpr unsigned long long kWaitNs = 1000000000ull;   // bounded barrier wait: 1 s
constexpr unsigned kSpinLimit = 1u << 26;               // iteration backstop
constexpr int kPptMax = 4;
constexpr int kMaxStages = 16;
constexpr int kShuffleLevels = 5;
using u64 = unsigned long long;

template <typename R> struct CdfType;
template <> struct CdfType<double> { using T = double; };
template <> struct CdfType<float> { using T = u64; };

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// offset (in nodes) of tree level l for m leaves: levels 0..S stored back to back
__device__ __forceinline__ int tree_off(int m, int l) { return 2 * m - 2 * (m >> l); }

struct Layout {
    size_t tree, island, small, total;   // byte offsets
    size_t cdf, xs, red, mxr;            // island sub-offsets
    size_t cdf_stride, xs_stride, red_stride;
};

// tree region: 2m nodes, then per-warp partial sums of squares (8 warps x 8
// levels), the per-level sums (kMaxStages) and a few integers
constexpr int kQwSlots = 128;   // up to 16 warps x 8 levels

__host__ __device__ inline Layout make_layout(const StepParams& p)
{
    Layout L;
    const size_t rsz = p.fp64 ? 8 : 4;
    const size_t nwi = (size_t)((p.tpi + 31) / 32);           // warps per island
    const size_t treeb = align16(sizeof(double) * (2 * (size_t)p.m + kQwSlots + kMaxStages + 8));
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
                          + align16(rsz * (size_t)(p.dx * p.dx + p.dy * p.dx + kMaxDy));
    L.total = L.small + smallb;
    return L;
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
__device__ __forceinline__ V warp_sum(V v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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

// Island weight: double r in [0.5,1) (or 0) times 2^e.
struct XW {
    double r;
    int e;
};

// v = r 2^e with r in [0.5, 1), by exponent-field manipulation for normal v;
// frexp for subnormal v.
__device__ __forceinline__ XW xw_from_bits(double v, int e_add)
{
    XW w;
    const long long b = __double_as_longlong(v);
    if (b <= 0 || b >= (0x7ffLL << 52)) {       // zero, negative, inf or NaN
        w.r = 0.0;
        w.e = 0;
        return w;
    }
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

// Arithmetic of the cascade for each precision (see file comment).
template <bool FX> struct Casc;
template <> struct Casc<false> {
    using V = double;
    using Qt = double;
    static constexpr int kFrac = 0;           // leaf = W 2^-emax
    __device__ static V leaf(double r, int de) { return ldexp(r, de); }
    __device__ static Qt qv(V v) { return v; }
    __device__ static double to_d(V v) { return v; }
    __device__ static bool pick_lo(V lo, V hi, uint32_t w) { return unif_f64(w) * (lo + hi) < lo; }
};
template <> struct Casc<true> {
    using V = u64;
    using Qt = float;
    static constexpr int kFrac = 50;          // leaf = W 2^(50-emax), largest leaf < 2^50
    __device__ static V leaf(double r, int de)
    {
        const int sh = 3 - de;
        const u64 mant = ((u64)__double_as_longlong(r) & ((1ull << 52) - 1)) | (1ull << 52);
        return sh < 64 ? (mant >> sh) : 0ull;
    }
    __device__ static Qt qv(V v) { return __ull2float_rn(v) * 0x1p-62f; }
    __device__ static double to_d(V v) { return (double)v; }
    // u (lo + hi) < lo with u = (2w+1) 2^-33, exactly: (2w+1)(lo+hi) < 2^33 lo in 128 bits
    __device__ static bool pick_lo(V lo, V hi, uint32_t w)
    {
        const u64 w2 = 2ull * (u64)w + 1ull;
        const u64 sum = lo + hi;
        const u64 p_lo = w2 * sum, p_hi = __umul64hi(w2, sum);
        const u64 r_lo = lo << 33, r_hi = lo >> 31;
        return (p_hi < r_hi) || (p_hi == r_hi && p_lo < r_lo);
    }
};

// ---------------------------------------------------------------------------
// Cascade of step tp for filter c (see file comment).  Every thread of the CTA
// calls it; four block barriers.  Outputs in shared memory: own_wr/own_we/
// own_src for the CTA's islands; records written by the filter's designated CTA.
// ---------------------------------------------------------------------------
template <bool FX>
__device__ void cascade(const StepParams& p, int c, int tp, int k0, const Stream& st, double* raw,
                        double* own_wr, int* own_we, int* own_src, bool designated)
{
    using C = Casc<FX>;
    using V = typename C::V;
    using Qt = typename C::Qt;
    const int m = p.m, S = p.S, tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const double* wr = p.wr[tp & 1] + (size_t)c * m;
    const int* we = p.we[tp & 1] + (size_t)c * m;
    V* tree = reinterpret_cast<V*>(raw);
    Qt* Qw = reinterpret_cast<Qt*>(raw + 2 * m);                 // [nw][8]
    Qt* Q = reinterpret_cast<Qt*>(raw + 2 * m + kQwSlots);       // [kMaxStages]
    int* iscal = reinterpret_cast<int*>(raw + 2 * m + kQwSlots + kMaxStages);

    // 1. largest binary exponent among nonzero weights (positive bit patterns)
    int emax = INT_MIN;
    for (int k = tid; k < m; k += nthr) {
        const int e = __ldcg(&we[k]);
        if (__double_as_longlong(__ldcg(&wr[k])) > 0 && e > emax) emax = e;
    }
    emax = warp_max(emax);
    if (tid == 0) iscal[0] = INT_MIN;
    __syncthreads();
    if (lane == 0) atomicMax(&iscal[0], emax);
    __syncthreads();
    emax = iscal[0];
    const bool dead = (emax == INT_MIN);

    // 2. leaves and the lower tree levels, 32 leaves per warp pass; each lane
    //    holding a node adds its square to that level's partial sum
    const int L5 = S < kShuffleLevels ? S : kShuffleLevels;
    Qt qa[kShuffleLevels + 1];
#pragma unroll
    for (int l = 0; l <= kShuffleLevels; ++l) qa[l] = (Qt)0;
    for (int ch = warp; ch * 32 < m; ch += nw) {
        const int k = ch * 32 + lane;
        V v = (V)0;
        if (k < m) {
            const double r = __ldcg(&wr[k]);
            if (!dead && __double_as_longlong(r) > 0) v = C::leaf(r, __ldcg(&we[k]) - emax);
            tree[k] = v;
            const Qt q = C::qv(v);
            qa[0] += q * q;
        }
#pragma unroll
        for (int l = 1; l <= kShuffleLevels; ++l) {
            if (l <= L5) {
                v += __shfl_down_sync(0xffffffffu, v, 1 << (l - 1));
                if ((lane & ((1 << l) - 1)) == 0 && (k >> l) < (m >> l)) {
                    tree[tree_off(m, l) + (k >> l)] = v;
                    const Qt q = C::qv(v);
                    qa[l] += q * q;
                }
            }
        }
    }
#pragma unroll
    for (int l = 0; l <= kShuffleLevels; ++l) {
        const Qt s = warp_sum(qa[l]);
        if (lane == 0) Qw[warp * 8 + l] = s;
    }
    __syncthreads();

    // 3. one warp: upper levels, per-level sums of squares, s*, records
    if (warp == 0) {
        if (lane <= L5) {
            Qt s = (Qt)0;
            for (int w = 0; w < nw; ++w) s += Qw[w * 8 + lane];
            Q[lane] = s;
        }
        for (int l = L5 + 1; l <= S; ++l) {
            __syncwarp();
            const int n = m >> l;
            Qt acc = (Qt)0;
            for (int b = lane; b < n; b += 32) {
                const V v = tree[tree_off(m, l - 1) + 2 * b] + tree[tree_off(m, l - 1) + 2 * b + 1];
                tree[tree_off(m, l) + b] = v;
                const Qt q = C::qv(v);
                acc += q * q;
            }
            acc = warp_sum(acc);
            if (lane == 0) Q[l] = acc;
        }
        __syncwarp();
        const V tot = tree[tree_off(m, S)];
        const Qt tq = C::qv(tot);
        bool quiet = false;
        if (lane < S) {
            const int s = lane + 1;
            // stage s interacts iff ENF_s < tau, i.e. Tot^2 2^(s-1) < tau m Q_{s-1}
            quiet = (tot > (V)0) && !(tq * tq * (Qt)(1u << (s - 1)) < (Qt)p.tau * (Qt)m * Q[s - 1]);
        }
        const unsigned qm = __ballot_sync(0xffffffffu, quiet);
        if (lane == 0) {
            int ss;
            if (p.mode == 0) ss = 1;
            else if (p.mode == 1) ss = S + 1;
            else ss = qm ? __ffs(qm) : S + 1;              // first quiet stage
            iscal[1] = ss;
            if (designated) {
                if (p.trace || tp == p.T) {
                    // log Z^N_tp = log(m^-1 sum_k W^k), sum_k W^k = Tot 2^(emax - kFrac)
                    const double lz = (tot > (V)0)
                        ? log(C::to_d(tot)) - log((double)m) + (double)(emax - C::kFrac) * 0.6931471805599453
                        : -INFINITY;
                    if (p.trace) p.trace[(size_t)c * p.T + (tp - 1)] = lz;
                    if (tp == p.T) p.logz[c] = lz;
                }
                if (p.sstar) p.sstar[(size_t)c * p.T + (tp - 1)] = ss;
                if (p.enf) {
                    double* e = p.enf + ((size_t)c * p.T + (tp - 1)) * (S + 1);
                    double last = 1.0;
                    for (int s = 1; s <= S; ++s) {
                        const int sr = s <= ss ? s : ss;
                        const double v = (tot > (V)0)
                            ? (double)tq * (double)tq * ldexp(1.0, sr - 1) / ((double)m * (double)Q[sr - 1]) : 0.0;
                        e[s] = v;
                        if (s == ss) last = v;
                    }
                    if (tp < p.T) p.enf[((size_t)c * p.T + tp) * (S + 1)] = (tot > (V)0) ? (ss <= S ? last : 1.0) : 0.0;
                }
            }
        }
    }
    __syncthreads();

    // 4. the CTA's islands: new weight (block mean, unnormalised) and inherited block
    const int ss = iscal[1];
    const int lvl = ss - 1;
    for (int g = tid; g < p.G; g += nthr) {
        const int k = k0 + g;
        XW w{0.0, 0};
        if (!dead) w = xw_from_bits(C::to_d(tree[tree_off(m, lvl) + (k >> lvl)]), emax - C::kFrac - lvl);
        own_wr[g] = w.r;
        own_we[g] = w.e;
        int j = k;
        for (int s = lvl; s >= 1; --s) {
            const int l = s - 1, b = 1 << l, pi = j >> l;
            const V lo = tree[tree_off(m, l) + (pi & ~1)];
            const V hi = tree[tree_off(m, l) + (pi | 1)];
            const uint32_t wu = st.draw((uint32_t)j, (uint32_t)tp, KIND_ISLAND, (uint32_t)s).x;
            j = C::pick_lo(lo, hi, wu) ? (j & ~b) : (j | b);
        }
        own_src[g] = j;
    }
    __syncthreads();
}

enum { OP_STEP = 0, OP_PREPARE = 1, OP_FITS = 2, OP_PERSIST_GRID = 3, OP_PERSIST_CTA = 4 };

}  // namespace

// ---------------------------------------------------------------------------
// Prologue: model constants of every filter (and the NGM drift table), once
// per pass.
// ---------------------------------------------------------------------------
template <typename R, int MODEL>
__global__ void airpf_prologue_kernel(StepParams p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && p.bar != nullptr) {
        p.bar[0] = 0u;
        p.bar[1] = 0u;
        *p.err = 0u;
    }
    if (i < p.B && (p.active == nullptr || p.active[i] != 0)) {
        ModelPar<R> mp;
        model_setup<R, MODEL>(mp, p.theta + (size_t)i * p.theta_dim, p.dx, p.dy);
        reinterpret_cast<ModelPar<R>*>(p.mpar)[i] = mp;
    }
    if (MODEL == NGM && i < p.T) reinterpret_cast<R*>(p.drift)[i] = (R)(8.0 * cos(1.2 * (double)(i + 1)));
}

// ---------------------------------------------------------------------------
// Step t for the G islands k0.. of filter c (see file comment).  Called by every
// thread of the CTA; all barriers inside are CTA-uniform.
template <typename R, int MODEL, int DX>
__device__ __forceinline__ void step_body(const StepParams& p, int t, int c, int k0, unsigned char* smem)
{
    using Cdf = typename CdfType<R>::T;
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
        if (designated && tid == 0 && p.enf) p.enf[(size_t)c * p.T * (p.S + 1)] = 1.0;
        __syncthreads();
    } else {
        cascade<sizeof(R) == 4>(p, c, t - 1, k0, st, tree, own_wr, own_we, own_src, designated);
    }

    // ---- lineage of step t-1: parent of particle (k, i) among time-(t-1) particles ----
    if (p.anc != nullptr && t >= 2) {
        const int* ires = p.ires[(t - 1) & 1] + (size_t)c * N;
        int* anc = p.anc + ((size_t)c * p.T + (t - 2)) * N;
        for (int q = tid; q < p.G * M; q += blockDim.x) {
            const int g = q / M, i = q - g * M;
            const int par = own_src[g];
            anc[(k0 + g) * M + i] = par * M + __ldcg(&ires[par * M + i]);
        }
    }
    if (t == p.T + 1) return;

    // ---- island work of step t ----
    Cdf* cdf_all = reinterpret_cast<Cdf*>(smem + L.island + L.cdf);
    R* xs_all = reinterpret_cast<R*>(smem + L.island + L.xs);
    double* red_all = reinterpret_cast<double*>(smem + L.island + L.red);
    double* mxr_all = reinterpret_cast<double*>(smem + L.island + L.mxr);
    const int nwi = (p.tpi + 31) >> 5;

    R* Am = mshared;
    R* Cm = mshared + dx * dx;
    R* yv = Cm + p.dy * dx;
    if (MODEL == LGSSM) {
        for (int q = tid; q < dx * dx + p.dy * dx; q += blockDim.x) mshared[q] = (R)p.mdata[q];
    }
    for (int q = tid; q < p.dy; q += blockDim.x) yv[q] = (R)p.y[(size_t)(t - 1) * p.dy + q];
    ModelPar<R> mp = reinterpret_cast<const ModelPar<R>*>(p.mpar)[c];
    if (MODEL == NGM) mp.drift = reinterpret_cast<const R*>(p.drift)[t - 1];
    __syncthreads();     // also orders the cascade's smem reads before the island work reuses it

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
                    if (d < dx) xp[d] = __ldcg(&Xp[((size_t)c * dx + d) * N + (size_t)par * M + i]);
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
            const u64 hi = total >> 32;
            const uint32_t lo = (uint32_t)(total & 0xffffffffull);
            target[r] = (u64)wres[r] * hi + (u64)__umulhi(wres[r], lo);
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
                w = xw_from_bits(exp(f) * ((double)total * p.inv_M) * wr0, own_we[g] + (int)n);
            } else {
                // float log-weights: exp of the reduced argument in float, the
                // product in double, the exponent bookkeeping in integers
                const float mxf = fminf(fmaxf((float)mx, -1.0e7f), 1.0e7f);
                const float n = floorf(mxf * 1.44269504f);
                float f = fmaf(-n, 0.693145752f, mxf);
                f = fmaf(-n, 1.42860677e-06f, f);
                const double ef = (double)__expf(f);
                w = xw_from_bits(ef * ((double)total * p.inv_M) * wr0, own_we[g] + (int)n - 31);
            }
        }
        p.wr[t & 1][(size_t)c * p.m + k] = w.r;
        p.we[t & 1][(size_t)c * p.m + k] = w.e;
    }
}

// ---------------------------------------------------------------------------
// Grid barrier of the cooperative persistent kernel (generation counter).  The
// wait is bounded: after kSpinLimit sleeps the CTA sets the error word and every
// CTA leaves the time loop at its next barrier.  bar[0] counts arrivals, bar[1]
// is the generation; both and *err are zeroed by the prologue.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

__device__ bool grid_barrier(unsigned* bar, unsigned* err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g0 = ld_acquire_gpu(bar + 1);
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned it = 0;
            const unsigned long long t0 = global_ns();
            while (ld_acquire_gpu(bar + 1) == g0) {
                if (++it > kSpinLimit || global_ns() - t0 > kWaitNs) {
                    atomicExch(err, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        if (ld_acquire_gpu(err) != 0u) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename R, int MODEL, int DX>
__global__ void __launch_bounds__(kMaxThreads) airpf_step_kernel(StepParams p, int t)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int cpf = p.m / p.G;                 // CTAs per filter
    const int c = blockIdx.x / cpf;
    const int k0 = (blockIdx.x - c * cpf) * p.G;
    if (p.active != nullptr && p.active[c] == 0) return;   // uniform over the CTA
    step_body<R, MODEL, DX>(p, t, c, k0, smem);
}

// All T+1 steps in one launch.  GRID: the filter spans several co-resident CTAs
// (cooperative launch), steps separated by the grid barrier.  Otherwise one CTA
// holds a whole filter and __syncthreads separates the steps.
template <typename R, int MODEL, int DX, bool GRID>
__global__ void __launch_bounds__(GRID ? kMaxThreads : kMaxCtaThreads) airpf_persistent_kernel(StepParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int cpf = p.m / p.G;
    const int c = blockIdx.x / cpf;
    const int k0 = (blockIdx.x - c * cpf) * p.G;
    const bool act = (p.active == nullptr || p.active[c] != 0);
    if (!GRID && !act) return;
    // fault-injection hook: CTA 0 leaves before the first barrier, so the other
    // CTAs' bounded wait runs out (tests the timeout path)
    if (GRID && p.inject_stall && blockIdx.x == 0) return;
    for (int t = 1; t <= p.T + 1; ++t) {
        if (act) step_body<R, MODEL, DX>(p, t, c, k0, smem);
        if (t <= p.T) {
            if (GRID) {
                if (!grid_barrier(p.bar, p.err)) return;
            } else {
                __syncthreads();
            }
        }
    }
}

__global__ void set_run_kernel(RunParams* r, uint32_t iter, uint32_t chain0)
{
    r->iter = iter;
    r->chain0 = chain0;
}

// ---------------------------------------------------------------------------
size_t step_smem_bytes(const StepParams& p) { return make_layout(p).total; }

size_t model_par_bytes() { return sizeof(ModelPar<double>); }

void choose_mapping(int m, int M, int fp64, int want_ppt, int want_g, int* tpi, int* ppt, int* G)
{
    (void)fp64;
    // particles per thread: requested (1, 2 or 4) or 4; threads per island a
    // multiple of 32 covering M; islands per CTA up to 256 threads, or the
    // requested count (a whole filter, up to 512 threads, when want_g >= m)
    int pp = (want_ppt == 1 || want_ppt == 2 || want_ppt == 4) ? want_ppt : kPptMax;
    int t = 32;
    while (t * pp < M && t < kMaxThreads) t *= 2;
    if (t * pp < M) pp = (M + t - 1) / t;
    *tpi = t;
    *ppt = (M + t - 1) / t;
    int g = kMaxThreads / t;
    if (want_g >= m && m * t <= kMaxCtaThreads) g = m;
    else if (want_g > 0 && want_g < g) g = want_g;
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
    if (p.fp64) {
        switch (p.model) {
        case AR1: return launch_typed<double, AR1, 1>(p, t, stream, op, fits);
        case SV: return launch_typed<double, SV, 1>(p, t, stream, op, fits);
        case NGM: return launch_typed<double, NGM, 1>(p, t, stream, op, fits);
        case TOY: return launch_typed<double, TOY, 1>(p, t, stream, op, fits);
        case LGSSM: return launch_typed<double, LGSSM, kMaxDx>(p, t, stream, op, fits);
        }
    } else {
        switch (p.model) {
        case AR1: return launch_typed<float, AR1, 1>(p, t, stream, op, fits);
        case SV: return launch_typed<float, SV, 1>(p, t, stream, op, fits);
        case NGM: return launch_typed<float, NGM, 1>(p, t, stream, op, fits);
        case TOY: return launch_typed<float, TOY, 1>(p, t, stream, op, fits);
        case LGSSM: return launch_typed<float, LGSSM, kMaxDx>(p, t, stream, op, fits);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t prepare_step(const StepParams& p) { return dispatch(p, 0, nullptr, OP_PREPARE, nullptr); }

cudaError_t launch_step(const StepParams& p, int t, cudaStream_t stream)
{
    return dispatch(p, t, stream, OP_STEP, nullptr);
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

cudaError_t launch_set_run(RunParams* d_run, uint32_t iter, uint32_t chain0, cudaStream_t stream)
{
    set_run_kernel<<<1, 1, 0, stream>>>(d_run, iter, chain0);
    return cudaGetLastError();
}

}  // namespace airpf
