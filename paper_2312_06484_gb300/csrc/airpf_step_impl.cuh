// airpf_step_impl.cuh -- the AIRPF time step on sm_103a (kernel templates;
// instantiated per precision, model and particles per thread in
// airpf_launch_inst.cu).
//
// A pass of Algorithm 1 (Heine, arXiv 2312.06484, main loop) is a prologue
// launch that derives every filter's model constants, then, for t = 1..T, an
// island-step launch (every CTA of every filter) followed by a cascade launch
// (one CTA per filter), and a last island-step launch for t = T+1 that only
// records the lineage of step T -- replayed from a CUDA graph.  Where a filter
// fits one CTA, one persistent launch runs all steps instead (the CTA runs the
// cascade itself between block barriers); the cooperative-grid launch runs the
// cascade in the filter's first CTA between two bounded grid barriers.
// CTA j of a filter owns the G islands j*G .. j*G+G-1.
// The default launch form is fused steps: one island-step launch per step in
// which every CTA first runs the previous step's cascade itself from all m/G
// CTA records (the stage-1 test alone on most steps), then its islands; split
// steps (above 512 CTAs per filter) keep the separate one-CTA cascade kernel,
// which leaves the upper tree in global memory for the island CTAs.  With
// programmatic dependent launch each kernel draws its random numbers before it
// waits for the previous one.
//
// Variants on the same kernels: radix r = 2^b interactions (stages over groups of
// r islands) take the adaptive decision at the first binary stage of each group
// of b, where the r-ary stage's ENF lies in the same tree, and walk one r-way
// choice per island and stage (walk_src); adaptive internal
// resampling (recording instantiation) carries log(M omega) per particle and
// skips an island's resampling while its ESS is at least tau_int M.
//
// Island weights W^k are kept unnormalised, as in Algorithm 1, in an extended
// range (mantissa plus integer binary exponent).  At the end of step t each
// CTA publishes a record of its islands' weights: the largest binary exponent
// e_j and the binary tree of block sums over its G islands (levels 0..g,
// g = log2 G) relative to 2^e_j, with the per-level sums of squares.  Level l
// of the tree over all m islands holds the sums over aligned blocks of 2^l
// islands; levels below g are inside the records, levels g..S form the upper
// tree over the m/G record tops.
//
// Cascade kernel of step t (Algorithm 1, interaction stages s = 1..S): read
// each record once, rescale the record tops by exact powers of two to the
// largest exponent, build the upper tree by warp shuffles.  After s-1
// interacting butterfly stages (eq. (3)) every island weight is the mean of
// its aligned block of 2^(s-1) islands, so
//   ENF_{t,s} = Tot^2 2^(s-1) / (m sum_b B_{s-1,b}^2)
// for every stage from one tree; the interacting stages form a prefix (a stage
// with alpha = I leaves the weights, hence the ENF, unchanged), so
// s* = min{s : ENF_s >= tau} (adaptation line of Algorithm 1).  Island k's new
// weight W^k_{t+1,0} is its block mean at level s*-1 and the block it inherits
// is src(k) = c_1(c_2(...c_{s*-1}(k))), where c_s(j) picks the lower island of
// {j, j xor 2^(s-1)} iff u_{t,s,j} (W_lo + W_hi) < W_lo.  The kernel writes the
// summary (s*, largest exponent), the upper-tree level s*-1 when it lies above
// the CTA level, src(k) when s* > 1, and log Z^N_t = log(m^-1 sum_k W^k)
// (Section 2) from the tree total when it is recorded.
//
// Island-step kernel of step t+1, per CTA:
//  1. load the summary, the CTA's own record and (s* > 1) the inherited
//     blocks; issue the loads of the CTA's own particle block (the parents
//     when the island keeps its block) and draw the step's random numbers
//     (Philox, Box-Muller) while they are in flight;
//  2. mutate the inherited internally-resampled block through K_{t+1}
//     (Algorithm 1, last stage), weight by g_{t+1}, island maximum, inclusive
//     CDF, M multinomial draws by binary search (internal resample), gather,
//     store, and W^k_{t+1,1} = W^k_{t+1,0} M^-1 sum g;
//  3. publish the CTA's record.
//
// Arithmetic.  FP64 path: particles, CDF, island weights (double mantissa),
// block sums and sums of squares in double, so every decision agrees with an
// FP64 reference to rounding.  FP32-mixed path: particles and log-weights in
// float; the CDF is an exact 32-bit fixed-point prefix sum of the weights
// quantised to 2^-(31 - ceil(log2 M)) of the island maximum; island weights are
// 64-bit integer mantissas with an exponent, multiplied to 64 bits, and block
// sums are 64-bit fixed point (63 - log2 m fractional bits below the largest
// weight, so a sum over all m islands stays below 2^63);
// the ENF test uses float; the island choice is decided exactly in 128-bit
// integers; log Z is formed in double.  The common factor 1/M of the island
// weights is left out of the FP32-mixed weights and restored in log Z.  The
// FP32-mixed path issues no FP64-pipe instruction per particle or island.
#pragma once
#include <climits>
#include <cstdio>

#include "airpf_device.cuh"
#include "airpf_internal.h"

namespace airpf {

namespace {

constexpr int kMaxThreads = 512;      // per-step and grid-persistent CTAs
constexpr int kMaxCtaThreads = 512;   // a whole filter in one CTA
constexpr int kMinCtasPerSm = 2;      // register budget: 64 per thread at 512 threads
constexpr int kCascadeThreads = 1024; // the cascade kernel's CTA (split steps: one per filter)
constexpr int kMaxWarps = 32;         // per-warp partial slots of the cascade
constexpr int kDefaultThreads = 256;  // default CTA size of the per-step launch (measured best, fused steps)
constexpr unsigned long long kWaitNs = 1000000000ull;   // bounded barrier wait: 1 s
constexpr unsigned kSpinLimit = 1u << 26;               // iteration backstop
constexpr int kMaxStages = 16;
constexpr int kShuffleLevels = 5;
constexpr int kCachedChunks = 2;      // record chunks a lane keeps in registers
constexpr int kQw = 16;               // per-warp partial slots (one per tree level)
constexpr int kGroupLog = kTailGroupLog;   // split steps: CTA records per group of the tail cascade
constexpr int kGroupQ = 16;           // a group record's sums of squares (levels 0 .. g+gs-1)
using u64 = unsigned long long;

template <typename R> struct CdfType;
template <> struct CdfType<double> { using T = double; };
template <> struct CdfType<float> { using T = unsigned; };

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// offset (in nodes) of level l of a tree over n leaves: levels stored back to back
__host__ __device__ __forceinline__ int tree_off(int n, int l) { return 2 * n - 2 * (n >> l); }

struct Layout {
    size_t tree, island, small, total;   // byte offsets
    size_t cdf, xs, red, mxr, sqr;       // island sub-offsets
    size_t cdf_stride, xs_stride, red_stride;
};

// cascade region (in 8-byte slots): upper tree [2P], own record [2G], per-warp
// partial sums [16 warps][kQw], per-level sums [kMaxStages], a few integers
__host__ __device__ inline size_t cascade_slots(const StepParams& p)
{
    return 2 * (size_t)p.P + 2 * (size_t)p.G + kMaxWarps * kQw + kMaxStages + 8 + 3 * kMaxWarps;
}


__host__ __device__ inline Layout make_layout(const StepParams& p)
{
    Layout L;
    const size_t rsz = p.fp64 ? 8 : 4;
    const size_t nwi = (size_t)((p.tpi + 31) / 32);           // warps per island
    // the cascade region: cascade_all's (fused steps, persistent launches), or the split
    // steps' top cascade
    const size_t treeb = p.split ? align16(sizeof(double) * (2 * (size_t)p.G + 16)) : align16(sizeof(double) * cascade_slots(p));
    L.cdf_stride = rsz * (size_t)p.M;                          // double or u32
    L.xs_stride = align16(rsz * (size_t)p.M * p.dx);
    L.red_stride = sizeof(double) * nwi;
    L.cdf = 0;
    L.xs = L.cdf + align16(L.cdf_stride * p.G);
    L.red = L.xs + L.xs_stride * p.G;
    L.mxr = L.red + align16(L.red_stride * p.G);
    L.sqr = L.mxr + align16(L.red_stride * p.G);              // per-warp sums of squared weights
    const size_t islandb = L.sqr + align16(L.red_stride * p.G);
    L.tree = 0;
    L.island = 0;                                             // overlaps the cascade region
    L.small = align16(treeb > islandb ? treeb : islandb);
    const size_t smallb = align16(sizeof(double) * (size_t)p.G) + align16(2 * sizeof(int) * (size_t)p.G)
                          + align16(sizeof(double) * (size_t)p.G) + align16(sizeof(int) * (size_t)p.G)
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

// Barrier of the nthreads threads (a multiple of 32) that execute it with this
// id (1..15; id 0 is __syncthreads): the warps of one island sync among
// themselves without waiting for the CTA's other islands.
__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// max / sum over each aligned group of n lanes (n a power of 2, at most 32)
template <typename V>
__device__ __forceinline__ V group_max(V v, int n)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (o < n) {
            const V w = __shfl_xor_sync(0xffffffffu, v, o);
            v = (w > v) ? w : v;
        }
    }
    return v;
}

template <typename V>
__device__ __forceinline__ V group_sum(V v, int n)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        if (o < n) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of eight doubles at once (a reduce-scatter butterfly: at each of the first three
// levels a lane keeps half of its values and adds the partner's copy of that half; 7 + 2
// additions a lane instead of 8 x 5).  Returns at every lane the warp total of value
// (lane >> 2) & 7.
__device__ __forceinline__ double warp_reduce_scatter8(const double (&v)[8], int lane)
{
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
    double h4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        h4[i] = (b4 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[i + 4], 16);
    double h2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
        h2[i] = (b3 ? h4[i + 2] : h4[i]) + __shfl_xor_sync(0xffffffffu, b3 ? h4[i] : h4[i + 2], 8);
    double h = (b2 ? h2[1] : h2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? h2[0] : h2[1], 4);
    h += __shfl_xor_sync(0xffffffffu, h, 2);
    h += __shfl_xor_sync(0xffffffffu, h, 1);
    return h;
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

// max / sum over the whole CTA (blockDim a multiple of 32); sh: kMaxWarps slots
template <typename V>
__device__ __forceinline__ V block_max(V v, V* sh, int nw)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    V r = sh[0];
    for (int w = 1; w < nw; ++w) r = sh[w] > r ? sh[w] : r;
    return r;
}

template <typename V>
__device__ __forceinline__ V block_max(V v, V* sh)
{
    return block_max(v, sh, (int)(blockDim.x >> 5));
}

// Programmatic dependent launch: wait until the previous kernel of the stream
// has completed and its memory is visible (returns at once for a kernel
// launched without the attribute), and let the next kernel start launching.
__device__ __forceinline__ void dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// A thread's PPT consecutive particles as one vector access (the caller checks
// that the first index is a multiple of PPT), read through L2.
template <typename R, int PPT>
__device__ __forceinline__ void load_run(const R* src, R* out)
{
    if constexpr (sizeof(R) == 4 && PPT % 4 == 0) {
#pragma unroll
        for (int q = 0; q < PPT; q += 4) {
            const float4 v = __ldcg(reinterpret_cast<const float4*>(src) + q / 4);
            out[q] = v.x; out[q + 1] = v.y; out[q + 2] = v.z; out[q + 3] = v.w;
        }
    } else if constexpr (sizeof(R) == 4 && PPT == 2) {
        const float2 v = __ldcg(reinterpret_cast<const float2*>(src));
        out[0] = v.x; out[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < PPT; q += 2) {
            const double2 v = __ldcg(reinterpret_cast<const double2*>(src) + q / 2);
            out[q] = v.x; out[q + 1] = v.y;
        }
    }
}

template <typename R, int PPT>
__device__ __forceinline__ void store_run(R* dst, const R* in)
{
    if constexpr (sizeof(R) == 4 && PPT % 4 == 0) {
#pragma unroll
        for (int q = 0; q < PPT; q += 4)
            reinterpret_cast<float4*>(dst)[q / 4] = make_float4(in[q], in[q + 1], in[q + 2], in[q + 3]);
    } else if constexpr (sizeof(R) == 4 && PPT == 2) {
        *reinterpret_cast<float2*>(dst) = make_float2(in[0], in[1]);
    } else {
#pragma unroll
        for (int q = 0; q < PPT; q += 2) reinterpret_cast<double2*>(dst)[q / 2] = make_double2(in[q], in[q + 1]);
    }
}

// float value of a 64-bit integer by its leading-one position (truncated to 24
// bits; integer pipe only)
__device__ __forceinline__ float u64_to_float(u64 v)
{
    if (v == 0ull) return 0.0f;
    const int lz = __clzll(v);
    const u64 n = v << lz;
    return __uint_as_float(((unsigned)(190 - lz) << 23) | (unsigned)((n >> 40) & 0x7fffffu));
}

// Island weight as stored: 64 bits (a double in [0.5,1) on the FP64 path, an
// integer mantissa in [2^63, 2^64) on the FP32-mixed path; 0 = weight zero)
// and a binary exponent.
struct XW {
    u64 bits;
    int e;
};

// double v = r 2^e with r in [0.5, 1), by exponent-field manipulation for
// normal v; frexp for subnormal v.
__device__ __forceinline__ XW xw_from_double(double v, int e_add)
{
    XW w;
    const long long b = __double_as_longlong(v);
    if (b <= 0 || b >= (0x7ffLL << 52)) {       // zero, negative, inf or NaN
        w.bits = 0;
        w.e = 0;
        return w;
    }
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) {
        int e2;
        w.bits = (u64)__double_as_longlong(frexp(v, &e2));
        w.e = e2 + e_add;
        return w;
    }
    w.bits = (u64)((b & ~(0x7ffLL << 52)) | (1022LL << 52));
    w.e = ex - 1022 + e_add;
    return w;
}

// integer v 2^e_add, normalised so that the top bit of the mantissa is set;
// the stored value is mantissa 2^(e - 64)
__device__ __forceinline__ XW xw_from_u64(u64 v, int e_add)
{
    XW w;
    if (v == 0ull) {
        w.bits = 0;
        w.e = 0;
        return w;
    }
    const int lz = __clzll(v);
    w.bits = v << lz;
    w.e = e_add + 64 - lz;
    return w;
}

// Arithmetic of the cascade for each precision (see file comment).
// v 2^-sh for v >= 0 and sh >= 0: the exponent field lowered by sh on the integer pipe when
// the result stays normal (exact, as ldexp); ldexp itself for a zero, subnormal or
// non-finite v, or a result that would be subnormal
__device__ __forceinline__ double scale_down(double v, int sh)
{
    const long long b = __double_as_longlong(v);
    const int ex = (int)(b >> 52);                    // biased exponent of a non-negative v
    if ((unsigned)sh < (unsigned)ex && ex < 0x7FF) return __longlong_as_double(b - ((long long)sh << 52));
    return ldexp(v, -sh);
}

template <bool FX> struct Casc;
template <> struct Casc<false> {
    using V = double;
    using Qt = double;
    // leaf = W 2^-e_ref
    __device__ static int frac(const StepParams&) { return 0; }
    __device__ static bool positive(u64 b) { return (long long)b > 0; }
    __device__ static V leaf(u64 b, int de, int) { return ldexp(__longlong_as_double((long long)b), de); }
    __device__ static V rescale(V v, int sh) { return scale_down(v, sh); }
    __device__ static Qt qscale(Qt q, int sh2) { return scale_down(q, sh2); }
    __device__ static Qt qv(V v) { return v; }
    __device__ static double to_d(V v) { return v; }
    __device__ static XW weight(V bsum, int e_add) { return xw_from_double(bsum, e_add); }
    __device__ static Qt tau(const StepParams& p) { return p.tau; }
    // u tot < x, u = (w + 0.5) 2^-32
    __device__ static bool below(uint32_t w, V tot, V x) { return unif_f64(w) * tot < x; }
};
template <> struct Casc<true> {
    using V = u64;
    using Qt = float;
    // stored weight mantissa * 2^(e-64); leaf = mantissa >> (e_ref - e + 64 - frac)
    // = W 2^(frac - e_ref) < 2^frac.  With frac = 63 - log2 m a sum over all m
    // islands stays below 2^63.
    __device__ static int frac(const StepParams& p) { return 63 - p.S; }
    __device__ static bool positive(u64 b) { return b != 0ull; }
    __device__ static V leaf(u64 b, int de, int fr)
    {
        const int sh = 64 - fr - de;
        return sh < 64 ? (b >> sh) : 0ull;
    }
    __device__ static V rescale(V v, int sh) { return sh < 64 ? (v >> sh) : 0ull; }
    __device__ static Qt qscale(Qt q, int sh2) { return sh2 < 250 ? ldexpf(q, -sh2) : 0.0f; }
    __device__ static Qt qv(V v) { return u64_to_float(v) * 0x1p-62f; }
    __device__ static double to_d(V v) { return (double)v; }
    __device__ static XW weight(V bsum, int e_add) { return xw_from_u64(bsum, e_add); }
    __device__ static Qt tau(const StepParams& p) { return p.tau_f; }
    // u tot < x with u = (2w+1) 2^-33, exactly: (2w+1) tot < 2^33 x in 128 bits
    __device__ static bool below(uint32_t w, V tot, V x)
    {
        const u64 w2 = 2ull * (u64)w + 1ull;
        const u64 p_lo = w2 * tot, p_hi = __umul64hi(w2, tot);
        const u64 r_lo = x << 33, r_hi = x >> 31;
        return (p_hi < r_hi) || (p_hi == r_hi && p_lo < r_lo);
    }
};

template <typename V> __device__ __forceinline__ bool pos_v(V v) { return v > (V)0; }
// a sum of non-negative weights (never NaN) is positive iff its bit pattern is
template <> __device__ __forceinline__ bool pos_v<double>(double v) { return __double_as_longlong(v) > 0; }

// ---------------------------------------------------------------------------
// Cascade of step tp for filter c (see file comment), run by one CTA: the
// cascade kernel's, or the persistent kernel's that holds the filter (or its
// first CTA).  Reads the CTA records of step tp, builds the upper tree, decides
// s*, and writes what the next step needs (the summary, the upper-tree level of
// the block means when it lies above the CTAs, the inherited blocks when a
// stage interacted), log Z and the records of the run.  Every thread of the
// CTA calls it.
// ---------------------------------------------------------------------------
// The run's records of step tp (one thread): log Z^N_tp when traced or at
// tp = T, s*, and ENF_{tp,1..S} (stages from s* on repeat ENF_{s*}) with
// ENF_{tp+1,0}.  Q[l] = sum over level-l blocks of the squared block sums,
// filled at least up to level s*-1.
template <bool FX>
__device__ void cascade_records(const StepParams& p, int c, int tp, int ss, typename Casc<FX>::V tot, int emax,
                                const typename Casc<FX>::Qt* Q)
{
    using C = Casc<FX>;
    const int m = p.m, S = p.S;
    const auto tq = C::qv(tot);
    if (p.trace || tp == p.T) {
        // log Z^N_tp = log(m^-1 sum_k W^k), sum_k W^k = Tot 2^(emax - frac);
        // the FP32-mixed weights leave out M^-tp
        double lz = pos_v(tot)
            ? log(C::to_d(tot)) - log((double)m) + (double)(emax - C::frac(p)) * 0.6931471805599453
            : -INFINITY;
        if (FX) lz -= (double)tp * log((double)p.M);
        if (p.trace) p.trace[(size_t)c * p.T + (tp - 1)] = lz;
        if (tp == p.T) p.logz[c] = lz;
    }
    // the records count stages of r = 2^rb islands: stage s starts at binary stage
    // rb (s-1) + 1, and s* - 1 binary stages interacted (a multiple of rb, or S)
    const int Sr = S / p.rb, ssr = (ss - 1) / p.rb + 1;
    if (p.sstar) p.sstar[(size_t)c * p.T + (tp - 1)] = ssr;
    if (p.enf) {
        double* e = p.enf + ((size_t)c * p.T + (tp - 1)) * (Sr + 1);
        double last = 1.0;
        for (int s = 1; s <= Sr; ++s) {
            const int sb = p.rb * (s - 1) + 1;
            const int sr = sb <= ss ? sb : ss;
            const double v = pos_v(tot)
                ? (double)tq * (double)tq * ldexp(1.0, sr - 1) / ((double)m * (double)Q[sr - 1]) : 0.0;
            e[s] = v;
            if (s == ssr) last = v;
        }
        if (tp < p.T) p.enf[((size_t)c * p.T + tp) * (Sr + 1)] = pos_v(tot) ? (ssr <= Sr ? last : 1.0) : 0.0;
    }
}

// The block sums of step tp (tree level l: sums over aligned blocks of 2^l
// islands), where the island CTAs of step tp+1 find them:
//  * levels below g: the CTA records, each in its own scale 2^pe;
//  * split steps, levels g .. g+gs-1: the group records of the tail cascade
//    (groups of 2^gs CTAs), each in its own scale 2^ge;
//  * above: the upper tree ut in the 2^emax scale (fused steps: from level g,
//    in shared memory; split steps: from level g+gs, the top tree in utg).
// at(l, q, false) gives a node in its source's scale, at(l, q, true) in the
// 2^emax scale; weight(l, q) the extended-range weight of a block mean.
template <bool FX>
struct BlockSums {
    using C = Casc<FX>;
    using V = typename C::V;
    const StepParams& p;
    int c, tp, emax;
    const V* ut;             // upper tree (shared or global memory)
    bool ut_global;
    bool tail;               // split steps: group records between the CTA records and ut

    __device__ const int* pe() const { return p.pe[tp & 1] + (size_t)c * p.P; }
    __device__ const V* pt() const { return reinterpret_cast<const V*>(p.pt[tp & 1]) + (size_t)c * p.P * 2 * p.G; }
    __device__ int top_level() const { return tail ? p.g + p.gs : p.g; }
    __device__ V utv(int i) const { return ut_global ? __ldcg(&ut[i]) : ut[i]; }
    // does the tree between levels L and Lt (a group of r members) lie in one source?
    __device__ bool local(int L, int Lt) const
    {
        const int g = p.g, h = top_level();
        return Lt <= g || L >= h || (tail && L >= g && Lt <= h);
    }
    // node q of level l and its source's binary exponent (the node is V * 2^(exp - frac))
    __device__ V raw(int l, int q, int& ex) const
    {
        const int g = p.g;
        if (l < g) {
            const int jc = q >> (g - l);
            ex = __ldcg(&pe()[jc]);
            return __ldcg(&pt()[(size_t)jc * 2 * p.G + tree_off(p.G, l) + (q - (jc << (g - l)))]);
        }
        if (l < top_level()) {
            const int u = l - g, gr = q >> (p.gs - u), GS = 1 << p.gs;
            ex = __ldcg(&p.ge[tp & 1][(size_t)c * p.NG + gr]);
            const V* gt = reinterpret_cast<const V*>(p.gtr[tp & 1]) + ((size_t)c * p.NG + gr) * 2 * GS;
            return __ldcg(&gt[tree_off(GS, u) + (q - (gr << (p.gs - u)))]);
        }
        ex = emax;
        return utv(tree_off(tail ? p.NG : p.P, l - top_level()) + q);
    }
    __device__ V at(int l, int q, bool common) const
    {
        int ex;
        const V v = raw(l, q, ex);
        if (!common || l >= top_level()) return v;
        return ex == INT_MIN ? (V)0 : C::rescale(v, emax - ex);
    }
    // W = (block sum at level l) / 2^l, extended range
    __device__ XW weight(int l, int q) const
    {
        int ex;
        const V v = raw(l, q, ex);
        if (ex == INT_MIN) return XW{0ull, 0};
        return C::weight(v, ex - C::frac(p) - l);
    }
};

// src(k), the block island k holds after the interacting stages of step tp:
// lvl = s*-1 binary levels, i.e. lvl/rb stages of r = 2^rb islands, walked from
// the last interacting stage down, j = k at the top.  At stage s the island j
// draws a member of its group (the r aligned blocks of level L = rb (s-1) under
// j's block of level L + rb) with probability proportional to the members'
// block sums, which are proportional to their weights before the stage: the
// first member c with u tot < C_c (C the cumulative sums in member order, tot
// the group's sum), found by descending the rb binary tree levels under the
// group's node with the one uniform u of (tp, s, j).  With every weight zero it
// takes the last member.  A group whose tree lies in one source (a CTA record,
// a group record, the upper tree) is compared in that source's scale, else in
// the 2^emax scale.
template <bool FX>
__device__ int walk_src(const BlockSums<FX>& bs, const Stream& st, int k, int lvl)
{
    using C = Casc<FX>;
    using V = typename C::V;
    const int rb = bs.p.rb, tp = bs.tp;
    int j = k;
    for (int s = lvl / rb; s >= 1; --s) {
        const int L = rb * (s - 1), Lt = L + rb;
        const bool common = !bs.local(L, Lt);
        const uint32_t wu = st.draw((uint32_t)j, (uint32_t)tp, KIND_ISLAND, (uint32_t)s).x;
        int n = (j >> Lt) << 1;                   // left child of the group's node, level Lt-1
        V left = bs.at(Lt - 1, n, common);
        const V tot = left + bs.at(Lt - 1, n + 1, common);
        V acc = (V)0;
        for (int l = Lt - 1;; --l) {
            if (!C::below(wu, tot, acc + left)) {
                acc += left;
                ++n;
            }
            if (l == L) break;
            n <<= 1;
            left = bs.at(l - 1, n, common);
        }
        const int mask = ((1 << rb) - 1) << L;
        j = (j & ~mask) | ((n << L) & mask);
    }
    return j;
}

// Where the cascade's result goes: to global memory for the next step's CTAs
// (the summary, cup, nsrc), or, when a CTA runs the cascade itself before its
// island work (fused step), straight into that CTA's own island slots.
struct CascadeOwn {
    int k0;            // first island of the CTA
    u64* w;            // [G] weight mantissas
    int* we;           // [G] weight exponents
    int* src;          // [G] inherited blocks
};

// A CTA's own islands after the cascade of step tp: the weight W^k_{tp+1,0}
// (the block mean at level s*-1) and the inherited block src(k), walked from
// stage s*-1 down.
template <bool FX>
__device__ void own_outputs(const BlockSums<FX>& bs, const Stream& st, int ss, const CascadeOwn& own)
{
    using C = Casc<FX>;
    const StepParams& p = bs.p;
    const int G = p.G, g = p.g;
    const int lvl = ss - 1;
    const bool dead = (bs.emax == INT_MIN);
    for (int gi = threadIdx.x; gi < G; gi += blockDim.x) {
        const int k = own.k0 + gi;
        XW w{0ull, 0};
        if (!dead) {
            if (lvl == 0 && g == 0 && !bs.tail) {   // the island is the CTA: its record top, rescaled
                const int ej = __ldcg(&bs.pe()[own.k0]);
                if (ej != INT_MIN)
                    w = C::weight(C::rescale(__ldcg(&bs.pt()[(size_t)own.k0 * 2 * G]), bs.emax - ej),
                                  bs.emax - C::frac(p));
            } else {
                w = bs.weight(lvl, k >> lvl);
            }
        }
        own.w[gi] = w.bits;
        own.we[gi] = w.e;
        own.src[gi] = walk_src<FX>(bs, st, k, lvl);
    }
}

// OWN: the result goes to the calling CTA's own islands (fused steps), so the
// code that writes it for the next step's CTAs is compiled out
// FP: the filter's shape fixed at compile time (FP = 1: m = 1024 islands in 256 CTAs of
// 4 islands and 256 threads, the fused shape of the 1024 x 256 workload) or read at run
// time (FP = 0); the loops over the records then unroll.
template <bool FX, bool OWN = false, int FP = 0>
__device__ void cascade_all(const StepParams& p, int c, int tp, const Stream& st, double* raw,
                            const CascadeOwn* own = nullptr, bool records = true)
{
    using C = Casc<FX>;
    using V = typename C::V;
    using Qt = typename C::Qt;
    const int m = FP ? 1024 : p.m, S = FP ? 10 : p.S, P = FP ? 256 : p.P, G = FP ? 4 : p.G, g = FP ? 2 : p.g;
    const int SU = S - g;
    const int tid = threadIdx.x, nthr = FP ? 256 : (int)blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const int* pe = p.pe[tp & 1] + (size_t)c * P;
    const V* pt = reinterpret_cast<const V*>(p.pt[tp & 1]) + (size_t)c * P * 2 * G;
    const Qt* pq = reinterpret_cast<const Qt*>(p.pq[tp & 1]) + (size_t)c * P * 8;
    // the upper tree [2P]: in shared memory, or (split steps) in global memory,
    // where the next step's island kernels read it
    // (split steps run their cascade as group_cascade + top_cascade instead)
    const int uo = 2 * P;
    V* ut = reinterpret_cast<V*>(raw);
    Qt* Qw = reinterpret_cast<Qt*>(raw + uo + 2 * G);             // [nw][kQw]
    Qt* Q = reinterpret_cast<Qt*>(raw + uo + 2 * G + kMaxWarps * kQw);   // [kMaxStages]
    int* iscal = reinterpret_cast<int*>(raw + uo + 2 * G + kMaxWarps * kQw + kMaxStages);
    double* wpart = raw + uo + 2 * G + kMaxWarps * kQw + kMaxStages + 8;     // [3][kMaxWarps] per-warp partials
    int* w_emax = reinterpret_cast<int*>(wpart);
    V* w_tot = reinterpret_cast<V*>(wpart + kMaxWarps);
    Qt* w_q0 = reinterpret_cast<Qt*>(wpart + 2 * kMaxWarps);

    // 0. (own islands) the CTA's own record, needed on the common path s* = 1,
    //    loaded together with the other records
    V own_leaf = (V)0;
    int own_e = INT_MIN;
    if (OWN && tid < G) {
        const int jo = own->k0 >> g;
        own_leaf = __ldcg(&pt[(size_t)jo * 2 * G + tid]);
        own_e = __ldcg(&pe[jo]);
    }

    // 1. the lane's records (read once, all fields at once) and the largest
    //    exponent over the records with a nonzero top
    constexpr int kRec = kCachedChunks;
    int re[kRec];
    V rt[kRec];
    Qt rq[kRec][4];
    int emax = INT_MIN;
#pragma unroll
    for (int i = 0; i < kRec; ++i) {
        const int j = (warp + i * nw) * 32 + lane;
        re[i] = INT_MIN;
        rt[i] = (V)0;
#pragma unroll
        for (int l = 0; l < 4; ++l) rq[i][l] = (Qt)0;
        if (j < P) {
            re[i] = __ldcg(&pe[j]);
            rt[i] = __ldcg(&pt[(size_t)j * 2 * G + tree_off(G, g)]);
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (l < g) rq[i][l] = __ldcg(&pq[(size_t)j * 8 + l]);
        }
    }
#pragma unroll
    for (int i = 0; i < kRec; ++i)
        if (pos_v(rt[i]) && re[i] > emax) emax = re[i];
    for (int j = (warp + kRec * nw) * 32 + lane; j < P; j += 32 * nw) {
        const int e = __ldcg(&pe[j]);
        if (pos_v(__ldcg(&pt[(size_t)j * 2 * G + tree_off(G, g)])) && e > emax) emax = e;
    }
    emax = warp_max(emax);
    if (lane == 0) w_emax[warp] = emax;
    __syncthreads();
    emax = INT_MIN;
    for (int w = 0; w < nw; ++w) emax = max(emax, w_emax[w]);
    const bool dead = (emax == INT_MIN);

    // 1b. fast path.  Stage 1 needs only Tot = sum_k W^k and Q_0 = sum_k (W^k)^2
    //     (ENF_1 = Tot^2 / (m Q_0)); when it does not interact (always under
    //     NEVER, and on most ADAPTIVE steps) s* = 1, every island keeps its own
    //     weight and block, and the tree of block sums is not needed.
    if (p.mode != 1) {
        V tpart = (V)0;
        Qt qpart = (Qt)0;
        for (int i = 0, j = warp * 32 + lane; j < P; ++i, j += 32 * nw) {
            int e;
            V top;
            Qt q0r = (Qt)0;
            if (i < kRec) {
                e = INT_MIN;
                top = (V)0;
#pragma unroll
                for (int r = 0; r < kRec; ++r)
                    if (r == i) {
                        e = re[r];
                        top = rt[r];
                        q0r = rq[r][0];
                    }
            } else {
                e = __ldcg(&pe[j]);
                top = __ldcg(&pt[(size_t)j * 2 * G + tree_off(G, g)]);
                if (g >= 1) q0r = __ldcg(&pq[(size_t)j * 8]);
            }
            if (!dead && pos_v(top)) {
                const int sh = emax - e;
                const V v = C::rescale(top, sh);
                tpart += v;
                if (g >= 1) {
                    qpart += C::qscale(q0r, 2 * sh);
                } else {
                    const Qt q = C::qv(v);
                    qpart += q * q;
                }
            }
        }
        V tot = (V)0;
        Qt q0 = (Qt)0;
        if (!FX && nw <= 16) {
            // FP64: the two sums in the two half-warps after one exchange (lanes 0-15 the
            // weights, 16-31 the squares: 5 additions a thread instead of 10); then the
            // warps' partials the same way over lanes 0 .. nw-1 and 16 .. 16+nw-1
            const bool hi = (lane & 16) != 0;
            double h = (double)(hi ? qpart : tpart) +
                       __shfl_xor_sync(0xffffffffu, (double)(hi ? tpart : qpart), 16);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
            if (lane == 0) w_tot[warp] = (V)h;
            if (lane == 16) w_q0[warp] = (Qt)h;
            __syncthreads();
            const int lw = lane & 15;
            double v = 0.0;
            if (lw < nw) v = hi ? (double)w_q0[lw] : (double)w_tot[lw];
#pragma unroll
            for (int o = 8; o > 0; o >>= 1)
                if (o < nw) v += __shfl_xor_sync(0xffffffffu, v, o);
            tot = (V)__shfl_sync(0xffffffffu, v, 0);
            q0 = (Qt)__shfl_sync(0xffffffffu, v, 16);
        } else {
            tpart = warp_sum(tpart);
            qpart = warp_sum(qpart);
            if (lane == 0) {
                w_tot[warp] = tpart;
                w_q0[warp] = qpart;
            }
            __syncthreads();
            for (int w = 0; w < nw; ++w) {
                tot += w_tot[w];
                q0 += w_q0[w];
            }
        }
        const Qt tq = C::qv(tot);
        const bool quiet1 = p.mode == 0 || (pos_v(tot) && !(tq * tq < C::tau(p) * (Qt)m * q0));
        if (quiet1) {
            if (tid == 0 && records) {
                Q[0] = q0;
                cascade_records<FX>(p, c, tp, 1, tot, emax, Q);
            }
            if (OWN) {
                // s* = 1: every own island keeps its weight (level 0 of the own
                // record, or the rescaled record top when the CTA is one island)
                // and its block
                if (tid < G) {
                    XW w{0ull, 0};
                    if (!dead && own_e != INT_MIN)
                        w = g >= 1 ? C::weight(own_leaf, own_e - C::frac(p))
                                   : C::weight(C::rescale(own_leaf, emax - own_e), emax - C::frac(p));
                    own->w[tid] = w.bits;
                    own->we[tid] = w.e;
                    own->src[tid] = own->k0 + tid;
                }
                return;
            }
            if (tid == 0) {
                p.csum[(size_t)c * 4 + 0] = 1;
                p.csum[(size_t)c * 4 + 1] = emax;
            }
            if (g == 0) {     // level 0 lies above the CTAs: the rescaled record tops
                for (int j = tid; j < P; j += nthr) {
                    const int e = __ldcg(&pe[j]);
                    const V top = __ldcg(&pt[(size_t)j * 2 * G]);
                    reinterpret_cast<V*>(p.cup)[(size_t)c * P + j] =
                        (!dead && pos_v(top)) ? C::rescale(top, emax - e) : (V)0;
                }
            }
            return;
        }
    }

    // 2. upper leaves (record tops rescaled to 2^emax), the lower upper-tree
    //    levels by warp shuffles, and every level's partial sum of squares
    const int L5 = SU < kShuffleLevels ? SU : kShuffleLevels;
    Qt qlow[4];                        // global levels 0..g-1 (from the records)
    Qt qu[kShuffleLevels + 1];         // global levels g..g+L5 (upper tree)
#pragma unroll
    for (int l = 0; l < 4; ++l) qlow[l] = (Qt)0;
#pragma unroll
    for (int u = 0; u <= kShuffleLevels; ++u) qu[u] = (Qt)0;
    int ci = 0;
    for (int ch = warp; ch * 32 < P; ch += nw, ++ci) {
        const int j = ch * 32 + lane;
        V v = (V)0;
        if (j < P) {
            int e = INT_MIN;
            V top = (V)0;
            Qt ql[4] = {(Qt)0, (Qt)0, (Qt)0, (Qt)0};
            if (ci < kRec) {
#pragma unroll
                for (int i = 0; i < kRec; ++i)
                    if (i == ci) {
                        e = re[i];
                        top = rt[i];
#pragma unroll
                        for (int l = 0; l < 4; ++l) ql[l] = rq[i][l];
                    }
            } else {
                e = __ldcg(&pe[j]);
                top = __ldcg(&pt[(size_t)j * 2 * G + tree_off(G, g)]);
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    if (l < g) ql[l] = __ldcg(&pq[(size_t)j * 8 + l]);
            }
            if (!dead && pos_v(top)) {
                const int sh = emax - e;
                v = C::rescale(top, sh);
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    if (l < g) qlow[l] += C::qscale(ql[l], 2 * sh);
            }
            ut[j] = v;
            const Qt q = C::qv(v);
            qu[0] += q * q;
        }
#pragma unroll
        for (int u = 1; u <= kShuffleLevels; ++u) {
            if (u <= L5) {
                v += __shfl_down_sync(0xffffffffu, v, 1 << (u - 1));
                if ((lane & ((1 << u) - 1)) == 0 && (j >> u) < (P >> u)) {
                    ut[tree_off(P, u) + (j >> u)] = v;
                    const Qt q = C::qv(v);
                    qu[u] += q * q;
                }
            }
        }
    }
    if constexpr (!FX && FP == 1) {
        // FP64, fixed shape (g = 2, L5 = 5): the eight per-level partial sums reduced together
        double vals[8] = {qlow[0], qlow[1], qu[0], qu[1], qu[2], qu[3], qu[4], qu[5]};
        const double s = warp_reduce_scatter8(vals, lane);
        if ((lane & 3) == 0) Qw[warp * kQw + (lane >> 2)] = s;
    } else {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (l < g) {
                const Qt s = warp_sum(qlow[l]);
                if (lane == 0) Qw[warp * kQw + l] = s;
            }
        }
#pragma unroll
        for (int u = 0; u <= kShuffleLevels; ++u) {
            if (u <= L5) {
                const Qt s = warp_sum(qu[u]);
                if (lane == 0) Qw[warp * kQw + g + u] = s;
            }
        }
    }
    __syncthreads();

    // 3. one warp: remaining upper levels, per-level sums, s*, records
    if (warp == 0) {
        if (lane <= g + L5 && lane < kQw) {
            Qt s = (Qt)0;
            for (int w = 0; w < nw; ++w) s += Qw[w * kQw + lane];
            Q[lane] = s;
        }
        if (SU > L5) {
            // level L5 has n5 = P >> L5 nodes; the levels above them in
            // registers when n5 <= 32, in shared memory otherwise
            const int n5 = P >> L5;
            if (n5 <= 32) {
                V v = lane < n5 ? ut[tree_off(P, L5) + lane] : (V)0;
                Qt qs[kQw];
#pragma unroll
                for (int l = 0; l < kQw; ++l) qs[l] = (Qt)0;
#pragma unroll
                for (int du = 1; du <= 5; ++du) {
                    const int u = L5 + du;
                    if (u <= SU) {
                        v += __shfl_down_sync(0xffffffffu, v, 1 << (du - 1));
                        if ((lane & ((1 << du) - 1)) == 0 && (lane >> du) < (P >> u)) {
                            ut[tree_off(P, u) + (lane >> du)] = v;
                            const Qt q = C::qv(v);
#pragma unroll
                            for (int l = 0; l < kQw; ++l)
                                if (l == du) qs[l] += q * q;
                        }
                    }
                }
#pragma unroll
                for (int du = 1; du <= 5; ++du) {
                    if (L5 + du <= SU) {
                        const Qt sq = warp_sum(qs[du]);
                        if (lane == 0) Q[g + L5 + du] = sq;
                    }
                }
            } else {
                for (int u = L5 + 1; u <= SU; ++u) {
                    __syncwarp();
                    const int n = P >> u;
                    Qt acc = (Qt)0;
                    for (int b = lane; b < n; b += 32) {
                        const V v = ut[tree_off(P, u - 1) + 2 * b] + ut[tree_off(P, u - 1) + 2 * b + 1];
                        ut[tree_off(P, u) + b] = v;
                        const Qt q = C::qv(v);
                        acc += q * q;
                    }
                    acc = warp_sum(acc);
                    if (lane == 0) Q[g + u] = acc;
                }
            }
        }
        __syncwarp();
        const V tot = ut[tree_off(P, SU)];
        const Qt tq = C::qv(tot);
        bool quiet = false;
        if (lane < S) {
            const int s = lane + 1;
            // stage s interacts iff ENF_s < tau, i.e. Tot^2 2^(s-1) < tau m Q_{s-1}; with radix
            // 2^rb only the first binary stage of each group decides (for the whole group)
            quiet = (s - 1) % p.rb == 0 && pos_v(tot) && !(tq * tq * (Qt)(1u << (s - 1)) < C::tau(p) * (Qt)m * Q[s - 1]);
        }
        const unsigned qm = __ballot_sync(0xffffffffu, quiet);
        if (lane == 0) {
            int ss;
            if (p.mode == 0) ss = 1;
            else if (p.mode == 1) ss = S + 1;
            else ss = qm ? __ffs(qm) : S + 1;              // first quiet stage
            iscal[1] = ss;
            if (records) cascade_records<FX>(p, c, tp, ss, tot, emax, Q);
        }
    }
    __syncthreads();

    // 4. for the next step: the summary (s*, largest exponent), the upper-tree
    //    level holding the block means when they span several CTAs, and every
    //    island's inherited block when any stage interacted
    const int ss = iscal[1];
    const int lvl = ss - 1;
    if (OWN) {
        const BlockSums<FX> bs{p, c, tp, emax, ut, false, false};
        own_outputs<FX>(bs, st, ss, *own);
        return;
    }
    if (tid == 0) {
        p.csum[(size_t)c * 4 + 0] = ss;
        p.csum[(size_t)c * 4 + 1] = emax;
    }
    if (lvl >= g) {
        const int n = P >> (lvl - g);
        for (int b = tid; b < n; b += nthr)
            reinterpret_cast<V*>(p.cup)[(size_t)c * P + b] = ut[tree_off(P, lvl - g) + b];
    }
    if (lvl >= 1) {
        const BlockSums<FX> bs{p, c, tp, emax, ut, false, false};
        for (int k = tid; k < m; k += nthr) p.nsrc[(size_t)c * m + k] = walk_src<FX>(bs, st, k, lvl);
    }
}

// log of an island weight as stored (FP32-mixed: 64-bit mantissa times
// 2^(e-64), the common factor M^-t left out; FP64: a double times 2^e)
template <bool FX>
__device__ __forceinline__ double xw_log(u64 bits, int e)
{
    if (bits == 0ull) return -INFINITY;
    return FX ? log((double)bits) + (double)(e - 64) * 0.6931471805599453
              : log(__longlong_as_double((long long)bits)) + (double)e * 0.6931471805599453;
}

// One warp's sums of x_d and x_d^2 over its particles of island k at step t (the
// island terms of the output measures), written to the warp's slot: part s = 0
// the mutated particles, s = 1 the internally resampled ones.
template <typename R, int DX>
__device__ __forceinline__ void moment_sums(const StepParams& p, int c, int t, int k, int wi, int lane, int dx,
                                            int s, const R* s1, const R* s2)
{
    double* slot = p.fsum + ((((size_t)c * p.T + (t - 1)) * p.m + k) * p.fm_nw + wi) * 4 * dx + (size_t)s * 2 * dx;
#pragma unroll
    for (int d = 0; d < DX; ++d) {
        if (d < dx) {
            const R a = warp_sum(s1[d]), b = warp_sum(s2[d]);
            if (lane == 0) {
                slot[d] = (double)a;
                slot[dx + d] = (double)b;
            }
        }
    }
}

// Record of the CTA's island weights after step t (see file comment); warp 0.
template <bool FX>
__device__ void publish_record(const StepParams& p, int c, int t, int jo, const u64* nw_bits, const int* nw_e)
{
    using C = Casc<FX>;
    using V = typename C::V;
    using Qt = typename C::Qt;
    const int G = p.G, g = p.g, lane = threadIdx.x & 31;
    const bool has = lane < G;
    const u64 b = has ? nw_bits[lane] : 0ull;
    const int e = has ? nw_e[lane] : INT_MIN;
    const bool ok = has && C::positive(b);
    const int ej = group_max(ok ? e : INT_MIN, G);     // G <= 16: lanes G.. hold no island
    V v = (ok && ej != INT_MIN) ? C::leaf(b, e - ej, C::frac(p)) : (V)0;
    V* rec = reinterpret_cast<V*>(p.pt[t & 1]) + ((size_t)c * p.P + jo) * 2 * G;
    Qt* pq = reinterpret_cast<Qt*>(p.pq[t & 1]) + ((size_t)c * p.P + jo) * 8;
    Qt q[4] = {(Qt)0, (Qt)0, (Qt)0, (Qt)0};
    if (has) {
        rec[lane] = v;
        const Qt x = C::qv(v);
        q[0] = x * x;
    }
#pragma unroll
    for (int l = 1; l <= kShuffleLevels; ++l) {
        if (l <= g) {
            v += __shfl_down_sync(0xffffffffu, v, 1 << (l - 1));
            if ((lane & ((1 << l) - 1)) == 0 && has) {
                rec[tree_off(G, l) + (lane >> l)] = v;
                const Qt x = C::qv(v);
#pragma unroll
                for (int r = 1; r < 4; ++r)
                    if (r == l) q[r] += x * x;
            }
        }
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (l < g) {
            const Qt s = group_sum(q[l], G);
            if (lane == 0) pq[l] = s;
        }
    }
    if (lane == 0) p.pe[t & 1][(size_t)c * p.P + jo] = ej;
}

// Sums of squares of one tree level per slot, reduced over the CTA: every thread adds
// its part of slot l (l < n), lane 0 of each warp leaves the warp's sums in qw, and the
// first n threads sum the warps into out.
template <typename Qt>
__device__ __forceinline__ void block_sum_slots(const Qt (&part)[kGroupQ], int n, Qt* qw, Qt* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int l = 0; l < kGroupQ; ++l) {
        if (l < n) {
            const Qt v = warp_sum(part[l]);
            if (lane == 0) qw[warp * kGroupQ + l] = v;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < n) {
        Qt v = (Qt)0;
        for (int w = 0; w < nw; ++w) v += qw[w * kGroupQ + threadIdx.x];
        out[threadIdx.x] = v;
    }
    __syncthreads();
}

// A block-sum tree over n = 2^ln leaves held one per thread (thread i holds leaf i;
// blockDim >= n, a multiple of 32): levels 0 .. ln into nd (tree_off(n, l)
// layout), and the sums of squares of the nodes of levels 0 .. ln-1 into
// Q[q0 + l].  Warp shuffles for the levels inside a warp, warp 0 above them.
template <bool FX>
__device__ __forceinline__ void leaf_tree(typename Casc<FX>::V v, int ln, typename Casc<FX>::V* nd,
                                          typename Casc<FX>::Qt* qw, typename Casc<FX>::Qt* Q, int q0, int nw)
{
    using C = Casc<FX>;
    using V = typename C::V;
    using Qt = typename C::Qt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = 1 << ln;
    const bool has = tid < n;
    auto wsum = [&](Qt x, int l) {
        x = warp_sum(x);
        if (lane == 0) qw[warp * kGroupQ + l] = x;
    };
    if (has) nd[tid] = v;
    if (ln > 0) {
        const Qt x = has ? C::qv(v) : (Qt)0;
        wsum(x * x, 0);
    }
#pragma unroll
    for (int u = 1; u <= kShuffleLevels; ++u) {
        if (u <= ln) {
            v += __shfl_down_sync(0xffffffffu, v, 1 << (u - 1));
            const bool node = (lane & ((1 << u) - 1)) == 0 && has;
            if (node) nd[tree_off(n, u) + (tid >> u)] = v;
            if (u < ln) {
                const Qt x = node ? C::qv(v) : (Qt)0;
                wsum(x * x, u);
            }
        }
    }
    __syncthreads();
    // the warps' sums cover levels 0 .. min(ln-1, 5)
    if (tid < (ln < kShuffleLevels + 1 ? ln : kShuffleLevels + 1)) {
        Qt acc = (Qt)0;
        for (int w = 0; w < nw; ++w) acc += qw[w * kGroupQ + tid];
        Q[q0 + tid] = acc;
    }
    // levels above a warp: warp 0 over the (at most 32) nodes of level 5
    if (ln > kShuffleLevels && warp == 0) {
        const int nt = n >> kShuffleLevels;
        V w = lane < nt ? nd[tree_off(n, kShuffleLevels) + lane] : (V)0;
        for (int u = kShuffleLevels + 1; u <= ln; ++u) {
            const int du = u - kShuffleLevels;
            w += __shfl_down_sync(0xffffffffu, w, 1 << (du - 1));
            const bool node = (lane & ((1 << du) - 1)) == 0 && lane < nt;
            if (node) nd[tree_off(n, u) + (lane >> du)] = w;
            if (u < ln) {
                const Qt x = node ? C::qv(w) : (Qt)0;
                const Qt sq = warp_sum(x * x);
                if (lane == 0) Q[q0 + u] = sq;
            }
        }
    }
    __syncthreads();
}

// Split steps: the cascade of step tp in one kernel of NG x B CTAs.  The P CTA
// records of a filter form NG groups of GS = 2^gs consecutive records.
//  (1) group_cascade: CTA grp reduces group grp to a group record -- the largest
//      exponent ge over its records, the block-sum subtree of levels g .. g+gs over
//      its record tops (rescaled to 2^ge), and the sums of squares of levels
//      0 .. g+gs-1 in that scale.
//  (2) top_cascade, by the filter's last CTA: the largest exponent emax over the
//      group records and the stage-1 test; when stage 1 interacts, the tree above
//      the groups (levels g+gs .. S, 2^emax scale) and every level's sum of
//      squares, s*, and the top tree (utg) for step tp+1; the run's records and the
//      summary (s*, emax).
// The island CTAs of step tp+1 then walk their islands' choices through the CTA
// records, the group records and the top tree.  Group records are double-buffered
// by step like the CTA records.  (Measured before: one cascade CTA reading all
// 16384 CTA records of the m = 65536 workload, 21 us a step; the group reduction
// in the tail of the island kernel behind per-CTA tickets, slower, the device-scope
// fence before each island CTA's ticket holding that CTA's slot; the top of the
// cascade in every island CTA, much slower on that workload, where stage 1
// interacts on a third to a half of the steps and every CTA then built the top
// tree.)
// The split cascade's shape: CTA-record levels g, group levels gs, groups NG, binary
// stages S and the cascade CTA's warps, read at run time (FIX = 0) or fixed at compile
// time (FIX = 1) for the m = 65536-island filter of 4-island CTAs (16384 CTA records,
// 128 groups of 128, 128-thread CTAs), whose loops then unroll.
template <int FIX> struct SplitShape {
    int g, gs, NG, S, nw;
    __device__ explicit SplitShape(const StepParams& p)
        : g(p.g), gs(p.gs), NG(p.NG), S(p.S), nw((int)(blockDim.x >> 5)) {}
};
template <> struct SplitShape<1> {
    static constexpr int g = 2, gs = 7, NG = 128, S = 16, nw = 4;
    __device__ explicit SplitShape(const StepParams&) {}
};
__host__ inline bool split_shape_fixed(const StepParams& p, int threads)
{
    return p.g == 2 && p.gs == 7 && p.NG == 128 && p.S == 16 && threads == 128;
}

template <bool FX, int FIX>
__device__ void group_cascade(const StepParams& p, int c, int tp, int grp, unsigned char* sm)
{
    using C = Casc<FX>;
    using V = typename C::V;
    using Qt = typename C::Qt;
    const SplitShape<FIX> sp(p);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = sp.nw;
    const int g = sp.g, G = 1 << g, NG = sp.NG, gs = sp.gs, GS = 1 << gs, P = NG << gs;
    const int h = g + gs;                    // level of the group root
    const int par = tp & 1;
    V* nd = reinterpret_cast<V*>(sm);                                             // [2 GS] tree nodes
    double* rs = reinterpret_cast<double*>(sm + align16(sizeof(double) * 2 * GS));
    Qt* qw = reinterpret_cast<Qt*>(rs);                                           // [kMaxWarps][kGroupQ]
    Qt* Q = reinterpret_cast<Qt*>(rs + kMaxWarps * kGroupQ);                      // [kMaxStages]
    int* red = reinterpret_cast<int*>(rs + kMaxWarps * kGroupQ + kMaxStages);     // [kMaxWarps]
    Qt* qr = reinterpret_cast<Qt*>(rs + kMaxWarps * kGroupQ + kMaxStages + kMaxWarps);   // [kMaxWarps][4]

    // one record a thread: exponent, top, sums of squares of levels < g
    const size_t r0 = (size_t)c * P + (size_t)grp * GS;
    const bool has = tid < GS;
    int e = INT_MIN;
    V top = (V)0;
    Qt q[4] = {(Qt)0, (Qt)0, (Qt)0, (Qt)0};
    if (has) {
        e = __ldcg(&p.pe[par][r0 + tid]);
        top = __ldcg(&reinterpret_cast<const V*>(p.pt[par])[(r0 + tid) * 2 * G + tree_off(G, g)]);
#pragma unroll
        for (int l = 0; l < 4; ++l)
            if (l < g) q[l] = __ldcg(&reinterpret_cast<const Qt*>(p.pq[par])[(r0 + tid) * 8 + l]);
    }
    const bool ok = has && pos_v(top) && e != INT_MIN;
    const int em = block_max(ok ? e : INT_MIN, red, nw);
    const int sh = ok ? em - e : 0;
    // the records' levels below g, rescaled to 2^em
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (l < g) {
            const Qt x = warp_sum(ok ? C::qscale(q[l], 2 * sh) : (Qt)0);
            if (lane == 0) qr[warp * 4 + l] = x;
        }
    }
    leaf_tree<FX>(ok ? C::rescale(top, sh) : (V)0, gs, nd, qw, Q, g, nw);
    if (tid < g) {
        Qt acc = (Qt)0;
        for (int w = 0; w < nw; ++w) acc += qr[w * 4 + tid];
        Q[tid] = acc;
    }
    __syncthreads();
    V* gt = reinterpret_cast<V*>(p.gtr[par]) + ((size_t)c * NG + grp) * 2 * GS;
    for (int i = tid; i < 2 * GS - 1; i += 32 * nw) gt[i] = nd[i];
    Qt* gq = reinterpret_cast<Qt*>(p.gqs[par]) + ((size_t)c * NG + grp) * kGroupQ;
    if (tid < h) gq[tid] = Q[tid];
    if (tid == 0) p.ge[par][(size_t)c * NG + grp] = em;
}

// shared-memory bytes of the split steps' cascade kernels (both): a tree over the
// larger of a group's records and the filter's groups, reduction slots
__host__ __device__ inline size_t split_cascade_smem_bytes(const StepParams& p)
{
    const size_t n = (size_t)((1 << p.gs) > p.NG ? (1 << p.gs) : p.NG);
    return align16(sizeof(double) * 2 * n)
           + align16(sizeof(double) * (kMaxWarps * kGroupQ + kMaxStages + kMaxWarps + kMaxWarps * kGroupQ + 4));
}

template <bool FX, int FIX>
__device__ void top_cascade(const StepParams& p, int c, int tp, unsigned char* sm)
{
    using C = Casc<FX>;
    using V = typename C::V;
    using Qt = typename C::Qt;
    const SplitShape<FIX> sp(p);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = sp.nw;
    const int g = sp.g, NG = sp.NG, gs = sp.gs, GS = 1 << gs, P = NG << gs, S = sp.S, m = 1 << S;
    const int h = g + gs, par = tp & 1;
    V* nd = reinterpret_cast<V*>(sm);                                             // [2 NG]
    double* rs = reinterpret_cast<double*>(sm + align16(sizeof(double) * 2 * NG));
    Qt* qw = reinterpret_cast<Qt*>(rs);                                           // [kMaxWarps][kGroupQ]
    Qt* Q = reinterpret_cast<Qt*>(rs + kMaxWarps * kGroupQ);                      // [kMaxStages]
    int* red = reinterpret_cast<int*>(rs + kMaxWarps * kGroupQ + kMaxStages);     // [kMaxWarps]
    Qt* qr = reinterpret_cast<Qt*>(rs + kMaxWarps * kGroupQ + kMaxStages + kMaxWarps);   // [kMaxWarps][kGroupQ]
    // one group record a thread: exponent, root, sums of squares of levels < h
    const bool has = tid < NG;
    int e = INT_MIN;
    V r = (V)0;
    if (has) {
        e = __ldcg(&p.ge[par][(size_t)c * NG + tid]);
        r = __ldcg(&reinterpret_cast<const V*>(p.gtr[par])[((size_t)c * NG + tid) * 2 * GS + tree_off(GS, gs)]);
    }
    // the group's sums of squares of levels < h, loaded with the rest (one round trip)
    const Qt* gq = reinterpret_cast<const Qt*>(p.gqs[par]) + ((size_t)c * NG + (has ? tid : 0)) * kGroupQ;
    Qt qg[kGroupQ];
#pragma unroll
    for (int l = 0; l < kGroupQ; ++l) qg[l] = (has && l < h) ? __ldcg(&gq[l]) : (Qt)0;
    const bool ok = has && pos_v(r) && e != INT_MIN;
    const int emax = block_max(ok ? e : INT_MIN, red, nw);
    const int sh = ok ? emax - e : 0;
    const V leaf = ok ? C::rescale(r, sh) : (V)0;
    // stage 1 first: it needs only the total and level 0's sum of squares (ENF_1 =
    // Tot^2 / (m Q_0)); when it does not interact (always under NEVER, and on most
    // adaptive steps) s* = 1, the islands keep their blocks and no tree is needed
    if (p.mode != 1) {
        V* vred = reinterpret_cast<V*>(qr);                 // [kMaxWarps] (qr is free until below)
        const V ts = warp_sum(leaf);
        const Qt q0s = warp_sum(ok ? C::qscale(qg[0], 2 * sh) : (Qt)0);
        if (lane == 0) {
            vred[warp] = ts;
            qw[warp] = q0s;
        }
        __syncthreads();
        V tot = (V)0;
        Qt q0 = (Qt)0;
        for (int w = 0; w < nw; ++w) {
            tot += vred[w];
            q0 += qw[w];
        }
        const Qt tq = C::qv(tot);
        const bool quiet1 = p.mode == 0 || (pos_v(tot) && !(tq * tq < C::tau(p) * (Qt)m * q0));
        if (quiet1) {
            if (tid == 0) {
                Q[0] = q0;
                cascade_records<FX>(p, c, tp, 1, tot, emax, Q);
                p.csum[(size_t)c * 4 + 0] = 1;
                p.csum[(size_t)c * 4 + 1] = emax;
            }
            return;
        }
        __syncthreads();                                    // vred, qw reused below
    }
#pragma unroll
    for (int l = 0; l < kGroupQ; ++l) {
        if (l < h) {
            const Qt x = warp_sum(ok ? C::qscale(qg[l], 2 * sh) : (Qt)0);
            if (lane == 0) qr[warp * kGroupQ + l] = x;
        }
    }
    leaf_tree<FX>(leaf, S - h, nd, qw, Q, h, nw);
    if (tid < h) {
        Qt acc = (Qt)0;
        for (int w = 0; w < nw; ++w) acc += qr[w * kGroupQ + tid];
        Q[tid] = acc;
    }
    __syncthreads();
    const V tot = nd[tree_off(NG, S - h)];
    if (warp == 0) {
        const Qt tq = C::qv(tot);
        bool quiet = false;
        if (lane < S) {
            const int s = lane + 1;
            // stage s interacts iff ENF_s < tau; with radix 2^rb only the first binary
            // stage of each group of rb decides
            quiet = (s - 1) % p.rb == 0 && pos_v(tot) &&
                    !(tq * tq * (Qt)(1u << (s - 1)) < C::tau(p) * (Qt)m * Q[s - 1]);
        }
        const unsigned qm = __ballot_sync(0xffffffffu, quiet);
        if (lane == 0) {
            const int ss = p.mode == 0 ? 1 : (p.mode == 1 ? S + 1 : (qm ? __ffs(qm) : S + 1));
            cascade_records<FX>(p, c, tp, ss, tot, emax, Q);
            p.csum[(size_t)c * 4 + 0] = ss;
            p.csum[(size_t)c * 4 + 1] = emax;
        }
    }
    V* ut = reinterpret_cast<V*>(p.utg) + (size_t)c * 2 * P;
    for (int i = tid; i < 2 * NG - 1; i += 32 * nw) ut[i] = nd[i];
}

enum { OP_STEP = 0, OP_PREPARE = 1, OP_FITS = 2, OP_PERSIST_GRID = 3, OP_PERSIST_CTA = 4, OP_CASCADE = 5,
       OP_WIDE_FITS = 6 };

__host__ __device__ inline size_t cascade_smem_bytes(const StepParams& p) { return align16(sizeof(double) * cascade_slots(p)); }

}  // namespace

// ---------------------------------------------------------------------------
// Prologue: model constants of every filter (and the NGM drift table), once
// per pass; also clears the grid barrier and the error word.
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
    if (p.split && i < p.B) p.tick[i] = 0u;       // the split cascade's tickets
}

// ---------------------------------------------------------------------------
// Step t for the G islands k0.. of filter c (see file comment).  Called by every
// thread of the CTA; all barriers inside are CTA-uniform.
// ---------------------------------------------------------------------------
// LV: which launch the body serves, fixed at compile time for the per-step
// kernels (1 fused steps, 2 split steps) or chosen at run time (0).  MC: the island
// size M fixed at compile time (0: read at run time), with TPI = MC / PPT threads an
// island; the loops over an island's particles, the search and the CDF layout then
// unroll and fold (about 13% fewer issue cycles on the m = 65536 x M = 256 workload).
template <typename R, int MODEL, int DX, int PPT, bool REC = true, int LV = 0, int MC = 0>
__device__ __forceinline__ void step_body(const StepParams& p, int t, int c, int k0, unsigned char* smem,
                                          bool dep = false)
{
    using Cdf = typename CdfType<R>::T;
    constexpr bool FX = sizeof(R) == 4;
    constexpr int TPI = MC > 0 ? MC / PPT : 0;
    static_assert(MC == 0 || (TPI >= 32 && (TPI & (TPI - 1)) == 0 && TPI * PPT == MC), "MC = PPT x 2^k, 2^k >= 32");
    const int tid = threadIdx.x;
    const int N = p.N, M = MC > 0 ? MC : p.M, dx = p.dx;
    const int tpi = TPI > 0 ? TPI : p.tpi;
    constexpr int LG_TPI = TPI >= 512 ? 9 : TPI >= 256 ? 8 : TPI >= 128 ? 7 : TPI >= 64 ? 6 : 5;
    const int lg_tpi = TPI > 0 ? LG_TPI : p.lg_tpi;
    const int jo = k0 >> p.g;                  // G, tpi and m/G are powers of 2: shifts, not divisions
    const Layout L = make_layout(p);
    double* tree = reinterpret_cast<double*>(smem + L.tree);
    u64* own_w = reinterpret_cast<u64*>(smem + L.small);
    int* own_we = reinterpret_cast<int*>(smem + L.small + align16(sizeof(double) * p.G));
    int* own_src = own_we + p.G;
    u64* new_w = reinterpret_cast<u64*>(smem + L.small + align16(sizeof(double) * p.G)
                                        + align16(2 * sizeof(int) * p.G));
    int* new_we = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(new_w) + align16(sizeof(double) * p.G));
    double* scal = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(new_we) + align16(sizeof(int) * p.G));
    R* mshared = reinterpret_cast<R*>(reinterpret_cast<unsigned char*>(scal) + align16(sizeof(double) * 16));
    const RunParams run = *p.run;
    const Stream st{p.seed_lo, p.seed_hi, run.iter, (run.chain0 + (uint32_t)c) << 8};
    const bool designated = (k0 == 0);

    // ---- 1. before any dependency: the step's noise (and at t = 1 the prior
    //      draw), from the run parameters and model constants only, which the
    //      kernels of this pass never write ----
    const int g = tid >> lg_tpi, li = tid & (tpi - 1);
    const int lane = tid & 31, wi = li >> 5;   // warp index within the island
    const int k = k0 + g;
    const R* Xp = reinterpret_cast<const R*>(p.X[(t - 1) & 1]);
    const bool vec = (M % PPT) == 0;       // a thread's particles are one aligned vector
    R xp[PPT][DX];
    R z[PPT][DX > 1 ? DX : 1];
    uint32_t w0[PPT], wres[PPT];
    ModelPar<R> mp;
    if (t <= p.T) {
        mp = reinterpret_cast<const ModelPar<R>*>(p.mpar)[c];
        if (MODEL == NGM) mp.drift = reinterpret_cast<const R*>(p.drift)[t - 1];
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            w0[r] = 0;
            wres[r] = 0;
        }
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int i = li * PPT + r;
            if (i < M) {
                const uint32_t unit = (uint32_t)(k * M + i);
                if (t == 1) model_prior<R, MODEL, DX>(mp, st, unit, dx, xp[r]);
                // one-normal models: the thread's particles 2q, 2q+1 share a block
                // (a vector run starts at an even unit: M is a multiple of PPT)
                if constexpr (DX == 1 && MODEL != TOY && MODEL != CP && PPT % 2 == 0) {
                    if (vec) {
                        if ((r & 1) == 0)
                            step_noise_pair<R>(st, unit, (uint32_t)t, z[r][0], z[r + 1][0], w0[r], w0[r + 1], wres[r],
                                               wres[r + 1]);
                        continue;
                    }
                }
                model_step_noise<R, MODEL, DX>(mp, st, unit, (uint32_t)t, dx, z[r], w0[r], wres[r]);
            }
        }
    }

    // the step's observation (and the LGSSM matrices): inputs that no kernel of
    // the pass writes, loaded now so that their latency is off the critical path
    if (t <= p.T) {
        if (MODEL == LGSSM)
            for (int q = tid; q < dx * dx + p.dy * dx; q += blockDim.x) mshared[q] = (R)p.mdata[q];
        for (int q = tid; q < p.dy; q += blockDim.x)
            mshared[dx * dx + p.dy * dx + q] = (R)p.y[(size_t)(t - 1) * p.dy + q];
        if (MODEL == CP && tid == 0) {      // the step's log C(n, k), after y = (k, n)
            const double kk = p.y[(size_t)(t - 1) * p.dy], nn = p.y[(size_t)(t - 1) * p.dy + 1];
            mshared[dx * dx + p.dy * dx + 2] = (R)(lgamma(nn + 1.0) - lgamma(kk + 1.0) - lgamma(nn - kk + 1.0));
        }
    }

    // Split steps: the island kernel of step t-1 has completed before this one starts
    // (the cascade kernel between them lets this kernel launch only after its own wait
    // on that kernel), so the rows and CTA records of step t-1 may be read before the
    // wait; only the cascade's outputs need it.  Fused steps launch directly after the
    // previous island kernel and must wait first.
    constexpr bool kSplitOnly = (LV == 2);
    const bool split_path = kSplitOnly || (LV == 0 && p.split);
    typename Casc<FX>::V own_top = 0;       // the own CTA record's island node (level 0)
    int own_ex = INT_MIN;
    if (kSplitOnly && t >= 2 && t <= p.T && p.g >= 1 && tid < p.G) {
        own_ex = __ldcg(&p.pe[(t - 1) & 1][(size_t)c * p.P + jo]);
        own_top = __ldcg(&reinterpret_cast<const typename Casc<FX>::V*>(p.pt[(t - 1) & 1])
                             [((size_t)c * p.P + jo) * 2 * p.G + tree_off(p.G, 0) + tid]);
    }
    auto load_own_block = [&]() {           // the own block (the parents when the island keeps it)
        if (vec && li * PPT < M) {
#pragma unroll
            for (int d = 0; d < DX; ++d) {
                if (d < dx) {
                    R v[PPT];
                    load_run<R, PPT>(&Xp[((size_t)c * dx + d) * N + (size_t)k * M + li * PPT], v);
#pragma unroll
                    for (int r = 0; r < PPT; ++r) xp[r][d] = v[r];
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < PPT; ++r) {
                const int i = li * PPT + r;
                if (i < M) {
#pragma unroll
                    for (int d = 0; d < DX; ++d)
                        if (d < dx) xp[r][d] = __ldcg(&Xp[((size_t)c * dx + d) * N + (size_t)k * M + i]);
                }
            }
        }
    };
    if (kSplitOnly && t >= 2 && t <= p.T) load_own_block();

    // ---- 2. everything below reads what earlier kernels of the pass wrote ----
    if (dep) {
        dependency_wait();
        allow_dependents();
    }
    if (!kSplitOnly && t >= 2 && t <= p.T) load_own_block();

    // the own islands' weight and source block (written by the cascade of step t-1)
    if (t == 1) {
        for (int gi = tid; gi < p.G; gi += blockDim.x) {
            // W = 1: 0.5 2^1 as a double, 2^63 2^(1-64) as an integer mantissa
            own_w[gi] = FX ? (1ull << 63) : (u64)__double_as_longlong(0.5);
            own_we[gi] = 1;
            own_src[gi] = k0 + gi;
        }
        if (designated && tid == 0 && p.enf) p.enf[(size_t)c * p.T * (p.S / p.rb + 1)] = 1.0;
    } else if (LV == 1 || LV == 3 || (LV == 0 && p.fused)) {
        // this CTA runs the cascade of step t-1 itself, from every CTA record of
        // the filter (the first CTA also writes log Z and the run's records)
        const CascadeOwn own{k0, own_w, own_we, own_src};
        if (MC == 256 && p.m == 1024 && p.G == 4 && blockDim.x == 256)   // the fixed shape (uniform)
            cascade_all<FX, true, 1>(p, c, t - 1, st, tree, &own, designated);
        else
            cascade_all<FX, true>(p, c, t - 1, st, tree, &own, designated);
    } else if (split_path) {
        // the cascade kernel of step t-1 left s*, the largest exponent, the group
        // records and the top tree; this CTA derives its islands' weights and walks.
        // Every thread reads the summary itself (a broadcast load, no barrier).
        const int ss = __ldcg(&p.csum[(size_t)c * 4 + 0]);
        const int emax = __ldcg(&p.csum[(size_t)c * 4 + 1]);
        if (kSplitOnly && ss == 1 && p.g >= 1) {
            // no stage interacted: each island keeps its block and its weight, level 0
            // of the own CTA record (loaded before the wait)
            if (tid < p.G) {
                XW w{0ull, 0};
                if (emax != INT_MIN && own_ex != INT_MIN) w = Casc<FX>::weight(own_top, own_ex - Casc<FX>::frac(p));
                own_w[tid] = w.bits;
                own_we[tid] = w.e;
                own_src[tid] = k0 + tid;
            }
        } else {
            const CascadeOwn own{k0, own_w, own_we, own_src};
            const BlockSums<FX> bs{p, c, t - 1, emax,
                                   reinterpret_cast<const typename Casc<FX>::V*>(p.utg) + (size_t)c * 2 * p.P, true,
                                   true};
            own_outputs<FX>(bs, st, ss, own);
        }
    } else {
        // the cascade's summary of step t-1, this CTA's record of step t-1 and
        // (used only if some stage interacted) the inherited blocks
        int* csum_sh = reinterpret_cast<int*>(scal) + 4;
        u64* rec_sh = reinterpret_cast<u64*>(tree);
        if (tid < 2) csum_sh[tid] = __ldcg(&p.csum[(size_t)c * 4 + tid]);
        if (tid == 2) csum_sh[2] = __ldcg(&p.pe[(t - 1) & 1][(size_t)c * p.P + jo]);
        if (tid < 2 * p.G - 1)
            rec_sh[tid] = __ldcg(&reinterpret_cast<const u64*>(p.pt[(t - 1) & 1])[((size_t)c * p.P + jo) * 2 * p.G + tid]);
        for (int gi = tid; gi < p.G; gi += blockDim.x) own_src[gi] = __ldcg(&p.nsrc[(size_t)c * p.m + k0 + gi]);
        __syncthreads();
        const int ss = csum_sh[0], emax = csum_sh[1], ej = csum_sh[2];
        const int lvl = ss - 1;
        for (int gi = tid; gi < p.G; gi += blockDim.x) {
            XW w{0ull, 0};
            if (emax != INT_MIN) {
                if (lvl < p.g) {
                    if (ej != INT_MIN)
                        w = Casc<FX>::weight(reinterpret_cast<const typename Casc<FX>::V*>(rec_sh)[tree_off(p.G, lvl) + (gi >> lvl)],
                                             ej - Casc<FX>::frac(p) - lvl);
                } else {
                    const typename Casc<FX>::V b =
                        __ldcg(&reinterpret_cast<const typename Casc<FX>::V*>(p.cup)[(size_t)c * p.P + ((k0 + gi) >> lvl)]);
                    w = Casc<FX>::weight(b, emax - Casc<FX>::frac(p) - lvl);
                }
            }
            own_w[gi] = w.bits;
            own_we[gi] = w.e;
            if (ss == 1) own_src[gi] = k0 + gi;
        }
    }

    __syncthreads();

    // ---- lineage of step t-1: parent of particle (k, i) among time-(t-1) particles ----
    if (REC && p.anc != nullptr && t >= 2) {
        const int* ires = p.ires[(t - 1) & 1] + (size_t)c * N;
        int* anc = p.anc + ((size_t)c * p.T + (t - 2)) * N;
        for (int q = tid; q < p.G * M; q += blockDim.x) {
            const int gq = q / M, i = q - gq * M;
            const int par = own_src[gq];
            anc[(k0 + gq) * M + i] = par * M + __ldcg(&ires[par * M + i]);
        }
    }
    if (t == p.T + 1) return;

    // ---- 3. island work of step t ----
    Cdf* cdf_all = reinterpret_cast<Cdf*>(smem + L.island + L.cdf);
    R* xs_all = reinterpret_cast<R*>(smem + L.island + L.xs);
    Cdf* red_all = reinterpret_cast<Cdf*>(smem + L.island + L.red);
    R* mxr_all = reinterpret_cast<R*>(smem + L.island + L.mxr);
    const int nwi = (tpi + 31) >> 5;

    R* Am = mshared;                 // filled before the dependency wait (ordered by the barrier above)
    R* Cm = mshared + dx * dx;
    R* yv = Cm + p.dy * dx;

    const int par = own_src[g];
    Cdf* cdf = cdf_all + (size_t)g * M;
    R* xs = reinterpret_cast<R*>(reinterpret_cast<unsigned char*>(xs_all) + L.xs_stride * g);
    Cdf* red = red_all + (size_t)g * (L.red_stride / sizeof(Cdf));
    R* mxr = mxr_all + (size_t)g * (L.red_stride / sizeof(R));
    double* sqr = reinterpret_cast<double*>(smem + L.island + L.sqr) + (size_t)g * (L.red_stride / sizeof(double));
    // adaptive internal resampling: log(M omega) of the parents, from the inherited block
    // (0 after the parent island resampled; the prior draws at t = 1 carry 0)
    const bool air = REC && p.air;
    R lo[PPT];
#pragma unroll
    for (int r = 0; r < PPT; ++r) lo[r] = (R)0;
    if (air && t >= 2) {
        const R* Lp = reinterpret_cast<const R*>(p.lom[(t - 1) & 1]);
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int i = li * PPT + r;
            if (i < M) lo[r] = __ldcg(&Lp[(size_t)c * N + (size_t)par * M + i]);
        }
    }
    R* Xc = reinterpret_cast<R*>(p.X[t & 1]);

    R xv[PPT][DX];
    R lv[PPT];
    if (t >= 2 && par != k && vec && li * PPT < M) {   // the island inherits another island's block
#pragma unroll
        for (int d = 0; d < DX; ++d) {
            if (d < dx) {
                R v[PPT];
                load_run<R, PPT>(&Xp[((size_t)c * dx + d) * N + (size_t)par * M + li * PPT], v);
#pragma unroll
                for (int r = 0; r < PPT; ++r) xp[r][d] = v[r];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        lv[r] = (R)(-INFINITY);
        const int i = li * PPT + r;
        if (i < M) {
            if (t >= 2 && par != k && !vec) {
#pragma unroll
                for (int d = 0; d < DX; ++d)
                    if (d < dx) xp[r][d] = __ldcg(&Xp[((size_t)c * dx + d) * N + (size_t)par * M + i]);
            }
            model_transition<R, MODEL, DX>(mp, dx, xp[r], xv[r], Am, z[r], w0[r]);
            lv[r] = model_logg<R, MODEL, DX>(mp, yv, dx, p.dy, xv[r], Cm);
            if (air) lv[r] += lo[r];             // log(M omega_i g_t(x_i))
        }
    }
    if (REC && p.grad) {
        // states for the gradient pass: the prior draws x_0 (slot 0, at t = 1)
        // and the time-t particles at the checkpoints (every ckpt steps, and T)
        const int slot = (t % p.ckpt == 0) ? t / p.ckpt : (t == p.T ? p.nck - 1 : -1);
        // [slot][N][DX]: a particle's components together (the backward pass gathers
        // them by parent)
        R* xck = reinterpret_cast<R*>(p.xck) + (size_t)c * p.nck * DX * N;
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int i = li * PPT + r;
            if (i < M) {
                const size_t gi = (size_t)k * M + i;
#pragma unroll
                for (int d = 0; d < DX; ++d) {
                    if (d < dx) {
                        if (t == 1) xck[gi * DX + d] = xp[r][d];
                        if (slot >= 0) xck[((size_t)slot * N + gi) * DX + d] = xv[r][d];
                    }
                }
            }
        }
    }

    if (REC && p.fmom) {       // output measure at s = 0: the mutated particles
        R s1[DX], s2[DX];
#pragma unroll
        for (int d = 0; d < DX; ++d) {
            s1[d] = (R)0;
            s2[d] = (R)0;
#pragma unroll
            for (int r = 0; r < PPT; ++r) {
                if (li * PPT + r < M) {
                    s1[d] += xv[r][d];
                    s2[d] += xv[r][d] * xv[r][d];
                }
            }
        }
        moment_sums<R, DX>(p, c, t, k, wi, lane, dx, 0, s1, s2);
    }

    // island maximum of the log-weights (no NaN among them); FP64: taken on their order keys
    // by the integer pipe
    R mx;
    if constexpr (!FX) {
        long long km = order_key(lv[0]);
#pragma unroll
        for (int r = 1; r < PPT; ++r) {
            const long long kr = order_key(lv[r]);
            km = kr > km ? kr : km;
        }
        mx = from_order_key(warp_max(km));
    } else {
        mx = lv[0];
#pragma unroll
        for (int r = 1; r < PPT; ++r) mx = (lv[r] > mx) ? lv[r] : mx;
        mx = warp_max(mx);
    }
    // an island of several warps (then G <= 8) syncs on its own barrier 1 + g
    if (nwi > 1) {
        if (lane == 0) mxr[wi] = mx;
        named_sync(1 + g, tpi);
        R v = mxr[0];
        for (int w = 1; w < nwi; ++w) v = (mxr[w] > v) ? mxr[w] : v;
        mx = v;
    }
    bool alive;
    if constexpr (!FX) alive = above_neg_inf(mx);
    else alive = (mx > (R)(-INFINITY));

    // The CDF in shared memory, each 128-byte row of it XOR-swizzled by its row
    // index: the binary search's probes at one depth share their low address
    // bits (all are -1 modulo a power of 2), which would put them in one bank;
    // the swizzle spreads them.  Only when M fills whole rows (islands stay
    // row-aligned); a thread's PPT consecutive entries stay in one 16-byte group.
    constexpr int kRowShift = sizeof(Cdf) == 4 ? 5 : 4;
    const int rowmask = (M & ((1 << kRowShift) - 1)) == 0 ? (1 << kRowShift) - 1 : 0;
    auto cdf_ix = [rowmask](int i) { return i ^ ((i >> kRowShift) & rowmask); };
    // Islands of M = 2^k particles keep the CDF as a search tree in breadth-first
    // (Eytzinger) order instead: C_j (j < M-1) at node (r >> (z+1)) + 2^(k-1-z) of the
    // complete tree over the M-1 boundaries, r = j+1 its in-order rank and z = ctz(r),
    // and the total C_{M-1} at node 0.  The search then walks node -> 2 node + [C <= u],
    // one shared-memory load, compare and index update per level, and the answer
    // (the number of boundaries at or below u) is the first i with C_i > u.  The probes
    // of one level lie in 2^l consecutive words, so the shallow levels need no swizzle.
    const bool eyt = M >= 2 && (M & (M - 1)) == 0;
    const int lgM = 31 - __clz(M);
    auto eyt_ix = [lgM, M](int j) {
        if (j == M - 1) return 0;
        const int r = j + 1, z = __ffs(r) - 1;
        return (r >> (z + 1)) + (1 << (lgM - 1 - z));
    };

    // weights and the thread-local inclusive prefix
    Cdf part[PPT];
    Cdf run_sum = 0;
    double sq = 0.0;                // sum of squared weights (adaptive internal resampling)
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        Cdf w = 0;
        if (alive && (FX ? lv[r] > (R)(-INFINITY) : above_neg_inf((double)lv[r]))) {
            if constexpr (!FX) w = exp_tab(lv[r] - mx);
            else w = __float2uint_rn(__expf(lv[r] - mx) * p.cdf_scale);
        }
        run_sum += w;
        part[r] = run_sum;
        if (air) sq += (double)w * (double)w;
    }
    if (air) sq = warp_sum(sq);
    // island-wide exclusive offset of this thread
    Cdf incl = warp_incl_scan(run_sum, lane);
    Cdf excl = incl - run_sum;
    if (nwi > 1) {
        if (lane == 31) red[wi] = incl;
        if (air && lane == 0) sqr[wi] = sq;
        named_sync(1 + g, tpi);
        Cdf off = 0;
        for (int w = 0; w < wi; ++w) off += red[w];
        excl += off;
        if (air) {
            sq = 0.0;
            for (int w = 0; w < nwi; ++w) sq += sqr[w];
        }
    }
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int i = li * PPT + r;
        if (i < M) {
            cdf[eyt ? eyt_ix(i) : cdf_ix(i)] = excl + part[r];
#pragma unroll
            for (int d = 0; d < DX; ++d)
                if (d < dx) xs[(size_t)d * M + i] = xv[r][d];
        }
    }
    if (nwi > 1) named_sync(1 + g, tpi);    // an island of one warp needs only the warp
    else __syncwarp();
    const Cdf total = cdf[eyt ? 0 : cdf_ix(M - 1)];

    // multinomial draws: ancestor of draw j = first i with C_i > u_j C_{M-1}.
    // Fixed-depth branchless lower bound, the thread's draws advanced together.
    int* ires_out = (REC && p.ires[t & 1] != nullptr) ? p.ires[t & 1] + (size_t)c * N + (size_t)k * M : nullptr;
    Cdf target[PPT];
    int base[PPT];
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        base[r] = 0;
        if constexpr (!FX) target[r] = unif_f64(wres[r]) * total;
        else target[r] = __umulhi(wres[r], total);       // floor(w total / 2^32) < total
    }
    // adaptive internal resampling: the island resamples only when the ESS of its
    // weights, total^2 / sum w^2, is below tau_int M (the same for every thread of it)
    const bool resample = !(air && alive) || ((double)total * (double)total / sq < p.tau_int * (double)M);
    if (resample && eyt) {
        int node[PPT];
#pragma unroll
        for (int r = 0; r < PPT; ++r) node[r] = 1;
        if constexpr (!FX) {
            // FP64: non-negative doubles compared as their bit patterns (integer pipe)
            const long long* cdfb = reinterpret_cast<const long long*>(cdf);
            long long tb[PPT];
#pragma unroll
            for (int r = 0; r < PPT; ++r) tb[r] = __double_as_longlong(target[r]);
            for (int l = 0; l < lgM; ++l) {
#pragma unroll
                for (int r = 0; r < PPT; ++r) node[r] = 2 * node[r] + (cdfb[node[r]] <= tb[r] ? 1 : 0);
            }
        } else if constexpr (MC > 0 && TPI == 32) {
            // one warp an island (every lane holds particles, and `resample` is the island's,
            // so the whole warp is here): the tree's top five levels, nodes 1 .. 31, from the
            // lanes' registers by shuffles (lane 0 holds the total, which no probe reads), the
            // rest from shared memory
            const Cdf top = cdf[lane];
            int l = 0;
            for (; l < 5 && l < lgM; ++l) {
#pragma unroll
                for (int r = 0; r < PPT; ++r)
                    node[r] = 2 * node[r] + (__shfl_sync(0xffffffffu, top, node[r]) <= target[r] ? 1 : 0);
            }
            for (; l < lgM; ++l) {
#pragma unroll
                for (int r = 0; r < PPT; ++r) node[r] = 2 * node[r] + (cdf[node[r]] <= target[r] ? 1 : 0);
            }
        } else {
            for (int l = 0; l < lgM; ++l) {
#pragma unroll
                for (int r = 0; r < PPT; ++r) node[r] = 2 * node[r] + (cdf[node[r]] <= target[r] ? 1 : 0);
            }
        }
#pragma unroll
        for (int r = 0; r < PPT; ++r) base[r] = node[r] - M;
    } else if (resample) {
        if constexpr (!FX) {
            // FP64: the CDF and the targets are non-negative doubles, whose order is the
            // order of their bit patterns as 64-bit integers: the same decisions, compared
            // on the integer pipe instead of the FP64 pipe
            const long long* cdfb = reinterpret_cast<const long long*>(cdf);
            long long tb[PPT];
#pragma unroll
            for (int r = 0; r < PPT; ++r) tb[r] = __double_as_longlong(target[r]);
            for (int n = M; n > 1;) {
                const int half = n >> 1;
#pragma unroll
                for (int r = 0; r < PPT; ++r) {
                    const long long v = cdfb[cdf_ix(base[r] + half - 1)];
                    base[r] = (v > tb[r]) ? base[r] : base[r] + half;
                }
                n -= half;
            }
        } else {
            for (int n = M; n > 1;) {
                const int half = n >> 1;
#pragma unroll
                for (int r = 0; r < PPT; ++r) {
                    const Cdf v = cdf[cdf_ix(base[r] + half - 1)];
                    base[r] = (v > target[r]) ? base[r] : base[r] + half;
                }
                n -= half;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < PPT; ++r) base[r] = li * PPT + r;
    }
    if (air) {                      // the particles' log(M omega) after this step
        R* Lc = reinterpret_cast<R*>(p.lom[t & 1]) + (size_t)c * N + (size_t)k * M;
        // a kept particle: log(M w_i / total), w_i = exp(lv_i - max) (total in the CDF's scale)
        const R lnorm = resample ? (R)0
                                 : (R)(log((double)M) - log((double)total) + (FX ? log((double)p.cdf_scale) : 0.0));
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int i = li * PPT + r;
            if (i < M) Lc[i] = resample ? (R)0 : lv[r] - mx + lnorm;
        }
    }
    R f1[DX], f2[DX];          // output measure at s = 1: the resampled particles
#pragma unroll
    for (int d = 0; d < DX; ++d) {
        f1[d] = (R)0;
        f2[d] = (R)0;
    }
    if (vec) {
        if (li * PPT < M) {
#pragma unroll
            for (int d = 0; d < DX; ++d) {
                if (d < dx) {
                    R v[PPT];
#pragma unroll
                    for (int r = 0; r < PPT; ++r) v[r] = xs[(size_t)d * M + (alive ? base[r] : li * PPT + r)];
                    store_run<R, PPT>(&Xc[((size_t)c * dx + d) * N + (size_t)k * M + li * PPT], v);
                    if (REC && p.fmom) {
#pragma unroll
                        for (int r = 0; r < PPT; ++r) {
                            f1[d] += v[r];
                            f2[d] += v[r] * v[r];
                        }
                    }
                }
            }
            if (ires_out) {
#pragma unroll
                for (int r = 0; r < PPT; ++r) ires_out[li * PPT + r] = alive ? base[r] : li * PPT + r;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int j = li * PPT + r;
            if (j < M) {
                const int a = alive ? base[r] : j;
#pragma unroll
                for (int d = 0; d < DX; ++d) {
                    if (d < dx) {
                        const R v = xs[(size_t)d * M + a];
                        Xc[((size_t)c * dx + d) * N + (size_t)k * M + j] = v;
                        if (REC && p.fmom) {
                            f1[d] += v;
                            f2[d] += v * v;
                        }
                    }
                }
                if (ires_out) ires_out[j] = a;
            }
        }
    }
    if (REC && p.fmom) moment_sums<R, DX>(p, c, t, k, wi, lane, dx, 1, f1, f2);

    // island weight W^k_{t,1} = W^k_{t,0} exp(max) (sum_i w_i) / M, extended range
    if (li == 0) {
        XW w{0ull, 0};
        const u64 wb0 = own_w[g];
        if (alive && wb0 != 0ull) {
            if constexpr (!FX) {
                double mxd = fmin(fmax((double)mx, -1.0e7), 1.0e7);
                const double n = floor(mxd * 1.4426950408889634);
                // two-constant reduction of mxd - n ln 2 (Cody and Waite, 1980)
                double f = fma(-n, 0.6931471805599453, mxd);
                f = fma(-n, 2.3190468138462996e-17, f);
                w = xw_from_double(exp(f) * ((double)total * p.inv_M) * __longlong_as_double((long long)wb0),
                                   own_we[g] + (int)n);
            } else {
                // exp(max) = 2^n e^f in float; the mantissa products in 64-bit integers:
                // W' = wm 2^(e-64) * ef24 2^(efe-23) * total 2^-cdf_bits * 2^n   (1/M left out)
                const float mxf = fminf(fmaxf(mx, -1.0e7f), 1.0e7f);
                const float n = floorf(mxf * 1.44269504f);
                float f = fmaf(-n, 0.693145752f, mxf);
                f = fmaf(-n, 1.42860677e-06f, f);
                const unsigned efb = __float_as_uint(__expf(f));
                const unsigned ef24 = (efb & 0x7fffffu) | 0x800000u;
                const int efe = (int)((efb >> 23) & 0xff) - 127;    // 0, or +-1 at the ends of [0, ln 2)
                const u64 p1 = __umul64hi(wb0, (u64)ef24 << 40);     // = wm ef24 2^-24
                const int l1 = __clzll(p1);
                const u64 q1 = p1 << l1;
                const int e1 = own_we[g] + 1 - l1 + efe;
                const int lt = __clzll((u64)total);
                const u64 p2 = __umul64hi(q1, (u64)total << lt);     // = q1 total 2^(lt-64)
                const int l2 = __clzll(p2);
                w.bits = p2 << l2;
                w.e = e1 + 64 - lt - l2 + (int)n - p.cdf_bits;
            }
        }
        new_w[g] = w.bits;
        new_we[g] = w.e;
        if (REC && p.fmom) {        // the output measures' island weights W_{t,0}, W_{t,1}
            double* fw = p.fw + (((size_t)c * p.T + (t - 1)) * p.m + k) * 2;
            fw[0] = xw_log<FX>(own_w[g], own_we[g]);
            fw[1] = xw_log<FX>(w.bits, w.e);
        }
        if (REC && p.grad) {        // log W^k_{t,1} (the FP32-mixed weights leave out M^-t)
            p.logw[((size_t)c * p.T + (t - 1)) * p.m + k] = xw_log<FX>(w.bits, w.e);
        }
    }
    __syncthreads();

    // ---- 4. the CTA's record of step t (the cascade reads it) ----
    if (tid < 32) publish_record<FX>(p, c, t, jo, new_w, new_we);
}

// ---------------------------------------------------------------------------
// Grid barrier of the cooperative persistent kernel (generation counter).  The
// wait is bounded: after 1 s (or kSpinLimit polls) the CTA sets the error word
// and every CTA leaves the time loop at its next barrier.  bar[0] counts
// arrivals, bar[1] is the generation; both and *err are zeroed by the prologue.
// ---------------------------------------------------------------------------
static __device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

static __device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

static __device__ bool grid_barrier(unsigned* bar, unsigned* err)
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
                ++it;
                if (it > kSpinLimit || ((it & 255u) == 0u && global_ns() - t0 > kWaitNs)) {
                    atomicExch(err, 1u);
                    ok = 0;
                    break;
                }
                if (it > 64u) __nanosleep(64);
            }
        }
        __threadfence();
        if (ld_acquire_gpu(err) != 0u) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// REC = false: a leaner instantiation for passes that record no lineage and
// keep nothing for the gradient (shorter instruction stream).  LV: 1 fused
// steps, 2 split steps, 0 either (and the recording passes); 3 fused steps
// with up to 128 registers a thread instead of 64 (no spills, half the resident
// CTAs: for grids that are one wave either way)
template <typename R, int MODEL, int DX, int PPT, bool REC, int LV, int MC = 0>
__global__ void __launch_bounds__(kMaxThreads, LV == 3 ? 1 : kMinCtasPerSm) airpf_step_kernel(StepParams p, int t)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int cpf = p.P;                       // CTAs per filter (a power of 2)
    int c, k0;
    if (p.ncta > 0) {                          // a range of each filter's CTAs (sharded passes)
        c = blockIdx.x >> p.lg_ncta;
        k0 = (p.cta0 + (int)(blockIdx.x - (c << p.lg_ncta))) * p.G;
    } else {
        c = blockIdx.x >> (p.S - p.g);
        k0 = (blockIdx.x - c * cpf) * p.G;
    }
    if (p.active != nullptr && p.active[c] == 0) return;   // uniform over the CTA
    step_body<R, MODEL, DX, PPT, REC, LV, MC>(p, t, c, k0, smem, p.pdl != 0);
}

// The cascade of step t: one CTA per filter.
template <typename R>
__global__ void __launch_bounds__(kCascadeThreads) airpf_cascade_kernel(StepParams p, int t)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int c = blockIdx.x;
    if (p.active != nullptr && p.active[c] == 0) return;
    if (p.pdl) {                  // the records are the island-step kernel's output
        dependency_wait();
        allow_dependents();
    }
    const RunParams run = *p.run;
    const Stream st{p.seed_lo, p.seed_hi, run.iter, (run.chain0 + (uint32_t)c) << 8};
    cascade_all<sizeof(R) == 4>(p, c, t, st, reinterpret_cast<double*>(smem));
}

// The split steps' cascade of step t: CTA j reduces group j mod NG of filter
// j / NG; the last of a filter's CTAs to finish its group (a ticket) runs the top.
// Publication: every thread's stores, a CTA barrier, one thread's device-scope fence
// and ticket; the last arrival fences before it reads.  The ticket wraps to zero by
// itself (atomicInc) and the prologue clears it.
template <typename R, int FIX = 0>
__global__ void __launch_bounds__(512) airpf_group_cascade_kernel(StepParams p, int t)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int last;
    const SplitShape<FIX> sp(p);
    const int c = blockIdx.x >> (sp.S - sp.g - sp.gs), grp = blockIdx.x & (sp.NG - 1);
    if (p.active != nullptr && p.active[c] == 0) return;
    if (p.pdl) {                  // the records are the island-step kernel's output
        dependency_wait();
        allow_dependents();
    }
    group_cascade<sizeof(R) == 4, FIX>(p, c, t, grp, smem);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicInc(&p.tick[c], (unsigned)(sp.NG - 1)) == (unsigned)(sp.NG - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    top_cascade<sizeof(R) == 4, FIX>(p, c, t, smem);
}

// All T+1 steps in one launch.  GRID: the filter spans several co-resident CTAs
// (cooperative launch); a step's records are published before a grid barrier,
// the filter's first CTA runs the cascade, and a second barrier releases the
// next step.  Otherwise one CTA holds a whole filter and runs its cascade
// itself between block barriers.
template <typename R, int MODEL, int DX, int PPT, bool GRID>
__global__ void __launch_bounds__(GRID ? kMaxThreads : kMaxCtaThreads, kMinCtasPerSm) airpf_persistent_kernel(StepParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int cpf = p.P;
    const int c = blockIdx.x >> (p.S - p.g);
    const int k0 = (blockIdx.x - c * cpf) * p.G;
    const bool act = (p.active == nullptr || p.active[c] != 0);
    if (!GRID && !act) return;
    // fault-injection hook: CTA 0 leaves before the first barrier, so the other
    // CTAs' bounded wait runs out (tests the timeout path)
    if (GRID && p.inject_stall && blockIdx.x == 0) return;
    const RunParams run = *p.run;
    const Stream st{p.seed_lo, p.seed_hi, run.iter, (run.chain0 + (uint32_t)c) << 8};
    for (int t = 1; t <= p.T + 1; ++t) {
        if (act) step_body<R, MODEL, DX, PPT>(p, t, c, k0, smem);
        if (t > p.T) break;
        if (GRID) {
            if (!grid_barrier(p.bar, p.err)) return;
            if (act && k0 == 0) cascade_all<sizeof(R) == 4>(p, c, t, st, reinterpret_cast<double*>(smem));
            if (!grid_barrier(p.bar, p.err)) return;
        } else {
            __syncthreads();
            cascade_all<sizeof(R) == 4>(p, c, t, st, reinterpret_cast<double*>(smem));
            __syncthreads();
        }
    }
}

// Launch with the programmatic-stream-serialization attribute: the kernel may
// begin while the previous kernel of the stream finishes, and waits for it with
// griddepcontrol.wait before touching that kernel's output.
template <typename K>
static cudaError_t launch_dependent(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                                    const StepParams& p, int t)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, p, t);
}

// The lean step kernels also come with the island size fixed at compile time, for
// islands of 4 particles a thread: M = 256 (64 threads an island) in both precisions and
// every lean launch form; in FP32 also M = 128, 512 and 1024 (32, 128 and 256 threads)
// for the fused (64-register) and split forms.  The FP64 steps are bound by the FP64
// pipe, which the compile-time size does not relieve.
constexpr int kFixedM = 256, kFixedPpt = 4;
__host__ inline bool fixed_island(const StepParams& p, int M, int ppt = kFixedPpt)
{
    return p.M == M && p.tpi == (M / ppt < 32 ? 32 : M / ppt);
}
__host__ inline bool fixed_island(const StepParams& p) { return fixed_island(p, kFixedM); }

// apply(kernel) to the fixed-size kernel of launch form LV for this context's island
// size, if there is one (returns false otherwise)
template <typename R, int MODEL, int DX, int PPT, int LV, typename F>
__host__ bool with_fixed_kernel(const StepParams& p, F&& apply)
{
    if constexpr (PPT == 8) {        // one warp an island of 256 (two and four warps for 512, 1024)
        if (fixed_island(p, 256, 8)) return apply(airpf_step_kernel<R, MODEL, DX, PPT, false, LV, 256>), true;
        if constexpr (LV != 3) {
            if (fixed_island(p, 512, 8)) return apply(airpf_step_kernel<R, MODEL, DX, PPT, false, LV, 512>), true;
            if (fixed_island(p, 1024, 8)) return apply(airpf_step_kernel<R, MODEL, DX, PPT, false, LV, 1024>), true;
        }
        return false;
    } else if constexpr (PPT != kFixedPpt) {
        return false;
    } else {
        if (fixed_island(p, 256)) return apply(airpf_step_kernel<R, MODEL, DX, PPT, false, LV, 256>), true;
        if constexpr (sizeof(R) == 4 && LV != 3) {
            if (fixed_island(p, 128)) return apply(airpf_step_kernel<R, MODEL, DX, PPT, false, LV, 128>), true;
            if (fixed_island(p, 512)) return apply(airpf_step_kernel<R, MODEL, DX, PPT, false, LV, 512>), true;
            if (fixed_island(p, 1024)) return apply(airpf_step_kernel<R, MODEL, DX, PPT, false, LV, 1024>), true;
        }
        return false;
    }
}

template <typename R, int MODEL, int DX, int PPT>
static cudaError_t launch_typed(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    const size_t smem = step_smem_bytes(p);
    const int block = p.G * p.tpi;
    const int grid = p.B * (p.ncta > 0 ? p.ncta : p.m / p.G);
    const int want = smem > 48 * 1024 ? (int)smem : 48 * 1024;
    if (op == OP_PREPARE) {
        // opt in to more than 48 KB of dynamic shared memory (outside any capture)
        cudaError_t e = cudaFuncSetAttribute(airpf_step_kernel<R, MODEL, DX, PPT, true, 0>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(airpf_step_kernel<R, MODEL, DX, PPT, false, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(airpf_step_kernel<R, MODEL, DX, PPT, false, 2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(airpf_step_kernel<R, MODEL, DX, PPT, false, 3>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        auto set_smem = [&](auto kernel) {
            if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        };
        with_fixed_kernel<R, MODEL, DX, PPT, 1>(p, set_smem);
        with_fixed_kernel<R, MODEL, DX, PPT, 2>(p, set_smem);
        with_fixed_kernel<R, MODEL, DX, PPT, 3>(p, set_smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(airpf_persistent_kernel<R, MODEL, DX, PPT, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(airpf_persistent_kernel<R, MODEL, DX, PPT, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        // (split steps use the group cascade kernel, whose shared memory stays small)
        const size_t cs = cascade_smem_bytes(p);
        if (e == cudaSuccess && !p.split && cs > 48 * 1024)
            e = cudaFuncSetAttribute(airpf_cascade_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs);
        return e;
    }
    if (op == OP_FITS) {
        // can every CTA of the grid-persistent kernel be resident at once?
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, airpf_persistent_kernel<R, MODEL, DX, PPT, true>,
                                                              block, smem);
        *fits = (e == cudaSuccess && block <= kMaxThreads && (long long)per_sm * sms >= grid) ? 1 : 0;
        return e;
    }
    if (op == OP_WIDE_FITS) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        bool fixed_done = false;
        if (e == cudaSuccess)
            fixed_done = with_fixed_kernel<R, MODEL, DX, PPT, 3>(p, [&](auto kernel) {
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
            });
        if (e == cudaSuccess && !fixed_done)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, airpf_step_kernel<R, MODEL, DX, PPT, false, 3>,
                                                              block, smem);
        *fits = (e == cudaSuccess && (long long)per_sm * sms >= grid) ? 1 : 0;
        return e;
    }
    if (op == OP_PERSIST_GRID) {
        StepParams q = p;
        void* args[] = {&q};
        return cudaLaunchCooperativeKernel((const void*)airpf_persistent_kernel<R, MODEL, DX, PPT, true>, dim3(grid),
                                           dim3(block), args, smem, stream);
    }
    if (op == OP_PERSIST_CTA) {
        airpf_persistent_kernel<R, MODEL, DX, PPT, false><<<grid, block, smem, stream>>>(p);
        return cudaGetLastError();
    }
    if (op == OP_CASCADE && p.split) {
        // CTAs of max(32, GS, NG) threads: one record a thread in both parts
        const size_t cs = split_cascade_smem_bytes(p);
        int tg = (1 << p.gs) > p.NG ? (1 << p.gs) : p.NG;
        if (tg < 32) tg = 32;
        if (split_shape_fixed(p, tg)) {
            if (p.pdl)
                return launch_dependent(airpf_group_cascade_kernel<R, 1>, dim3(p.NG * p.B), dim3(tg), cs, stream, p, t);
            airpf_group_cascade_kernel<R, 1><<<p.NG * p.B, tg, cs, stream>>>(p, t);
            return cudaGetLastError();
        }
        if (p.pdl) return launch_dependent(airpf_group_cascade_kernel<R>, dim3(p.NG * p.B), dim3(tg), cs, stream, p, t);
        airpf_group_cascade_kernel<R><<<p.NG * p.B, tg, cs, stream>>>(p, t);
        return cudaGetLastError();
    }
    if (op == OP_CASCADE) {
        const size_t cs = cascade_smem_bytes(p);
        if (p.pdl) return launch_dependent(airpf_cascade_kernel<R>, dim3(p.B), dim3(kCascadeThreads), cs, stream, p, t);
        airpf_cascade_kernel<R><<<p.B, kCascadeThreads, cs, stream>>>(p, t);
        return cudaGetLastError();
    }
    if (t == 0) {
        const int n = p.B > p.T ? p.B : p.T;
        airpf_prologue_kernel<R, MODEL><<<(n + 127) / 128, 128, 0, stream>>>(p);
        return cudaGetLastError();
    }
    // step 1 follows the prologue in plain stream order; later steps may start
    // launching while the previous cascade runs (programmatic dependent launch)
    // the lean instantiations (no recording, one launch form) where they apply
    const bool rec = p.anc != nullptr || p.grad != 0 || p.ires[0] != nullptr || p.fmom != 0 || p.air != 0;
    auto go = [&](auto kernel) -> cudaError_t {
        if (p.pdl && t >= 2) return launch_dependent(kernel, dim3(grid), dim3(block), smem, stream, p, t);
        kernel<<<grid, block, smem, stream>>>(p, t);
        return cudaGetLastError();
    };
    if (!rec) {                               // the compile-time island size, where there is one
        cudaError_t r = cudaSuccess;
        auto run = [&](auto kernel) { r = go(kernel); };
        if (p.fused && p.wide && with_fixed_kernel<R, MODEL, DX, PPT, 3>(p, run)) return r;
        if (p.fused && !p.wide && with_fixed_kernel<R, MODEL, DX, PPT, 1>(p, run)) return r;
        if (p.split && with_fixed_kernel<R, MODEL, DX, PPT, 2>(p, run)) return r;
    }
    if (!rec && p.fused)
        return p.wide ? go(airpf_step_kernel<R, MODEL, DX, PPT, false, 3>) : go(airpf_step_kernel<R, MODEL, DX, PPT, false, 1>);
    if (!rec && p.split) return go(airpf_step_kernel<R, MODEL, DX, PPT, false, 2>);
    return go(airpf_step_kernel<R, MODEL, DX, PPT, true, 0>);
}

// the kernels of one precision, model and particles-per-thread count (one
// explicit instantiation per triple in airpf_launch_inst.cu)
template <typename R, int MODEL, int PPT>
cudaError_t dispatch_inst(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    return launch_typed<R, MODEL, MODEL == LGSSM ? kMaxDx : 1, PPT>(p, t, stream, op, fits);
}

}  // namespace airpf
