// airpf_device.cuh -- device building blocks of the AIRPF hot path (sm_103a):
// the counter-based random streams and the state-space models.
//
// Random streams: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
//   key = (seed lo, seed hi), counter = (unit, t, iter, chainword | kind<<5 | sub).
// Models: Section 1.2, eq. (1) of Heine (arXiv 2312.06484); parameter layouts as
// in include/airpf.h.
#pragma once
#include <cstdint>
#include "airpf_exp_table.h"
#include "airpf_log_table.h"
#include "airpf_sincos_table.h"
#include <cmath>

namespace airpf {

enum Kind : uint32_t { KIND_INIT = 0, KIND_STEP = 1, KIND_ISLAND = 2, KIND_MH = 3 };
enum Model : int { AR1 = 0, SV = 1, NGM = 2, LGSSM = 3, TOY = 4, CP = 5 };

constexpr int kMaxDx = 8;
constexpr int kMaxDy = 8;
constexpr int kMaxTheta = kMaxDx + 2;

struct U4 {
    uint32_t x, y, z, w;
};

// Ten Philox rounds: two 32x32->64 multiplies per round (one wide multiply
// each), the Weyl key bump between rounds.
__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (uint32_t)p1;
        c2 = n2;
        c3 = (uint32_t)p0;
    }
    return U4{c0, c1, c2, c3};
}

// The identity of one filter's streams: seed key, PMMH iteration and chain.
struct Stream {
    uint32_t k0, k1, iter, chainword;   // chainword = chain << 8

    __device__ __forceinline__ U4 draw(uint32_t unit, uint32_t t, uint32_t kind, uint32_t sub) const
    {
        return philox4x32_10(unit, t, iter, chainword | (kind << 5) | sub, k0, k1);
    }
};

// (w + 1/2) 2^-32, exactly: 1 + (w + 1/2) 2^-32 assembled from its bits (w in mantissa bits
// 51..20, the half in bit 19), less 1 (exact for a value in [1, 2)); one FP64 instruction
__device__ __forceinline__ double unif_f64(uint32_t w)
{
    return __hiloint2double((int)(0x3FF00000u | (w >> 12)), (int)((w << 20) | (1u << 19))) - 1.0;
}

// x > -inf (false for NaN), decided on the bit pattern by the integer pipe
__device__ __forceinline__ bool above_neg_inf(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x7FFFFFFFFFFFFFFFull) <= 0x7FF0000000000000ull && b != 0xFFF0000000000000ull;
}

// A signed 64-bit integer in the order of the double x (not NaN): the bit pattern, with the
// magnitude bits of negative values flipped.  The map is its own inverse.
__device__ __forceinline__ long long order_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double from_order_key(long long k)
{
    return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFll));
}

// The double exponential of the FP64 path, table-driven (Tang, ACM TOMS 15(2), 1989):
// x = (256 k + j) ln 2 / 256 + r with |r| <= ln 2 / 512, exp(x) = 2^k 2^(j/256) e^r, e^r - 1
// by its Taylor polynomial through r^4 (the next term is below 0.2 ulp at |r| <= ln 2 / 512).
// At most about 1 ulp from the exact value; outside |x| <= 708 (overflow, subnormal results,
// infinities, NaN) it defers to the library function.
__device__ __forceinline__ double exp_tab(double x)
{
    // |x| <= 708 (false for NaN) on the bit pattern: 0x40862... is 708.0
    if (!(((unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull) <= 0x4086200000000000ull))
        return exp(x);
    // n = nearest integer to 256 x / ln 2, in the low bits of a sum with 1.5 2^52 (one
    // rounding, no conversion instructions)
    const double t = fma(x, kExpInvLn2xN, 0x1.8p52);
    const double dn = t - 0x1.8p52;
    const int n = __double2loint(t);
    double r = fma(-dn, kExpLn2dNHi, x);
    r = fma(-dn, kExpLn2dNLo, r);
    double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    const double p = fma(r * r, q, r);
    const double tj = __ldg(&kExp2Table[n & 255]);
    const double v = fma(tj, p, tj);
    return __longlong_as_double(__double_as_longlong(v) + ((long long)(n >> 8) << 52));
}

// The double logarithm of the FP64 path, table-driven (Tang, ACM TOMS 16(4), 1990): x = 2^e m,
// m in [1, 2), F = 1 + j/128 the nearest 128th to m, f = m - F (exact), s = f / F taken as
// f (1/F) with the reciprocal from the table, log x = e ln 2 + log F + log(1 + s) with
// log(1 + s) by its Taylor polynomial through s^7 (|s| <= 2^-8), e ln 2 + log F summed
// exactly from parts on a common grid.  At most about 1 ulp from the exact value.
// log_parts takes e and the 52 fraction bits of m.
__device__ __forceinline__ double log_parts(int e, long long mb)
{
    const double m = __longlong_as_double(mb | 0x3FF0000000000000LL);
    const int j = (int)(((mb >> 44) + 1) >> 1);                   // nearest 128th: 0 .. 128
    const double F = __longlong_as_double(0x3FF0000000000000LL + ((long long)j << 45));
    const double s = (m - F) * __ldg(&kLogInvF[j]);
    double q = fma(s, 1.0 / 7.0, -1.0 / 6.0);
    q = fma(s, q, 0.2);
    q = fma(s, q, -0.25);
    q = fma(s, q, 1.0 / 3.0);
    q = fma(s, q, -0.5);
    const double p = fma(s * s, q, s);
    const double de = (double)e;
    const double hi = fma(de, kLogLn2Hi, __ldg(&kLogFHi[j]));       // exact
    const double lo = fma(de, kLogLn2Lo, __ldg(&kLogFLo[j]));
    return hi + (lo + p);
}

// log x; zero, negative, subnormal and non-finite arguments (told apart on the bit pattern)
// defer to the library function
__device__ __forceinline__ double log_tab(double x)
{
    const long long b = __double_as_longlong(x);
    if (!(b >= 0x0010000000000000LL && b <= 0x7FEFFFFFFFFFFFFFLL)) return log(x);
    return log_parts((int)(b >> 52) - 1023, b & 0x000FFFFFFFFFFFFFLL);
}

// log of the uniform (w + 1/2) 2^-32 = v 2^-33, v = 2w + 1: the exponent and the fraction
// bits from the integer v (no conversion, no range test: the value is normal, in (0, 1));
// the same value as log_tab(unif_f64(w))
__device__ __forceinline__ double log_unif(uint32_t w)
{
    const unsigned long long v = 2ull * w + 1ull;                 // 1 .. 2^33 - 1
    const int msb = 63 - __clzll((long long)v);                   // 0 .. 32
    return log_parts(msb - 33, (long long)((v << (52 - msb)) & 0x000FFFFFFFFFFFFFull));
}

// sin(2 pi v) and cos(2 pi v), table-driven: 2 pi v = 2 pi j / 256 + x with j the nearest
// 256th and |x| <= pi / 256, the angle-addition formulas with the table's sin and cos of
// 2 pi j / 256 and Taylor polynomials of sin x through x^7 and cos x through x^6 (the next
// terms are below 1e-19).  Within a few 1e-16 of the exact values.
__device__ __forceinline__ void sincos2pi_parts(int j, double x, double* s, double* c)
{
    const double x2 = x * x;
    const double cx = fma(x2, fma(x2, fma(x2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
    const double sx = fma(x * x2, fma(x2, fma(x2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), x);
    const double sj = __ldg(&kSin256[j]), cj = __ldg(&kCos256[j]);
    *s = fma(sj, cx, cj * sx);
    *c = fma(cj, cx, -(sj * sx));
}

// v in [0, 1] (told apart on the bit pattern; other v defer to the library's sincos): the
// reduction is exact when v has at most 33 significant bits
__device__ __forceinline__ void sincos2pi_tab(double v, double* s, double* c)
{
    const long long b = __double_as_longlong(v);
    if (!(b >= 0 && b <= 0x3FF0000000000000LL)) {
        sincos(6.283185307179586 * v, s, c);
        return;
    }
    const double t = v * 256.0;
    const double tj = fma(1.0, t, 0x1.8p52);                        // nearest integer in the low bits
    const double f = t - (tj - 0x1.8p52);
    sincos2pi_parts(__double2loint(tj) & 255, f * kTwoPiDiv256, s, c);
}

// sin and cos of 2 pi (w + 1/2) 2^-32, reduced in integers: j = the nearest 256th, and
// 256 v - j = (2 (w - j 2^24) + 1) 2^-25 with the odd integer below 2^24 in magnitude
// (32-bit wrap-around gives the signed remainder for j = 256 too); the same values as
// sincos2pi_tab(unif_f64(w))
__device__ __forceinline__ void sincos2pi_unif(uint32_t w, double* s, double* c)
{
    const uint32_t j = ((w >> 23) + 1u) >> 1;                       // 0 .. 256
    const int r = (int)((w - (j << 24)) * 2u + 1u);
    sincos2pi_parts((int)(j & 255u), (double)r * (kTwoPiDiv256 * 0x1p-25), s, c);
}

// Box-Muller pair from two words: r = sqrt(-2 ln u0), angle 2 pi u1.
__device__ __forceinline__ void normal_pair(uint32_t w0, uint32_t w1, double& z0, double& z1)
{
    const double rad = sqrt(-2.0 * log_unif(w0));
    double s, c;
    sincos2pi_unif(w1, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

// float version on the SFU: cos(2 pi u) = -cos(pi (2u - 1)), same for sin.
__device__ __forceinline__ void normal_pair(uint32_t w0, uint32_t w1, float& z0, float& z1)
{
    const float u0 = fmaf((float)w0, 0x1p-32f, 0x1p-33f);
    const float r2 = fmaxf(-2.0f * __logf(u0), 1e-30f);
    const float rad = r2 * rsqrtf(r2);
    const float a = fmaf((float)w1, 0x1p-31f, 0x1p-32f) - 1.0f;
    float s, c;
    __sincosf(3.14159265358979f * a, &s, &c);
    z0 = -rad * c;
    z1 = -rad * s;
}

template <typename R> __device__ __forceinline__ R fexp(R v);
template <> __device__ __forceinline__ double fexp<double>(double v) { return exp_tab(v); }
template <> __device__ __forceinline__ float fexp<float>(float v) { return __expf(v); }
template <typename R> __device__ __forceinline__ R flog(R v);
template <> __device__ __forceinline__ double flog<double>(double v) { return log_tab(v); }
template <> __device__ __forceinline__ float flog<float>(float v) { return __logf(v); }
template <typename R> __device__ __forceinline__ R fsqrt(R v);
template <> __device__ __forceinline__ double fsqrt<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float fsqrt<float>(float v) { return sqrtf(v); }
template <typename R> __device__ __forceinline__ R fcos(R v);
template <> __device__ __forceinline__ double fcos<double>(double v) { return cos(v); }
template <> __device__ __forceinline__ float fcos<float>(float v) { return __cosf(v); }

// Per-filter model constants, computed once per CTA from theta.
template <typename R>
struct ModelPar {
    R th[kMaxTheta];
    R c0, c1, c2, c3;        // model-specific derived constants
    R drift;                 // per-step constant (NGM: 8 cos(1.2 t))
};

template <typename R, int MODEL>
__device__ __forceinline__ void model_setup(ModelPar<R>& p, const double* theta, int dx, int dy)
{
    const int nth = (MODEL == LGSSM) ? dx + 2 : (MODEL == AR1 ? 4 : (MODEL == TOY ? 2 : 3));
#pragma unroll
    for (int i = 0; i < kMaxTheta; ++i) p.th[i] = (i < nth) ? (R)theta[i] : (R)0;
    if (MODEL == AR1) {            // a, sv, sw, s0
        p.c0 = (R)(-0.9189385332046727 - log(theta[2]));   // -log sqrt(2 pi) - log sw
        p.c1 = (R)(1.0 / theta[2]);
    } else if (MODEL == SV) {      // mu, phi, sigma
        p.c0 = (R)(theta[2] / sqrt(1.0 - theta[1] * theta[1]));   // stationary sd
        p.c1 = (R)(-0.9189385332046727);
    } else if (MODEL == NGM) {     // q, r, p0
        p.c0 = (R)sqrt(theta[0]);
        p.c1 = (R)(-0.5 * log(2.0 * 3.141592653589793 * theta[1]));
        p.c2 = (R)(0.5 / theta[1]);
        p.c3 = (R)sqrt(theta[2]);
    } else if (MODEL == TOY) {     // stay, correct
        p.c0 = (R)(1.0 - theta[0]);
        p.c1 = (R)log(theta[1]);
        p.c2 = (R)log(1.0 - theta[1]);
    } else if (MODEL == CP) {      // p, alpha, beta: the gamma draws' d and c for alpha and beta
        const double aa = theta[1] < 1.0 ? theta[1] + 1.0 : theta[1];
        const double bb = theta[2] < 1.0 ? theta[2] + 1.0 : theta[2];
        const double da = aa - 1.0 / 3.0, db = bb - 1.0 / 3.0;
        p.c0 = (R)da;
        p.c1 = (R)(1.0 / sqrt(9.0 * da));
        p.c2 = (R)db;
        p.c3 = (R)(1.0 / sqrt(9.0 * db));
    } else {                       // LGSSM: sqrt(q), 1/(2r), -dy/2 log(2 pi r)
        const double r = exp(theta[dx + 1]);
        p.c0 = (R)sqrt(exp(theta[dx]));
        p.c1 = (R)(0.5 / r);
        p.c2 = (R)(-0.5 * dy * log(2.0 * 3.141592653589793 * r));
    }
    p.drift = (R)0;
}

// per-step constants of the transition at time t
template <typename R, int MODEL>
__device__ __forceinline__ void model_step_setup(ModelPar<R>& p, int t)
{
    if (MODEL == NGM) p.drift = (R)(8.0 * cos(1.2 * (double)t));
}

// Normals z[0..n-1] of (kind, unit, t): pair b gives z[2b], z[2b+1].  Also
// returns word 0 and word 2 of sub-block 0.  A transition with one normal
// shares its block with the neighbouring unit: units 2j and 2j+1 both draw
// block j of counter unit j; the even unit takes the cosine normal and words 0
// and 2, the odd unit the sine normal and words 1 and 3.
template <typename R, int NZ>
__device__ __forceinline__ void stream_normals(const Stream& st, uint32_t kind, uint32_t unit,
                                               uint32_t t, int n, R* z, uint32_t& w0, uint32_t& w2)
{
    if (NZ >= 1 && kind == KIND_STEP && n == 1) {
        const U4 b = st.draw(unit >> 1, t, kind, 0);
        R a, c;
        normal_pair(b.x, b.y, a, c);
        const bool odd = (unit & 1u) != 0u;
        z[0] = odd ? c : a;
        w0 = odd ? b.y : b.x;
        w2 = odd ? b.w : b.z;
        return;
    }
    const U4 b0 = st.draw(unit, t, kind, 0);
    w0 = b0.x;
    w2 = b0.z;
    if (NZ == 0) return;
    if (NZ == 1) {
        R z1;
        normal_pair(b0.x, b0.y, z[0], z1);
        return;
    }
    normal_pair(b0.x, b0.y, z[0], z[1]);
#pragma unroll
    for (int b = 1; b < (NZ + 1) / 2; ++b) {
        if (2 * b < n) {
            const U4 bb = st.draw(unit, t, kind, (uint32_t)b);
            R a, c;
            normal_pair(bb.x, bb.y, a, c);
            z[2 * b] = a;
            if (2 * b + 1 < NZ) z[2 * b + 1] = c;
        }
    }
}

// a / b: IEEE in double; the SFU reciprocal and a multiply in float (within 2 ulp for
// |b| < 2^126)
template <typename R> __device__ __forceinline__ R fdiv(R a, R b);
template <> __device__ __forceinline__ double fdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }

// x^2 / 20 (the growth model's observation mean) as two rounded products, x x and then 1/20
// rounded to R, not contracted into the subtraction that follows: within about 1 ulp of the
// quotient, at the cost of two multiplications instead of a division
template <typename R> __device__ __forceinline__ R ngm_obs_mean(R x);
template <> __device__ __forceinline__ double ngm_obs_mean<double>(double x) { return __dmul_rn(__dmul_rn(x, x), 0.05); }
template <> __device__ __forceinline__ float ngm_obs_mean<float>(float x) { return __fmul_rn(__fmul_rn(x, x), 0.05f); }

template <typename R> __device__ __forceinline__ R unif_r(uint32_t w);
template <> __device__ __forceinline__ double unif_r<double>(uint32_t w) { return unif_f64(w); }
template <> __device__ __forceinline__ float unif_r<float>(uint32_t w) { return fmaf((float)w, 0x1p-32f, 0x1p-33f); }

// Gamma(a, 1) by the method of Marsaglia and Tsang (ACM TOMS 26(3), 2000), with
// d = a' - 1/3 and c = 1/sqrt(9 d), a' = a (a >= 1, else a + 1): an attempt
// takes a normal z and a uniform u, v = (1 + c z)^3, and accepts d v if
// 1 + c z > 0 and log u < z^2/2 + d - d v + d log v.  Attempt j reads
// sub-block first + 2j of the stream (cosine normal of words 0 and 1, uniform
// of word 2); after kGammaTries rejections the draw is d.  For a < 1 the draw
// is scaled by U^(1/a), U from the word wboost.
constexpr int kGammaTries = 15;

template <typename R>
__device__ R gamma_draw(const Stream& st, uint32_t kind, uint32_t unit, uint32_t t, uint32_t first, R a, R d,
                        R c, uint32_t wboost)
{
    R g = d;
    for (int j = 0; j < kGammaTries; ++j) {
        const U4 b = st.draw(unit, t, kind, first + 2u * (uint32_t)j);
        R z, z1;
        normal_pair(b.x, b.y, z, z1);
        const R x1 = (R)1 + c * z;
        if (x1 <= (R)0) continue;
        const R v = x1 * x1 * x1;
        if (flog<R>(unif_r<R>(b.z)) < (R)0.5 * z * z + d - d * v + d * flog<R>(v)) {
            g = d * v;
            break;
        }
    }
    if (a < (R)1) g *= fexp<R>(flog<R>(unif_r<R>(wboost)) / a);
    return g;
}

// Beta(alpha, beta) = X / (X + Y): X ~ Gamma(alpha) from sub-blocks 1, 3, 5, ...,
// Y ~ Gamma(beta) from 2, 4, 6, ...; b0 is sub-block 0, whose words 3 and 1 are
// the two boosts.
template <typename R>
__device__ R beta_draw(const ModelPar<R>& p, const Stream& st, uint32_t kind, uint32_t unit, uint32_t t, const U4& b0)
{
    const R x = gamma_draw<R>(st, kind, unit, t, 1u, p.th[1], p.c0, p.c1, b0.w);
    const R y = gamma_draw<R>(st, kind, unit, t, 2u, p.th[2], p.c2, p.c3, b0.y);
    return x / (x + y);
}

// x_0 ~ pi_0
template <typename R, int MODEL, int DX>
__device__ __forceinline__ void model_prior(const ModelPar<R>& p, const Stream& st, uint32_t unit,
                                            int dx, R* x)
{
    if (MODEL == CP) {            // Beta(alpha, beta)
        x[0] = beta_draw<R>(p, st, KIND_INIT, unit, 0u, st.draw(unit, 0u, KIND_INIT, 0));
        return;
    }
    R z[DX > 1 ? DX : 1];
    uint32_t w0, w2;
    stream_normals<R, (MODEL == TOY) ? 0 : DX>(st, KIND_INIT, unit, 0u, dx, z, w0, w2);
    if (MODEL == AR1) x[0] = p.th[3] * z[0];
    if (MODEL == SV) x[0] = p.th[0] + p.c0 * z[0];
    if (MODEL == NGM) x[0] = p.c3 * z[0];
    if (MODEL == TOY) x[0] = (unif_f64(w0) < 0.5) ? (R)0 : (R)1;
    if (MODEL == LGSSM) {
#pragma unroll
        for (int d = 0; d < DX; ++d) if (d < dx) x[d] = z[d];
    }
}

// x_t = K_t(x_{t-1}, .) given the step's normals z (and word w0 for the binary
// model).  A (LGSSM) is row-major dx*dx in shared memory, diagonal from theta.
template <typename R, int MODEL, int DX>
__device__ __forceinline__ void model_transition(const ModelPar<R>& p, int dx, const R* xp, R* x, const R* A,
                                                 const R* z, uint32_t w0)
{
    if (MODEL == AR1) x[0] = p.th[0] * xp[0] + p.th[1] * z[0];
    if (MODEL == SV) x[0] = p.th[0] + p.th[1] * (xp[0] - p.th[0]) + p.th[2] * z[0];
    if (MODEL == NGM) {
        const R v = xp[0];
        x[0] = (R)0.5 * v + fdiv<R>((R)25 * v, (R)1 + v * v) + p.drift + p.c0 * z[0];
    }
    if (MODEL == TOY) x[0] = (unif_f64(w0) < (double)p.c0) ? (R)1 - xp[0] : xp[0];
    if (MODEL == CP) x[0] = (unif_f64(w0) < (double)p.th[0]) ? z[0] : xp[0];   // z: the jump's Beta draw
    if (MODEL == LGSSM) {
#pragma unroll
        for (int r = 0; r < DX; ++r) {
            if (r < dx) {
                R acc = 0;
#pragma unroll
                for (int c = 0; c < DX; ++c)
                    if (c < dx) acc += ((r == c) ? p.th[r] : A[r * dx + c]) * xp[c];
                x[r] = acc + p.c0 * z[r];
            }
        }
    }
}

// The step's random numbers of one unit: the transition normals z, word 0
// (binary model) and word 2 (internal-resampling draw) of sub-block 0.
// The change-point model draws its jump uniform (word 0) and, when it jumps
// (u < p), the Beta draw into z[0].
template <typename R, int MODEL, int DX>
__device__ __forceinline__ void model_step_noise(const ModelPar<R>& p, const Stream& st, uint32_t unit, uint32_t t,
                                                 int dx, R* z, uint32_t& w0, uint32_t& w2)
{
    if (MODEL == CP) {
        const U4 b = st.draw(unit, t, KIND_STEP, 0);
        w0 = b.x;
        w2 = b.z;
        z[0] = (R)0;
        if (unif_f64(b.x) < (double)p.th[0]) z[0] = beta_draw<R>(p, st, KIND_STEP, unit, t, b);
        return;
    }
    stream_normals<R, (MODEL == TOY) ? 0 : DX>(st, KIND_STEP, unit, t, dx, z, w0, w2);
}

// The step's random numbers of units u and u+1 (u even) of a one-normal model
// from their shared block (the rule of stream_normals, one draw for both).
template <typename R>
__device__ __forceinline__ void step_noise_pair(const Stream& st, uint32_t u_even, uint32_t t, R& za, R& zb,
                                                uint32_t& w0a, uint32_t& w0b, uint32_t& w2a, uint32_t& w2b)
{
    const U4 b = st.draw(u_even >> 1, t, KIND_STEP, 0);
    normal_pair(b.x, b.y, za, zb);
    w0a = b.x;
    w0b = b.y;
    w2a = b.z;
    w2b = b.w;
}

// x_t ~ K_t(x_{t-1}, .); returns the internal-resampling word of the unit.
template <typename R, int MODEL, int DX>
__device__ __forceinline__ uint32_t model_step(const ModelPar<R>& p, const Stream& st, uint32_t unit,
                                               uint32_t t, int dx, const R* xp, R* x, const R* A)
{
    R z[DX > 1 ? DX : 1];
    uint32_t w0, w2;
    model_step_noise<R, MODEL, DX>(p, st, unit, t, dx, z, w0, w2);
    model_transition<R, MODEL, DX>(p, dx, xp, x, A, z, w0);
    return w2;
}

// log g_t(y_t | x); NaN counts as -inf (weight zero).
template <typename R, int MODEL, int DX>
__device__ __forceinline__ R model_logg(const ModelPar<R>& p, const R* y, int dx, int dy, const R* x,
                                        const R* Cm)
{
    R l;
    if (MODEL == AR1) {
        const R e = (y[0] - x[0]) * p.c1;
        l = p.c0 - (R)0.5 * e * e;
    } else if (MODEL == SV) {
        l = p.c1 - (R)0.5 * x[0] - (R)0.5 * y[0] * y[0] * fexp<R>(-x[0]);
    } else if (MODEL == NGM) {
        const R e = y[0] - ngm_obs_mean<R>(x[0]);
        l = p.c1 - e * e * p.c2;
    } else if (MODEL == TOY) {
        l = (y[0] == x[0]) ? p.c1 : p.c2;
    } else if (MODEL == CP) {      // y = (k, n, log C(n, k)): k ~ Binomial(n, x)
        const R k = y[0], nk = y[1] - y[0];
        l = y[2];
        if (k > (R)0) l += k * flog<R>(x[0]);
        if (nk > (R)0) l += nk * log1p(-x[0]);
    } else {
        R ss = 0;
#pragma unroll
        for (int o = 0; o < kMaxDy; ++o) {
            if (o < dy) {
                R e = y[o];
#pragma unroll
                for (int c = 0; c < DX; ++c)
                    if (c < dx) e -= Cm[o * dx + c] * x[c];
                ss += e * e;
            }
        }
        l = p.c2 - ss * p.c1;
    }
    if constexpr (sizeof(R) == 8) return above_neg_inf((double)l) ? l : (R)(-INFINITY);
    else return (l > -INFINITY) ? l : (R)(-INFINITY);
}

}  // namespace airpf
