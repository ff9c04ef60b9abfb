/*
 * airpf_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential FP64 CPU restatement of the Augmented Island
 * Resampling Particle Filter (AIRPF) of Heine, "Augmented Island Resampling
 * Particle Filters for Particle Markov Chain Monte Carlo" (arXiv 2312.06484),
 * Algorithm 1, of the bootstrap particle filter (BPF) it reduces to for m = 1
 * (Section 2), and of particle marginal Metropolis-Hastings (Section 1.2).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It shares no code, header, table or constant generator
 * with the CUDA path; the two meet only through the written random-stream
 * specification below and the seeded inputs of the `synth` module.
 *
 * Random streams (counter-based, Philox4x32-10 of Salmon et al., SC'11):
 *   key     = (seed & 0xffffffff, seed >> 32)
 *   counter = (unit, t, iter, (chain << 8) | (kind << 5) | sub)
 *   kind 0 INIT  : prior draw of particle unit = k*M+i, t = 0, sub = normal pair b
 *   kind 1 STEP  : time t >= 1, g = k*M+i.  A transition with one normal:
 *                  counter unit = g >> 1, sub 0 (particles 2j, 2j+1 share
 *                  block j); g even takes the cosine normal and word 2 as its
 *                  internal-resampling uniform, g odd the sine normal and
 *                  word 3.  Otherwise unit = g, sub = normal pair b, and word 2
 *                  of sub 0 is the internal-resampling uniform of draw i
 *   kind 2 ISLAND: time t, unit = island j, sub = interaction stage s; word 0
 *   kind 3 MH    : PMMH iteration `iter`, t = 0; sub 0 unit b -> proposal
 *                  normals 2b, 2b+1; sub 1 unit 0 word 0 -> accept uniform
 *   change-point model (Beta draws): sub 0 words 0 (jump uniform, STEP only),
 *                  1 and 3 (boosts of the two gammas), 2 (resampling uniform);
 *                  gamma attempt j of X ~ Gamma(alpha) in sub 1 + 2j, of
 *                  Y ~ Gamma(beta) in sub 2 + 2j (words 0, 1 normal, word 2 uniform)
 *   uniform(w)    = (w + 0.5) * 2^-32
 *   normals(w0,w1): r = sqrt(-2 ln u(w0)), a = 2 pi u(w1); (r cos a, r sin a)
 *   the normal of dimension d is component (d & 1) of pair b = d >> 1.
 *
 * Readings of the paper taken here (the paper is silent on them):
 *   - time t = 1..T propagates x_{t-1} -> x_t (x_0 ~ prior), then weights
 *     with y_t: Algorithm 1 with pi_0 := law(x_1);
 *   - internal resampling is multinomial: draw j picks the first i with
 *     C_i > u_j * C_{M-1}, C the sequential FP64 CDF (Section 3.3, eq. (22));
 *   - an island whose particle weights are all zero keeps a_j = j;
 *   - a stage picks, for island k, the lower island of the pair
 *     {k, k xor 2^(s-1)} iff u * (W_lo + W_hi) < W_lo, one uniform per
 *     (t, s, k), independently over k (Section 3.3, eqs. (28)-(29)); with
 *     radix r, the first member c of k's group with C_c > u * sum W
 *     (C the cumulative member weights in member order);
 *   - adaptive interaction uses the strict test ENF < tau (Algorithm 1);
 *   - a NaN log-weight counts as -inf (weight zero);
 *   - change-point model (Section 4.2): the daily count k_t of the n_t articles
 *     is Binomial(n_t, x_t), y_t = (k_t, n_t); theta = (p, alpha, beta), p in
 *     [0, 1] (p = 0 and p = 1 are the closed-form special cases).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ----------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Section 4)             */
/* ----------------------------------------------------------------------- */
void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {            /* Weyl key schedule between rounds */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

enum { KIND_INIT = 0, KIND_STEP = 1, KIND_ISLAND = 2, KIND_MH = 3 };
enum { MODEL_AR1 = 0, MODEL_SV = 1, MODEL_NGM = 2, MODEL_LGSSM = 3, MODEL_TOY = 4, MODEL_CP = 5 };
enum { MODE_NEVER = 0, MODE_ALWAYS = 1, MODE_ADAPTIVE = 2 };
enum { TIE_NONE = 0, TIE_RESAMPLE = 1, TIE_ISLAND = 2, TIE_ENF = 3, TIE_ESS = 4 };

/* relative width of the tie band; 1e-12 for FP64 comparisons, set wider to
 * compare a float implementation draw by draw */
static double TIE_REL = 1e-12;

void oracle_set_tie_rel(double v) { TIE_REL = v > 0 ? v : 1e-12; }

/* Adaptive internal resampling (the paper's remark that its analysis holds for adaptive
 * internal resampling schemes): with tau_int in (0, 1], island k resamples internally at
 * step t only when the ESS of its particle weights w_i = omega_i g_t(x_i) is below
 * tau_int M, ESS = (sum w)^2 / sum w^2 (strict test, as the ENF test); otherwise its
 * particles stay and carry omega_i = w_i / sum w.  The island weight becomes W_{t,1} =
 * W_{t,0} sum_i omega_i g_t(x_i), with omega normalised per island (1/M after resampling),
 * which is M^-1 sum_i g_t(x_i) when every island resamples.  tau_int = 0: resample at every
 * step (Algorithm 1 as printed). */
static double TAU_INT = 0.0;

void oracle_set_tau_int(double v) { TAU_INT = (v > 0.0 && v <= 1.0) ? v : 0.0; }

/* Radix r = 2^b interactions (Section 2 restricts itself to r = 2 and states that the
 * analysis does not rely on it): m = r^S_r islands interact in S_r stages, stage s with
 * A_s = I_{r^(S_r - s)} (x) r^-1 1_r (x) I_{r^(s-1)}.  Island k's group at stage s is the r
 * islands whose base-r digits equal k's except digit s-1.  When the stage interacts
 * (Algorithm 1's adaptation line with the ENF of the weights before the stage), every
 * island's new weight is its group's mean (the normaliser line) and every island draws, from
 * its own uniform, one member of its group with probability proportional to the members'
 * weights (the selection line), independently of the other islands.  r = 2 is the binary
 * butterfly of eq. (3). */
static int RADIX_BITS = 1;

void oracle_set_radix(int r)
{
    int b = 0;
    while ((1 << b) < r) ++b;
    RADIX_BITS = (r >= 2 && (1 << b) == r) ? b : 1;
}

/* when set, oracle_airpf writes the output measures' moments [T][2][2][dx] here */
static double* MOMENTS_OUT = NULL;

void oracle_set_moments_out(double* p) { MOMENTS_OUT = p; }

/* When set, oracle_airpf marks, for every step t, which decisions fell within the tie band
 * (a diagnostic for comparing an implementation draw by draw; the arithmetic is unchanged):
 *   TIE_DRAW [T*N]: internal draw j of island k (index k*M+j) within the band of a CDF boundary
 *                   (or, with adaptive internal resampling, island k's ESS test);
 *   TIE_SRC  [T*m]: some island choice on the walk that gives island k its block was within
 *                   the band of a boundary;
 *   TIE_STEP [T]  : some ENF test of step t was within the band of tau. */
static uint8_t *TIE_DRAW = NULL, *TIE_SRC = NULL, *TIE_STEP = NULL;

void oracle_set_tie_masks(uint8_t* draw, uint8_t* src, uint8_t* step)
{
    TIE_DRAW = draw;
    TIE_SRC = src;
    TIE_STEP = step;
}

/* Eq. (output measure) of Section 2: pi^N_{t,s}(phi) = sum_k W^k_{t,s} M^-1 sum_i
 * phi(xi^{k,i}_{t,s}) / sum_k W^k_{t,s}, for phi = x_d (out[d]) and x_d^2
 * (out[dx + d]); lwk = log W^k_{t,s}, xs the particles.  NaN if every W is 0. */
static void output_moments(const double* lwk, const double* xs, int m, int M, int dx, double* out)
{
    double mx = -INFINITY;
    for (int k = 0; k < m; ++k) if (lwk[k] > mx) mx = lwk[k];
    for (int j = 0; j < 2 * dx; ++j) out[j] = mx > -INFINITY ? 0.0 : NAN;
    if (!(mx > -INFINITY)) return;
    double den = 0.0;
    for (int k = 0; k < m; ++k) {
        double wk = exp(lwk[k] - mx);
        den += wk;
        for (int d = 0; d < dx; ++d) {
            double s1 = 0.0, s2 = 0.0;
            for (int i = 0; i < M; ++i) {
                double v = xs[((size_t)k * M + i) * dx + d];
                s1 += v;
                s2 += v * v;
            }
            out[d] += wk * s1 / M;
            out[dx + d] += wk * s2 / M;
        }
    }
    for (int j = 0; j < 2 * dx; ++j) out[j] /= den;
}

typedef struct {
    uint64_t seed;
    uint32_t chain;
    uint32_t iter;
} stream_id;

static void draw(const stream_id* s, uint32_t unit, uint32_t t, uint32_t kind,
                 uint32_t sub, uint32_t out[4])
{
    uint32_t ctr[4] = { unit, t, s->iter, (s->chain << 8) | (kind << 5) | sub };
    uint32_t key[2] = { (uint32_t)(s->seed & 0xffffffffu), (uint32_t)(s->seed >> 32) };
    oracle_philox(ctr, key, out);
}

static double unif(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }

static void normal_pair(uint32_t w0, uint32_t w1, double* n0, double* n1)
{
    double rad = sqrt(-2.0 * log(unif(w0)));
    double ang = 2.0 * M_PI * unif(w1);
    *n0 = rad * cos(ang);
    *n1 = rad * sin(ang);
}

/* fills z[0..n-1] with the normals of (kind, unit, t); returns word 2 of
 * sub-block 0 and word 0 of sub-block 0 through w2/w0 when non-NULL.
 * A transition with one normal (n = 1) shares its block with the unit next
 * to it: units 2j and 2j+1 both draw block j; the even unit takes the cosine
 * normal and words 0 and 2, the odd unit the sine normal and words 1 and 3.
 * (The paper fixes the draws only in distribution; the two normals of one
 * Box-Muller pair are independent, as are the four words.) */
static void normals(const stream_id* s, uint32_t kind, uint32_t unit, uint32_t t,
                    int n, double* z, uint32_t* w0, uint32_t* w2)
{
    if (kind == KIND_STEP && n == 1) {
        uint32_t w[4];
        double a, c;
        int odd = (int)(unit & 1u);
        draw(s, unit >> 1, t, kind, 0, w);
        normal_pair(w[0], w[1], &a, &c);
        z[0] = odd ? c : a;
        if (w0) *w0 = odd ? w[1] : w[0];
        if (w2) *w2 = odd ? w[3] : w[2];
        return;
    }
    int pairs = n > 0 ? (n + 1) / 2 : 1;
    for (int b = 0; b < pairs; ++b) {
        uint32_t w[4];
        draw(s, unit, t, kind, (uint32_t)b, w);
        if (b == 0) {
            if (w0) *w0 = w[0];
            if (w2) *w2 = w[2];
        }
        if (n > 0) {
            double a, c;
            normal_pair(w[0], w[1], &a, &c);
            if (2 * b < n) z[2 * b] = a;
            if (2 * b + 1 < n) z[2 * b + 1] = c;
        }
    }
}

/* ----------------------------------------------------------------------- */
/* State-space models (Section 1.2, eq. (1)); parameter layout in synth/.  */
/* ----------------------------------------------------------------------- */
typedef struct {
    int model, dx, dy;
    const double* th;   /* model parameters */
    const double* md;   /* LGSSM: A (dx*dx row-major) then C (dy*dx) */
} model_t;

int oracle_model_valid(int model, int dx, const double* th)
{
    switch (model) {
    case MODEL_AR1: return th[1] > 0 && th[2] > 0 && th[3] > 0;
    case MODEL_SV:  return fabs(th[1]) < 1.0 && th[2] > 0;
    case MODEL_NGM: return th[0] > 0 && th[1] > 0 && th[2] > 0;
    case MODEL_TOY: return th[0] > 0 && th[0] < 1 && th[1] > 0 && th[1] < 1;
    case MODEL_LGSSM: return isfinite(th[dx]) && isfinite(th[dx + 1]);
    case MODEL_CP:  return th[0] >= 0 && th[0] <= 1 && th[1] > 0 && th[2] > 0;
    }
    return 0;
}

/* Gamma(a, 1) by the method of Marsaglia and Tsang (ACM TOMS 26(3), 2000): with
 * a' = a (a >= 1, else a + 1), d = a' - 1/3 and c = 1/sqrt(9 d), an attempt takes
 * a normal z and a uniform u, and with v = (1 + c z)^3 accepts d v if 1 + c z > 0
 * and log u < z^2/2 + d - d v + d log v.  Attempt j reads sub-block first + 2j of
 * the stream: the cosine normal of words 0 and 1, the uniform of word 2.  After
 * GAMMA_TRIES rejections the draw is d (each attempt is accepted with probability
 * above 0.95 for a' >= 1).  For a < 1 the draw is then scaled by U^(1/a), U from
 * the word wboost (Marsaglia and Tsang's boost). */
#define GAMMA_TRIES 15
static double gamma_draw(const stream_id* s, uint32_t kind, uint32_t unit, uint32_t t, uint32_t first,
                         double a, uint32_t wboost)
{
    double ap = a < 1.0 ? a + 1.0 : a;
    double d = ap - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    double g = d;
    for (int j = 0; j < GAMMA_TRIES; ++j) {
        uint32_t w[4];
        double z, z1;
        draw(s, unit, t, kind, first + 2u * (uint32_t)j, w);
        normal_pair(w[0], w[1], &z, &z1);
        double x1 = 1.0 + c * z;
        if (x1 <= 0.0) continue;
        double v = x1 * x1 * x1;
        if (log(unif(w[2])) < 0.5 * z * z + d - d * v + d * log(v)) {
            g = d * v;
            break;
        }
    }
    if (a < 1.0) g *= exp(log(unif(wboost)) / a);
    return g;
}

/* Beta(alpha, beta) = X / (X + Y) with X ~ Gamma(alpha) from sub-blocks 1, 3, 5, ...
 * and Y ~ Gamma(beta) from sub-blocks 2, 4, 6, ...; w0blk is sub-block 0, whose
 * words 3 and 1 are the two boosts. */
static double beta_draw(const stream_id* s, uint32_t kind, uint32_t unit, uint32_t t, double alpha,
                        double beta, const uint32_t w0blk[4])
{
    double x = gamma_draw(s, kind, unit, t, 1u, alpha, w0blk[3]);
    double y = gamma_draw(s, kind, unit, t, 2u, beta, w0blk[1]);
    return x / (x + y);
}

static void prior_sample(const model_t* md, const stream_id* s, uint32_t unit, double* x)
{
    if (md->model == MODEL_CP) {            /* x_0 ~ Beta(alpha, beta) */
        uint32_t w[4];
        draw(s, unit, 0, KIND_INIT, 0, w);
        x[0] = beta_draw(s, KIND_INIT, unit, 0, md->th[1], md->th[2], w);
        return;
    }
    double z[64];
    uint32_t w0;
    int nz = md->model == MODEL_TOY ? 0 : md->dx;
    normals(s, KIND_INIT, unit, 0, nz, z, &w0, NULL);
    const double* th = md->th;
    switch (md->model) {
    case MODEL_AR1: x[0] = th[3] * z[0]; break;
    case MODEL_SV:  x[0] = th[0] + th[2] / sqrt(1.0 - th[1] * th[1]) * z[0]; break;
    case MODEL_NGM: x[0] = sqrt(th[2]) * z[0]; break;
    case MODEL_TOY: x[0] = unif(w0) < 0.5 ? 0.0 : 1.0; break;
    case MODEL_LGSSM:
        for (int d = 0; d < md->dx; ++d) x[d] = z[d];
        break;
    }
}

/* x_t ~ K_t(x_{t-1}, .); returns the internal-resampling word of this unit */
static uint32_t transition(const model_t* md, const stream_id* s, uint32_t unit,
                           uint32_t t, const double* xp, double* x)
{
    if (md->model == MODEL_CP) {
        /* K(x, .) = (1 - p) delta_x + p Beta(alpha, beta): the jump iff u(word 0) < p;
         * word 2 is the internal-resampling uniform, as for every model */
        uint32_t w[4];
        draw(s, unit, t, KIND_STEP, 0, w);
        x[0] = unif(w[0]) < md->th[0] ? beta_draw(s, KIND_STEP, unit, t, md->th[1], md->th[2], w) : xp[0];
        return w[2];
    }
    double z[64];
    uint32_t w0, w2;
    int nz = md->model == MODEL_TOY ? 0 : md->dx;
    normals(s, KIND_STEP, unit, t, nz, z, &w0, &w2);
    const double* th = md->th;
    switch (md->model) {
    case MODEL_AR1: x[0] = th[0] * xp[0] + th[1] * z[0]; break;
    case MODEL_SV:  x[0] = th[0] + th[1] * (xp[0] - th[0]) + th[2] * z[0]; break;
    case MODEL_NGM: {
        double v = xp[0];
        x[0] = 0.5 * v + 25.0 * v / (1.0 + v * v) + 8.0 * cos(1.2 * (double)t) + sqrt(th[0]) * z[0];
        break;
    }
    case MODEL_TOY:
        x[0] = unif(w0) < 1.0 - th[0] ? 1.0 - xp[0] : xp[0];
        break;
    case MODEL_LGSSM: {
        int dx = md->dx;
        const double* A = md->md;
        double sq = sqrt(exp(th[dx]));
        for (int r = 0; r < dx; ++r) {
            double acc = 0.0;
            for (int c = 0; c < dx; ++c) {
                double a = (r == c) ? th[r] : A[r * dx + c];
                acc += a * xp[c];
            }
            x[r] = acc + sq * z[r];
        }
        break;
    }
    }
    return w2;
}

static double log_g(const model_t* md, const double* y, const double* x)
{
    const double* th = md->th;
    const double half_log_2pi = 0.5 * log(2.0 * M_PI);
    double l = -INFINITY;
    switch (md->model) {
    case MODEL_AR1: {
        double e = (y[0] - x[0]) / th[2];
        l = -half_log_2pi - log(th[2]) - 0.5 * e * e;
        break;
    }
    case MODEL_SV:
        l = -half_log_2pi - 0.5 * x[0] - 0.5 * y[0] * y[0] * exp(-x[0]);
        break;
    case MODEL_NGM: {
        double e = y[0] - x[0] * x[0] / 20.0;
        l = -0.5 * log(2.0 * M_PI * th[1]) - e * e / (2.0 * th[1]);
        break;
    }
    case MODEL_TOY:
        l = (y[0] == x[0]) ? log(th[1]) : log(1.0 - th[1]);
        break;
    case MODEL_CP: {                        /* y = (k, n): k ~ Binomial(n, x) */
        double k = y[0], n = y[1];
        l = lgamma(n + 1.0) - lgamma(k + 1.0) - lgamma(n - k + 1.0);
        if (k > 0) l += k * log(x[0]);
        if (n - k > 0) l += (n - k) * log1p(-x[0]);
        break;
    }
    case MODEL_LGSSM: {
        int dx = md->dx, dy = md->dy;
        const double* C = md->md + dx * dx;
        double r = exp(th[dx + 1]);
        double ss = 0.0;
        for (int o = 0; o < dy; ++o) {
            double e = y[o];
            for (int c = 0; c < dx; ++c) e -= C[o * dx + c] * x[c];
            ss += e * e;
        }
        l = -0.5 * dy * log(2.0 * M_PI * r) - ss / (2.0 * r);
        break;
    }
    }
    if (!(l > -INFINITY)) l = -INFINITY;   /* NaN counts as weight zero */
    return l;
}

/* exported single-particle model calls (pinned in the tests) */
double oracle_model_logg(int model, int dx, int dy, const double* th, const double* mdat,
                         const double* y, const double* x)
{
    model_t md = { model, dx, dy, th, mdat };
    return log_g(&md, y, x);
}

void oracle_model_prior(int model, int dx, int dy, const double* th, const double* mdat,
                        uint64_t seed, uint32_t chain, uint32_t iter, uint32_t unit, double* x)
{
    model_t md = { model, dx, dy, th, mdat };
    stream_id s = { seed, chain, iter };
    prior_sample(&md, &s, unit, x);
}

void oracle_model_step(int model, int dx, int dy, const double* th, const double* mdat,
                       uint64_t seed, uint32_t chain, uint32_t iter, uint32_t unit, uint32_t t,
                       const double* xp, double* x)
{
    model_t md = { model, dx, dy, th, mdat };
    stream_id s = { seed, chain, iter };
    transition(&md, &s, unit, t, xp, x);
}

/* ----------------------------------------------------------------------- */
/* helpers                                                                  */
/* ----------------------------------------------------------------------- */
static double log_sum_exp(const double* v, int n)
{
    double mx = -INFINITY;
    for (int i = 0; i < n; ++i) if (v[i] > mx) mx = v[i];
    if (mx == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(v[i] - mx);
    return mx + log(s);
}

/* effective number of filters (Algorithm 1): (m^-1 sum W)^2 / (m^-1 sum W^2),
 * from log-weights; 0 when every weight is zero */
static double enf_of(const double* lw, int m)
{
    double mx = -INFINITY;
    for (int k = 0; k < m; ++k) if (lw[k] > mx) mx = lw[k];
    if (mx == -INFINITY) return 0.0;
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < m; ++k) {
        double w = exp(lw[k] - mx);
        s1 += w;
        s2 += w * w;
    }
    return (s1 / m) * (s1 / m) / (s2 / m);
}

/* Multinomial internal resampling of one island (Algorithm 1, internal
 * resample): draw j takes the first i with C_i > u_j * C_{M-1}.  Returns 1 if
 * some draw fell within TIE_REL * C_{M-1} of a CDF boundary; flags[j] (if not
 * NULL) marks those draws. */
static int resample_island(const double* l, int M, const uint32_t* wres,
                           double* cdf, int32_t* a, uint8_t* flags)
{
    double mx = -INFINITY;
    for (int i = 0; i < M; ++i) if (l[i] > mx) mx = l[i];
    if (mx == -INFINITY) {                 /* all weights zero */
        for (int j = 0; j < M; ++j) a[j] = j;
        if (flags) memset(flags, 0, (size_t)M);
        return 0;
    }
    double acc = 0.0;
    for (int i = 0; i < M; ++i) {
        acc += exp(l[i] - mx);
        cdf[i] = acc;
    }
    double total = cdf[M - 1];
    int tie = 0;
    for (int j = 0; j < M; ++j) {
        double target = unif(wres[j]) * total;
        int i = 0;
        while (i < M - 1 && !(cdf[i] > target)) ++i;
        a[j] = i;
        double tol = TIE_REL * total;
        int near = fabs(cdf[i] - target) < tol || (i > 0 && fabs(cdf[i - 1] - target) < tol);
        if (near) tie = 1;
        if (flags) flags[j] = (uint8_t)near;
    }
    return tie;
}

static int ilog2(int m)
{
    int s = 0;
    while ((1 << s) < m) ++s;
    return s;
}

/* ----------------------------------------------------------------------- */
/* AIRPF, Algorithm 1, one stage at a time.                                 */
/* ----------------------------------------------------------------------- */
typedef struct {
    double* logz;        /* [1] log Z^N_T = log (m^-1 sum_k W^k) */
    double* logz_trace;  /* [T] log Z^N_t after step t, or NULL */
    int32_t* anc;        /* [T*N] parent (among the time-t particles) of the
                            particle k*M+i held after step t, or NULL */
    int32_t* src;        /* [T*m] island whose block island k holds after step t */
    double* enf;         /* [T*(S_r+1)] ENF_{t,0..S_r}, or NULL (S_r = log_r m stages) */
    int32_t* sstar;      /* [T] first non-interacting stage (S_r+1 if all interact) */
    double* xfinal;      /* [N*dx] particles after step T (before mutation), or NULL */
    int32_t* tie;        /* [2] first flagged tie: time t (0 = none) and kind */
} airpf_out;

int oracle_airpf(int model, int dx, int dy, int m, int M, int T, int mode, double tau,
                 uint64_t seed, uint32_t chain, uint32_t iter,
                 const double* theta, const double* mdat, const double* y,
                 double* logz, double* logz_trace, int32_t* anc, int32_t* src,
                 double* enf, int32_t* sstar, double* xfinal, int32_t* tie)
{
    if (m < 1 || (m & (m - 1)) || M < 1 || T < 1 || dx < 1 || dx > 64 || dy < 1) return 1;
    if (!(tau > 0.0 && tau <= 1.0)) return 1;
    if (TAU_INT > 0.0 && MOMENTS_OUT) return 1;   /* the output measures assume resampling */
    if (ilog2(m) % RADIX_BITS != 0) return 1;      /* m must be a power of the radix */
    const int N = m * M, S = ilog2(m), Sr = S / RADIX_BITS, radix = 1 << RADIX_BITS;
    model_t md = { model, dx, dy, theta, mdat };
    stream_id st = { seed, chain, iter };

    double* xa = malloc(sizeof(double) * N * dx);   /* parents of this step */
    double* x = malloc(sizeof(double) * N * dx);    /* propagated particles */
    double* xr = malloc(sizeof(double) * N * dx);   /* internally resampled */
    double* l = malloc(sizeof(double) * N);
    double* cdf = malloc(sizeof(double) * N);
    uint32_t* wres = malloc(sizeof(uint32_t) * N);
    int32_t* a = malloc(sizeof(int32_t) * N);
    double* lom = malloc(sizeof(double) * N);      /* log omega (adaptive internal resampling) */
    double* lom2 = malloc(sizeof(double) * N);
    double* lw = malloc(sizeof(double) * m);        /* log W^k */
    double* lw2 = malloc(sizeof(double) * m);
    int* idx = malloc(sizeof(int) * m);
    int* idx2 = malloc(sizeof(int) * m);
    int* tie_isl = calloc((size_t)m, sizeof(int));
    double* wc = malloc(sizeof(double) * radix);    /* group members' weights (relative) */
    double* cum = malloc(sizeof(double) * radix);   /* their cumulative sums */
    uint8_t* sflag = malloc((size_t)m);             /* a tied choice on island k's walk */
    uint8_t* sflag2 = malloc((size_t)m);
    if (tie) { tie[0] = 0; tie[1] = TIE_NONE; }

    /* initialisation: W^k_{0,0} = 1, particles from the prior */
    for (int g = 0; g < N; ++g) prior_sample(&md, &st, (uint32_t)g, xa + (size_t)g * dx);
    for (int k = 0; k < m; ++k) lw[k] = 0.0;
    for (int g = 0; g < N; ++g) lom[g] = -log((double)M);

    for (int t = 1; t <= T; ++t) {
        const double* yt = y + (size_t)(t - 1) * dy;
        int tie_now = TIE_NONE;
        /* ENF_{t,0} (diagnostic, Algorithm 1) */
        if (enf) enf[(size_t)(t - 1) * (Sr + 1)] = enf_of(lw, m);

        if (MOMENTS_OUT) memcpy(lw2, lw, sizeof(double) * m);      /* log W^k_{t,0} */
        /* mutation of every island's block through K_t, then weighting */
        #pragma omp parallel for schedule(static)
        for (int k = 0; k < m; ++k) {
            for (int i = 0; i < M; ++i) {
                int g = k * M + i;
                wres[g] = transition(&md, &st, (uint32_t)g, (uint32_t)t, xa + (size_t)g * dx,
                                     x + (size_t)g * dx);
                l[g] = log_g(&md, yt, x + (size_t)g * dx);
                if (TAU_INT > 0.0) l[g] += lom[g];     /* log(omega_i g_t(xi^{k,i})) */
            }
            const double* lk = l + (size_t)k * M;
            const double lse = log_sum_exp(lk, M);
            /* W^k_{t,1} = W^k_{t,0} * M^-1 sum_i g_t(xi^{k,i})  (sum_i omega_i g_t with
             * adaptive internal resampling) */
            lw[k] += TAU_INT > 0.0 ? lse : lse - log((double)M);
            /* internal resampling within island k: always, or when its ESS is below tau_int M */
            int resample = 1;
            tie_isl[k] = 0;
            if (TAU_INT > 0.0 && lse > -INFINITY) {
                double s1 = 0.0, s2 = 0.0, mx = -INFINITY;
                for (int i = 0; i < M; ++i) if (lk[i] > mx) mx = lk[i];
                for (int i = 0; i < M; ++i) {
                    double w = exp(lk[i] - mx);
                    s1 += w;
                    s2 += w * w;
                }
                double ess = s1 * s1 / s2, thr = TAU_INT * M;
                resample = ess < thr;
                if (fabs(ess - thr) < TIE_REL * thr) tie_isl[k] = 2;
            }
            uint8_t* dflag = TIE_DRAW ? TIE_DRAW + (size_t)(t - 1) * N + (size_t)k * M : NULL;
            if (resample) {
                if (resample_island(lk, M, wres + (size_t)k * M, cdf + (size_t)k * M, a + (size_t)k * M, dflag))
                    tie_isl[k] = tie_isl[k] ? tie_isl[k] : 1;
                for (int j = 0; j < M; ++j) lom2[(size_t)k * M + j] = -log((double)M);
            } else {
                for (int j = 0; j < M; ++j) {
                    a[k * M + j] = j;
                    lom2[(size_t)k * M + j] = lk[j] - lse;
                }
                if (dflag)
                    for (int j = 0; j < M; ++j) dflag[j] = 0;
            }
            if (dflag && tie_isl[k] == 2)                  /* the ESS test itself */
                for (int j = 0; j < M; ++j) dflag[j] = 1;
            for (int j = 0; j < M; ++j)
                memcpy(xr + ((size_t)k * M + j) * dx, x + ((size_t)k * M + a[k * M + j]) * dx,
                       sizeof(double) * dx);
        }
        for (int k = 0; k < m; ++k)
            if (tie_isl[k] && tie_now == TIE_NONE) tie_now = tie_isl[k] == 2 ? TIE_ESS : TIE_RESAMPLE;
        if (MOMENTS_OUT) {
            /* s = 0: the mutated particles with W_{t,0}; s = 1: the internally
             * resampled particles with W_{t,1} (before the interaction stages) */
            output_moments(lw2, x, m, M, dx, MOMENTS_OUT + (size_t)(t - 1) * 4 * dx);
            output_moments(lw, xr, m, M, dx, MOMENTS_OUT + (size_t)(t - 1) * 4 * dx + 2 * dx);
        }

        /* interaction stages s = 1..S_r (matrices A_s over groups of r islands) */
        for (int k = 0; k < m; ++k) idx[k] = k;
        for (int k = 0; k < m; ++k) sflag[k] = 0;
        int step_flag = 0;
        int first_quiet = Sr + 1;
        for (int s = 1; s <= Sr; ++s) {
            double e = enf_of(lw, m);
            if (enf) enf[(size_t)(t - 1) * (Sr + 1) + s] = e;
            int interact = (mode == MODE_ALWAYS) || (mode == MODE_ADAPTIVE && e < tau);
            if (mode == MODE_ADAPTIVE && fabs(e - tau) < TIE_REL * tau) {
                step_flag = 1;
                if (tie_now == TIE_NONE) tie_now = TIE_ENF;
            }
            if (!interact) {
                if (first_quiet == Sr + 1) first_quiet = s;
                continue;            /* alpha_s = I: weights and blocks unchanged */
            }
            const int stride = 1 << (RADIX_BITS * (s - 1));      /* r^(s-1) */
            for (int k = 0; k < m; ++k) {
                /* the group of k: base + c * stride, c = 0..r-1 */
                const int base = k & ~((radix - 1) * stride);
                double ref = -INFINITY;
                for (int c = 0; c < radix; ++c)
                    if (lw[base + c * stride] > ref) ref = lw[base + c * stride];
                double wsum = 0.0;
                for (int c = 0; c < radix; ++c) {
                    wc[c] = ref > -INFINITY ? exp(lw[base + c * stride] - ref) : 0.0;
                    wsum += wc[c];
                    cum[c] = wsum;
                }
                uint32_t w[4];
                draw(&st, (uint32_t)k, (uint32_t)t, KIND_ISLAND, (uint32_t)s, w);
                /* member c with probability W_c / sum W: the first c with C_c > u sum W
                 * (the last member when every weight is zero) */
                const double target = unif(w[0]) * wsum;
                int pick = 0;
                while (pick < radix - 1 && !(cum[pick] > target)) ++pick;
                int near = 0;
                for (int c = 0; c < radix - 1; ++c)
                    if (fabs(cum[c] - target) < TIE_REL * wsum) near = 1;
                if (near && tie_now == TIE_NONE) tie_now = TIE_ISLAND;
                idx2[k] = idx[base + pick * stride];
                sflag2[k] = (uint8_t)(sflag[base + pick * stride] | near);
                /* W^k_{t,s+1} = sum_l alpha_s^{kl} W^l_{t,s} = r^-1 sum_c W_c */
                lw2[k] = (ref > -INFINITY) ? ref + log(wsum / radix) : -INFINITY;
            }
            memcpy(idx, idx2, sizeof(int) * m);
            memcpy(sflag, sflag2, (size_t)m);
            memcpy(lw, lw2, sizeof(double) * m);
        }
        if (TIE_SRC) memcpy(TIE_SRC + (size_t)(t - 1) * m, sflag, (size_t)m);
        if (TIE_STEP) TIE_STEP[t - 1] = (uint8_t)step_flag;

        /* island k now holds the internally resampled block of island idx[k] */
        for (int k = 0; k < m; ++k) {
            memcpy(xa + (size_t)k * M * dx, xr + (size_t)idx[k] * M * dx, sizeof(double) * M * dx);
            memcpy(lom + (size_t)k * M, lom2 + (size_t)idx[k] * M, sizeof(double) * M);
            if (anc)
                for (int i = 0; i < M; ++i)
                    anc[(size_t)(t - 1) * N + k * M + i] = idx[k] * M + a[idx[k] * M + i];
            if (src) src[(size_t)(t - 1) * m + k] = idx[k];
        }
        if (sstar) sstar[t - 1] = first_quiet;
        if (logz_trace) logz_trace[t - 1] = log_sum_exp(lw, m) - log((double)m);
        if (tie && tie[0] == 0 && tie_now != TIE_NONE) { tie[0] = t; tie[1] = tie_now; }
    }
    *logz = log_sum_exp(lw, m) - log((double)m);
    if (xfinal) memcpy(xfinal, xa, sizeof(double) * N * dx);

    free(xa); free(x); free(xr); free(l); free(cdf); free(wres); free(a);
    free(lw); free(lw2); free(idx); free(idx2); free(tie_isl); free(lom); free(lom2); free(wc); free(cum);
    free(sflag); free(sflag2);
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Bootstrap particle filter (Gordon et al.), the m = 1 case of Section 2.  */
/* Written separately from oracle_airpf.  `unit0` offsets the particle      */
/* stream so that island k of an AIRPF run is reproduced with unit0 = k*M.  */
/* ----------------------------------------------------------------------- */
int oracle_bpf(int model, int dx, int dy, int M, int T, uint64_t seed, uint32_t chain,
               uint32_t iter, uint32_t unit0, const double* theta, const double* mdat,
               const double* y, double* logz, int32_t* anc, int32_t* tie)
{
    if (M < 1 || T < 1 || dx < 1 || dx > 64) return 1;
    model_t md = { model, dx, dy, theta, mdat };
    stream_id st = { seed, chain, iter };
    double* xp = malloc(sizeof(double) * M * dx);
    double* x = malloc(sizeof(double) * M * dx);
    double* l = malloc(sizeof(double) * M);
    double* cdf = malloc(sizeof(double) * M);
    uint32_t* wres = malloc(sizeof(uint32_t) * M);
    int32_t* a = malloc(sizeof(int32_t) * M);
    double lz = 0.0;
    if (tie) { tie[0] = 0; tie[1] = TIE_NONE; }
    for (int i = 0; i < M; ++i) prior_sample(&md, &st, unit0 + (uint32_t)i, xp + (size_t)i * dx);
    for (int t = 1; t <= T; ++t) {
        for (int i = 0; i < M; ++i) {
            wres[i] = transition(&md, &st, unit0 + (uint32_t)i, (uint32_t)t, xp + (size_t)i * dx,
                                 x + (size_t)i * dx);
            l[i] = log_g(&md, y + (size_t)(t - 1) * dy, x + (size_t)i * dx);
        }
        lz += log_sum_exp(l, M) - log((double)M);
        int tf = resample_island(l, M, wres, cdf, a, NULL);
        if (tie && tie[0] == 0 && tf) { tie[0] = t; tie[1] = TIE_RESAMPLE; }
        for (int j = 0; j < M; ++j) {
            memcpy(xp + (size_t)j * dx, x + (size_t)a[j] * dx, sizeof(double) * dx);
            if (anc) anc[(size_t)(t - 1) * M + j] = a[j];
        }
    }
    *logz = lz;
    free(xp); free(x); free(l); free(cdf); free(wres); free(a);
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Particle marginal Metropolis-Hastings (Andrieu et al. 2010; Section 1.2 */
/* and Theorem 1's remark): random-walk proposal on the components with     */
/* step > 0, independent uniform priors on [lo, hi], AIRPF estimate of Z.   */
/* The initial estimate uses iter = 0xffffffff; iteration j uses iter = j.  */
/* state[0] holds log Z of the current theta; pass state[0] = NaN to start. */
/* ----------------------------------------------------------------------- */
int oracle_pmmh(int model, int dx, int dy, int m, int M, int T, int mode, double tau,
                uint64_t seed, uint32_t chain, const double* mdat, const double* y,
                int d_theta, const double* step, const double* lo, const double* hi,
                double* theta /* [d_theta], in/out */, double* state_logz /* in/out */,
                uint32_t iter0, int iters, double* theta_out, double* logz_out, int32_t* n_accept)
{
    double prop[64];
    if (d_theta < 1 || d_theta > 64) return 1;
    int acc = 0;
    if (isnan(*state_logz)) {
        double lz;
        int rc = oracle_airpf(model, dx, dy, m, M, T, mode, tau, seed, chain, 0xffffffffu,
                              theta, mdat, y, &lz, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
        if (rc) return rc;
        *state_logz = lz;
    }
    for (int j = 0; j < iters; ++j) {
        uint32_t it = iter0 + (uint32_t)j;
        stream_id st = { seed, chain, it };
        double z[64];
        /* proposal normals: kind MH, sub 0, unit = pair index b, t = 0 */
        for (int b = 0; b < (d_theta + 1) / 2; ++b) {
            uint32_t w[4];
            draw(&st, (uint32_t)b, 0, KIND_MH, 0, w);
            double a, c;
            normal_pair(w[0], w[1], &a, &c);
            z[2 * b] = a;
            if (2 * b + 1 < d_theta) z[2 * b + 1] = c;
        }
        int inside = 1;
        for (int d = 0; d < d_theta; ++d) {
            prop[d] = theta[d] + step[d] * z[d];
            if (step[d] > 0.0 && !(prop[d] >= lo[d] && prop[d] <= hi[d])) inside = 0;
        }
        if (inside && !oracle_model_valid(model, dx, prop)) inside = 0;
        if (inside) {
            double lz;
            int rc = oracle_airpf(model, dx, dy, m, M, T, mode, tau, seed, chain, it,
                                  prop, mdat, y, &lz, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
            if (rc) return rc;
            uint32_t w[4];
            draw(&st, 0, 0, KIND_MH, 1, w);
            /* uniform priors cancel inside the box */
            if (log(unif(w[0])) < lz - *state_logz) {
                memcpy(theta, prop, sizeof(double) * d_theta);
                *state_logz = lz;
                ++acc;
            }
        }
        if (theta_out) memcpy(theta_out + (size_t)j * d_theta, theta, sizeof(double) * d_theta);
        if (logz_out) logz_out[j] = *state_logz;
    }
    if (n_accept) *n_accept = acc;
    return 0;
}

/* ----------------------------------------------------------------------- */
/* R independent runs (chains chain0 .. chain0+R-1), log Z of each.         */
/* ----------------------------------------------------------------------- */
int oracle_airpf_batch(int model, int dx, int dy, int m, int M, int T, int mode, double tau,
                       uint64_t seed, uint32_t chain0, uint32_t iter, int R,
                       const double* theta, const double* mdat, const double* y, double* logz)
{
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 4) reduction(|:bad)
    for (int r = 0; r < R; ++r) {
        int rc = oracle_airpf(model, dx, dy, m, M, T, mode, tau, seed, chain0 + (uint32_t)r, iter,
                              theta, mdat, y, logz + r, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
        bad |= rc;
    }
    return bad;
}

/* ----------------------------------------------------------------------- */
/* Gradients of log Z (test references for the adjoint and the Fisher score)*/
/* ----------------------------------------------------------------------- */

/* log f_t(x | xp): density of the transition K_t (Section 1.2, eq. (1)). */
static double log_f(const model_t* md, uint32_t t, const double* xp, const double* x)
{
    const double* th = md->th;
    const double l2pi = log(2.0 * M_PI);
    switch (md->model) {
    case MODEL_AR1: {
        double e = (x[0] - th[0] * xp[0]) / th[1];
        return -0.5 * l2pi - log(th[1]) - 0.5 * e * e;
    }
    case MODEL_SV: {
        double e = (x[0] - th[0] - th[1] * (xp[0] - th[0])) / th[2];
        return -0.5 * l2pi - log(th[2]) - 0.5 * e * e;
    }
    case MODEL_NGM: {
        double v = xp[0];
        double mu = 0.5 * v + 25.0 * v / (1.0 + v * v) + 8.0 * cos(1.2 * (double)t);
        double e = x[0] - mu;
        return -0.5 * log(2.0 * M_PI * th[0]) - e * e / (2.0 * th[0]);
    }
    case MODEL_LGSSM: {
        int dx = md->dx;
        const double* A = md->md;
        double q = exp(th[dx]), ss = 0.0;
        for (int r = 0; r < dx; ++r) {
            double mu = 0.0;
            for (int c = 0; c < dx; ++c) mu += ((r == c) ? th[r] : A[r * dx + c]) * xp[c];
            ss += (x[r] - mu) * (x[r] - mu);
        }
        return -0.5 * dx * log(2.0 * M_PI * q) - ss / (2.0 * q);
    }
    }
    return -INFINITY;
}

/* log of the prior density pi_0(x) of x_0 */
static double log_mu(const model_t* md, const double* x)
{
    const double* th = md->th;
    const double l2pi = log(2.0 * M_PI);
    switch (md->model) {
    case MODEL_AR1: {
        double e = x[0] / th[3];
        return -0.5 * l2pi - log(th[3]) - 0.5 * e * e;
    }
    case MODEL_SV: {
        double sd = th[2] / sqrt(1.0 - th[1] * th[1]), e = (x[0] - th[0]) / sd;
        return -0.5 * l2pi - log(sd) - 0.5 * e * e;
    }
    case MODEL_NGM:
        return -0.5 * log(2.0 * M_PI * th[2]) - x[0] * x[0] / (2.0 * th[2]);
    case MODEL_LGSSM: {
        double ss = 0.0;
        for (int d = 0; d < md->dx; ++d) ss += x[d] * x[d];
        return -0.5 * md->dx * l2pi - 0.5 * ss;
    }
    }
    return -INFINITY;
}

double oracle_model_logf(int model, int dx, int dy, const double* th, const double* mdat, uint32_t t,
                         const double* xp, const double* x)
{
    model_t md = { model, dx, dy, th, mdat };
    return log_f(&md, t, xp, x);
}

double oracle_model_logmu(int model, int dx, int dy, const double* th, const double* mdat, const double* x)
{
    model_t md = { model, dx, dy, th, mdat };
    return log_mu(&md, x);
}

/* The particles x_t (t = 0..T, time-t particles before resampling; x_0 the
 * prior draws) and the island log-weights log W^k_{t,1} of a run whose
 * lineage (anc, as oracle_airpf records it) and first quiet stages s*_t are
 * given: the random numbers are the run's, the ancestors and island choices
 * are held fixed, and the weights follow Algorithm 1 with the interacting
 * stages 1..s*_t-1 (after them every island weight is the mean of its block
 * of r^(s*_t-1) islands, r the radix).  xs [(T+1)*N*dx] and lw1 [T*m] may be NULL. */
static void fixed_lineage_pass(const model_t* md, const stream_id* st, int m, int M, int T, const double* y,
                               const int32_t* anc, const int32_t* sstar, double* xs, double* lw1,
                               double* logz, double* l_out)
{
    const int N = m * M, dx = md->dx;
    double* held = malloc(sizeof(double) * N * dx);
    double* x = malloc(sizeof(double) * N * dx);
    double* l = malloc(sizeof(double) * N);
    double* lw = malloc(sizeof(double) * m);
    double* lwn = malloc(sizeof(double) * m);
    for (int g = 0; g < N; ++g) prior_sample(md, st, (uint32_t)g, held + (size_t)g * dx);
    if (xs) memcpy(xs, held, sizeof(double) * N * dx);
    for (int k = 0; k < m; ++k) lw[k] = 0.0;
    for (int t = 1; t <= T; ++t) {
        const double* yt = y + (size_t)(t - 1) * md->dy;
        for (int g = 0; g < N; ++g) {
            transition(md, st, (uint32_t)g, (uint32_t)t, held + (size_t)g * dx, x + (size_t)g * dx);
            l[g] = log_g(md, yt, x + (size_t)g * dx);
        }
        if (l_out) memcpy(l_out + (size_t)(t - 1) * N, l, sizeof(double) * N);
        if (xs) memcpy(xs + (size_t)t * N * dx, x, sizeof(double) * N * dx);
        for (int k = 0; k < m; ++k) lw[k] += log_sum_exp(l + (size_t)k * M, M) - log((double)M);
        if (lw1) memcpy(lw1 + (size_t)(t - 1) * m, lw, sizeof(double) * m);
        /* block means over r^(s*_t - 1) = 2^lvl islands */
        int lvl = (sstar[t - 1] - 1) * RADIX_BITS, bs = 1 << lvl;
        for (int b = 0; b < m; b += bs) {
            double v = log_sum_exp(lw + b, bs) - lvl * log(2.0);
            for (int k = b; k < b + bs; ++k) lwn[k] = v;
        }
        memcpy(lw, lwn, sizeof(double) * m);
        /* held particles after step t */
        for (int g = 0; g < N; ++g)
            memcpy(held + (size_t)g * dx, x + (size_t)anc[(size_t)(t - 1) * N + g] * dx, sizeof(double) * dx);
    }
    *logz = log_sum_exp(lw, m) - log((double)m);
    free(held); free(x); free(l); free(lw); free(lwn);
}

/* log Z^N_T as a function of theta with the run's random numbers, ancestors and
 * s* held fixed: the quantity whose gradient the adjoint pass computes. */
int oracle_logz_fixed(int model, int dx, int dy, int m, int M, int T, uint64_t seed, uint32_t chain,
                      uint32_t iter, const double* theta, const double* mdat, const double* y,
                      const int32_t* anc, const int32_t* sstar, double* logz)
{
    if (m < 1 || (m & (m - 1)) || M < 1 || T < 1 || dx < 1 || dx > 64 || dy < 1) return 1;
    model_t md = { model, dx, dy, theta, mdat };
    stream_id st = { seed, chain, iter };
    fixed_lineage_pass(&md, &st, m, M, T, y, anc, sstar, NULL, NULL, logz, NULL);
    return 0;
}

/* Fisher-identity score along the lineages (Section 1.2 with the genealogy of
 * the particle system as the smoother): every time-t particle q carries the
 * final weight delta_t(q) of its descendants (delta_T = island share of the
 * final weight times the particle's share within its island; delta_{t-1} of a
 * parent = sum over its children), and
 *   score = sum_t sum_q delta_t(q) grad_theta [log f_t(x_t^q | parent) + log g_t(y_t | x_t^q)]
 *           + sum_q delta_0(q) grad_theta log pi_0(x_0^q).
 * The theta-gradients of the densities are central differences (step
 * h_d = 1e-6 max(1, |theta_d|)) of log_f, log_g and log_mu at fixed x. */
int oracle_fisher_score(int model, int dx, int dy, int m, int M, int T, uint64_t seed, uint32_t chain,
                        uint32_t iter, const double* theta, const double* mdat, const double* y,
                        const int32_t* anc, const int32_t* sstar, int d_theta, double* score)
{
    if (m < 1 || (m & (m - 1)) || M < 1 || T < 1 || dx < 1 || dx > 64 || dy < 1 || d_theta < 1 ||
        d_theta > 64)
        return 1;
    const int N = m * M;
    model_t md = { model, dx, dy, theta, mdat };
    stream_id st = { seed, chain, iter };
    double* xs = malloc(sizeof(double) * (size_t)(T + 1) * N * dx);
    double* lw1 = malloc(sizeof(double) * (size_t)T * m);
    double* l = malloc(sizeof(double) * (size_t)T * N);
    double* dl = malloc(sizeof(double) * N);
    double* dlp = malloc(sizeof(double) * N);
    double logz;
    fixed_lineage_pass(&md, &st, m, M, T, y, anc, sstar, xs, lw1, &logz, l);
    /* delta_T: island share x share within the island */
    double lz = log_sum_exp(lw1 + (size_t)(T - 1) * m, m);
    for (int k = 0; k < m; ++k) {
        const double* lk = l + (size_t)(T - 1) * N + (size_t)k * M;
        double li = log_sum_exp(lk, M);
        for (int i = 0; i < M; ++i) {
            double v = lw1[(size_t)(T - 1) * m + k] - lz + lk[i] - li;
            dl[k * M + i] = (v > -INFINITY) ? exp(v) : 0.0;
        }
    }
    double thp[64], thm[64];
    for (int d = 0; d < d_theta; ++d) score[d] = 0.0;
    for (int t = T; t >= 1; --t) {
        const double* yt = y + (size_t)(t - 1) * dy;
        const double* xt = xs + (size_t)t * N * dx;
        const double* xprev = xs + (size_t)(t - 1) * N * dx;
        for (int g = 0; g < N; ++g) {
            if (dl[g] == 0.0) continue;
            /* the parent of particle g of time t among the time-(t-1) particles */
            const double* xp = (t == 1) ? xprev + (size_t)g * dx
                                        : xprev + (size_t)anc[(size_t)(t - 2) * N + g] * dx;
            for (int d = 0; d < d_theta; ++d) {
                double h = 1e-6 * (fabs(theta[d]) > 1.0 ? fabs(theta[d]) : 1.0);
                memcpy(thp, theta, sizeof(double) * d_theta);
                memcpy(thm, theta, sizeof(double) * d_theta);
                thp[d] += h;
                thm[d] -= h;
                model_t mp = { model, dx, dy, thp, mdat }, mm = { model, dx, dy, thm, mdat };
                double fp = log_f(&mp, (uint32_t)t, xp, xt + (size_t)g * dx) + log_g(&mp, yt, xt + (size_t)g * dx);
                double fm = log_f(&mm, (uint32_t)t, xp, xt + (size_t)g * dx) + log_g(&mm, yt, xt + (size_t)g * dx);
                if (t == 1) {
                    fp += log_mu(&mp, xp);
                    fm += log_mu(&mm, xp);
                }
                score[d] += dl[g] * (fp - fm) / (2.0 * h);
            }
        }
        if (t >= 2) {
            for (int g = 0; g < N; ++g) dlp[g] = 0.0;
            for (int g = 0; g < N; ++g) dlp[anc[(size_t)(t - 2) * N + g]] += dl[g];
            memcpy(dl, dlp, sizeof(double) * N);
        }
    }
    free(xs); free(lw1); free(l); free(dl); free(dlp);
    return 0;
}

/* log Z and the Fisher score of one run at theta (the run's own lineage). */
static int logz_and_score(int model, int dx, int dy, int m, int M, int T, int mode, double tau, uint64_t seed,
                          uint32_t chain, uint32_t iter, const double* theta, const double* mdat, const double* y,
                          int d_theta, double* lz, double* score)
{
    const int N = m * M;
    int32_t* anc = malloc(sizeof(int32_t) * (size_t)T * N);
    int32_t* sstar = malloc(sizeof(int32_t) * (size_t)T);
    int rc = oracle_airpf(model, dx, dy, m, M, T, mode, tau, seed, chain, iter, theta, mdat, y, lz, NULL, anc,
                          NULL, NULL, sstar, NULL, NULL);
    if (!rc)
        rc = oracle_fisher_score(model, dx, dy, m, M, T, seed, chain, iter, theta, mdat, y, anc, sstar, d_theta,
                                 score);
    free(anc);
    free(sstar);
    return rc;
}

/* Particle marginal Metropolis-Hastings with a Langevin proposal driven by the
 * Fisher score g of each likelihood estimate:
 *   theta'_d = theta_d + h_d^2 g_d(theta) / 2 + h_d eps_d   (h_d = step[d]; h_d = 0 keeps theta_d)
 * accepted iff log u < log Z' - log Z + log q(theta | theta') - log q(theta' | theta),
 * q the proposal's normal density (uniform box priors cancel inside the box).
 * Streams as oracle_pmmh (kind MH: eps from sub 0, u from sub 1 word 0); the
 * initial estimate (state_logz NaN) uses iter 0xffffffff and also sets state_grad. */
int oracle_pmmh_langevin(int model, int dx, int dy, int m, int M, int T, int mode, double tau, uint64_t seed,
                         uint32_t chain, const double* mdat, const double* y, int d_theta, const double* step,
                         const double* lo, const double* hi, double* theta, double* state_logz,
                         double* state_grad, uint32_t iter0, int iters, double* theta_out, double* logz_out,
                         int32_t* n_accept)
{
    double prop[64], gp[64], eps[64];
    if (d_theta < 1 || d_theta > 64) return 1;
    int acc = 0;
    if (isnan(*state_logz)) {
        int rc = logz_and_score(model, dx, dy, m, M, T, mode, tau, seed, chain, 0xffffffffu, theta, mdat, y,
                                d_theta, state_logz, state_grad);
        if (rc) return rc;
    }
    for (int j = 0; j < iters; ++j) {
        uint32_t it = iter0 + (uint32_t)j;
        stream_id st = { seed, chain, it };
        for (int b = 0; b < (d_theta + 1) / 2; ++b) {
            uint32_t w[4];
            draw(&st, (uint32_t)b, 0, KIND_MH, 0, w);
            double a, c;
            normal_pair(w[0], w[1], &a, &c);
            eps[2 * b] = a;
            if (2 * b + 1 < d_theta) eps[2 * b + 1] = c;
        }
        int inside = 1;
        double lqf = 0.0;
        for (int d = 0; d < d_theta; ++d) {
            double h = step[d];
            prop[d] = theta[d] + 0.5 * h * h * state_grad[d] + h * eps[d];
            if (h > 0.0) {
                lqf -= 0.5 * eps[d] * eps[d];
                if (!(prop[d] >= lo[d] && prop[d] <= hi[d])) inside = 0;
            }
        }
        if (inside && !oracle_model_valid(model, dx, prop)) inside = 0;
        if (inside) {
            double lz;
            int rc = logz_and_score(model, dx, dy, m, M, T, mode, tau, seed, chain, it, prop, mdat, y, d_theta,
                                    &lz, gp);
            if (rc) return rc;
            double lqr = 0.0;
            for (int d = 0; d < d_theta; ++d) {
                double h = step[d];
                if (h > 0.0) {
                    double e = (theta[d] - prop[d] - 0.5 * h * h * gp[d]) / h;
                    lqr -= 0.5 * e * e;
                }
            }
            uint32_t w[4];
            draw(&st, 0, 0, KIND_MH, 1, w);
            if (log(unif(w[0])) < lz - *state_logz + lqr - lqf) {
                memcpy(theta, prop, sizeof(double) * d_theta);
                memcpy(state_grad, gp, sizeof(double) * d_theta);
                *state_logz = lz;
                ++acc;
            }
        }
        if (theta_out) memcpy(theta_out + (size_t)j * d_theta, theta, sizeof(double) * d_theta);
        if (logz_out) logz_out[j] = *state_logz;
    }
    if (n_accept) *n_accept = acc;
    return 0;
}
