/*
 * airpf.h -- C ABI of the GB300 (sm_103a) Augmented Island Resampling Particle
 * Filter library.
 *
 * The method is Algorithm 1 of K. Heine, "Augmented Island Resampling Particle
 * Filters for Particle Markov Chain Monte Carlo" (arXiv 2312.06484): m filters
 * ("islands") of M particles each; every time step weights the particles by
 * the observation density g_t (Algorithm 1, weighting), resamples M particles
 * multinomially inside each island (internal resample), then runs S = log2 m
 * interaction stages with the butterfly matrices A_s of eq. (3), each stage
 * active only while the effective number of filters (ENF) is below tau
 * (Algorithm 1, adaptation), and mutates through K_{t+1}.  The estimate
 * Z^N_T = m^-1 sum_k W^k_T of the marginal likelihood (Section 2,
 * gamma^N_n(1)) is unbiased (Theorem 1), which is what particle marginal
 * Metropolis-Hastings consumes (Section 1.2, Andrieu et al. 2010).
 *
 * Conventions for every entry point:
 *   - All pointers named d_* are DEVICE pointers; all others are host pointers.
 *   - The caller owns every input and output buffer and the device workspace.
 *     The library owns only the host-side context object.
 *   - Work is enqueued asynchronously on the stream given to airpf_create
 *     (a cudaStream_t passed as void*; NULL = legacy default stream), except
 *     where a function says it synchronises.
 *   - Arguments are checked before anything is launched; failures return a
 *     status code and leave a message for airpf_last_error.  The library never
 *     aborts or exits.
 *   - A context is not thread-safe: one host thread at a time per context.
 *   - log Z = -inf is a valid result (every particle weight became zero).
 *
 * Random numbers: counter-based Philox4x32-10 (Salmon et al., SC'11) with
 *   key = (seed & 0xffffffff, seed >> 32),
 *   counter = (unit, t, iter, ((chain0 + b) << 8) | (kind << 5) | sub)
 * for filter b of a batch, with kind 0 (prior draw of particle unit = k*M+i,
 * t = 0), 1 (transition noise of unit k*M+i at time t, normal pair `sub`;
 * word 2 of sub 0 drives internal-resampling draw i of island k), 2 (island
 * choice of island unit = j at stage sub = s, time t) and 3 (PMMH proposal
 * and acceptance).  uniform(w) = (w + 0.5) 2^-32; normals by Box-Muller.
 * Runs are therefore reproducible bit for bit given (seed, chain, iter) and
 * independent of the launch configuration.
 */
#ifndef AIRPF_H
#define AIRPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AIRPF_OK = 0,
    AIRPF_ERR_ARG = 1,          /* invalid argument (nothing was launched) */
    AIRPF_ERR_CUDA = 2,         /* a CUDA call failed; see airpf_last_error */
    AIRPF_ERR_WORKSPACE = 3,    /* workspace too small or misaligned */
    AIRPF_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
    AIRPF_ERR_UNSUPPORTED = 5   /* valid but not supported by this build */
} airpf_status;

/* State-space models (Section 1.2, eq. (1)).  theta layouts:
 *   AR1   [a, sigma_v, sigma_w, sigma_0]
 *   SV    [mu, phi, sigma]
 *   NGM   [q, r, p0]                       (variances)
 *   LGSSM [A_11..A_dd, log q, log r]       model_data = A (dx*dx), C (dy*dx), row-major
 *   TOY   [p_stay, p_correct]              binary HMM of Section 4.1
 *   CP    [p, alpha, beta]                 change-point model of Section 4.2: x_0 ~ Beta(alpha,
 *                                          beta), x jumps w.p. p to a fresh Beta(alpha, beta)
 *                                          draw; y_t = (k_t, n_t), k_t ~ Binomial(n_t, x_t);
 *                                          dx = 1, dy = 2; no gradient (the jump is discrete) */
typedef enum {
    AIRPF_MODEL_AR1 = 0,
    AIRPF_MODEL_SV = 1,
    AIRPF_MODEL_NGM = 2,
    AIRPF_MODEL_LGSSM = 3,
    AIRPF_MODEL_TOY = 4,
    AIRPF_MODEL_CP = 5
} airpf_model;

/* Interaction rule of Algorithm 1, adaptation line: NEVER gives m independent
 * bootstrap filters (alpha_s = I, Section 3), ALWAYS uses every A_s, ADAPTIVE
 * uses A_s iff ENF_{t,s} < tau. */
typedef enum {
    AIRPF_INTERACT_NEVER = 0,
    AIRPF_INTERACT_ALWAYS = 1,
    AIRPF_INTERACT_ADAPTIVE = 2
} airpf_interact;

/* FP64: every particle computation in double.  FP32_MIXED: propagation,
 * log-weights and the island log-sum-exp in float, internal-resampling CDF as
 * an exact fixed-point integer prefix sum; island weights (unnormalised, as
 * in Algorithm 1, with an integer binary exponent for range), their sums
 * (exact fixed point) and log Z in double. */
typedef enum {
    AIRPF_FP64 = 0,
    AIRPF_FP32_MIXED = 1
} airpf_precision;

/* How a pass over y_1..y_T is launched.  AUTO picks PERSISTENT_CTA when a
 * whole filter fits one CTA (m * threads-per-island <= 512), else STEPS.
 * STEPS: one launch per time step, replayed from a CUDA graph; each CTA
 * first runs the interaction cascade of the previous step from the per-CTA
 * summaries of the island weights, then its islands' step.  STEPS_SPLIT: the
 * cascade runs as a second kernel per step with one CTA per filter (AUTO
 * takes it when a filter spans more than 512 CTAs, where every CTA reading
 * every summary would cost more).  Consecutive per-step kernels overlap their
 * start with programmatic dependent launch.
 * PERSISTENT_CTA: one launch for all steps, one CTA per filter.
 * PERSISTENT_GRID: one cooperative launch for all steps, a bounded grid
 * barrier (1 s) between steps; a timed-out wait is reported by airpf_sync. */
typedef enum {
    AIRPF_LAUNCH_AUTO = 0,
    AIRPF_LAUNCH_STEPS = 1,
    AIRPF_LAUNCH_PERSISTENT_CTA = 2,
    AIRPF_LAUNCH_PERSISTENT_GRID = 3,
    AIRPF_LAUNCH_STEPS_SPLIT = 4
} airpf_launch;

typedef struct {
    int32_t model;          /* airpf_model */
    int32_t dx, dy;         /* state / observation dimension (1 unless LGSSM; dx <= 8, dy <= 8) */
    int32_t m;              /* islands per filter: a power of 2, 1..65536 */
    int32_t M;              /* particles per island: 1..1024 */
    int32_t T;              /* observations y_1..y_T, T >= 1 */
    int32_t B;              /* filters run together (a batch of independent runs), >= 1 */
    int32_t mode;           /* airpf_interact */
    double tau;             /* ENF threshold in (0, 1] (ENF normalised to [1/m, 1]) */
    int32_t precision;      /* airpf_precision */
    int32_t record;         /* bit 0: ancestors, bit 1: ENF and s*, bit 2: log Z trace, bit 3: kernel timing,
                               bit 4: gradient pass, bit 5: output measures (airpf_moments) */
    uint64_t seed;
    int32_t launch;         /* airpf_launch (a requested mode that cannot run: AIRPF_ERR_UNSUPPORTED) */
    int32_t reserved;       /* must be 0 */
    int32_t ppt;            /* particles per thread: 2, 4 or 8 (8: FP32 SV and NGM only), 0 =
                             * automatic (8 for FP32 SV and NGM split steps with M = 256, else 4
                             * above M = 64 and 2 up to it) */
    int32_t islands_per_cta;/* islands per CTA: a power of 2, 0 = automatic (capped at 512 threads) */
    int32_t ckpt;           /* AIRPF_RECORD_GRAD: states kept every ckpt steps, recomputed in
                               between during the backward pass (0 = every step) */
    double tau_int;         /* adaptive internal resampling (the remark after Algorithm 1): 0 = every
                               island resamples at every step (Algorithm 1 as printed); in (0, 1], island
                               k resamples at step t only when the ESS of its particle weights
                               w_i = omega_i g_t(x_i), (sum w)^2 / sum w^2, is below tau_int M, and
                               otherwise keeps its particles with omega_i = w_i / sum w; then
                               W_{t,1} = W_{t,0} sum_i omega_i g_t(x_i) (M^-1 sum_i g_t(x_i) when
                               omega = 1/M).  Not with AIRPF_RECORD_GRAD or AIRPF_RECORD_MOMENTS, nor
                               with airpf_run_static (AIRPF_ERR_UNSUPPORTED). */
    int32_t radix;          /* islands averaged per interaction stage, r = 2^b (0 or 2: the paper's
                               binary stages; Section 2 allows any r with m a power of r); m must be a
                               power of r.  There are S_r = log_r m stages; stage s averages aligned
                               groups of r islands (A_s = I (x) r^-1 1_r (x) I) and each island draws,
                               from its own uniform, one member of its group with probability
                               proportional to the members' weights, independently of the other
                               islands.  ENF records and s* count these S_r stages */
} airpf_config;

#define AIRPF_RECORD_LINEAGE 1
#define AIRPF_RECORD_ENF 2
#define AIRPF_RECORD_TRACE 4
#define AIRPF_RECORD_TIMING 8   /* STEPS launch only: CUDA events around each kernel (airpf_kernel_times) */
#define AIRPF_RECORD_GRAD 16    /* keep what airpf_grad's backward pass needs (all models but TOY and CP) */
#define AIRPF_RECORD_MOMENTS 32 /* keep what airpf_moments needs (the output measures' island terms) */

typedef struct airpf_ctx airpf_ctx;

/* Number of bytes of device workspace a context with this configuration needs.
 * Returns AIRPF_ERR_ARG for an invalid configuration. */
airpf_status airpf_workspace_bytes(const airpf_config* cfg, size_t* bytes);

/* Creates a context.  d_workspace: caller-owned device memory of at least
 * airpf_workspace_bytes(cfg) bytes, 256-byte aligned, kept alive until
 * airpf_destroy.  model_data: host array (LGSSM: dx*dx + dy*dx doubles; may be
 * NULL otherwise), copied.  stream: cudaStream_t as void*.  *out receives the
 * context (NULL on failure). */
airpf_status airpf_create(const airpf_config* cfg, void* d_workspace, size_t workspace_bytes,
                          const double* model_data, void* stream, airpf_ctx** out);

airpf_status airpf_destroy(airpf_ctx* ctx);

/* One AIRPF pass over y_1..y_T for each of the B filters (Algorithm 1).
 *   d_theta   [B * d_theta] model parameters of filter b at b*d_theta (FP64)
 *   d_y       [T * dy] observations, row t-1 = y_t (FP64)
 *   chain0    chain index of filter 0 (filter b uses chain0 + b; < 2^24)
 *   iter      iteration index of the random streams
 *   d_log_z   [B] out: log Z^N_T (FP64)
 *   d_anc     [B * T * N] out or NULL: int32 parent index (0..N-1, among the
 *             time-t particles) of particle k*M+i held after step t, t = 1..T
 *             (needs AIRPF_RECORD_LINEAGE)
 *   d_enf     [B * T * (S_r+1)] out or NULL: ENF_{t,0..S_r} (needs AIRPF_RECORD_ENF);
 *             S_r = log2 m, or log_r m with radix r
 *   d_sstar   [B * T] out or NULL: first non-interacting stage (S_r+1 = all interact)
 *   d_trace   [B * T] out or NULL: log Z^N_t after step t (needs AIRPF_RECORD_TRACE)
 * Asynchronous on the context's stream. */
airpf_status airpf_run(airpf_ctx* ctx, const double* d_theta, const double* d_y,
                       uint32_t chain0, uint32_t iter, double* d_log_z, int32_t* d_anc,
                       double* d_enf, int32_t* d_sstar, double* d_trace);

/* airpf_run with host buffers: copies theta (B*d_theta) and y (T*dy) to the
 * device, runs, copies log_z (B) back, and synchronises the stream before
 * returning.  For callers without device memory of their own. */
airpf_status airpf_run_host(airpf_ctx* ctx, const double* theta, const double* y,
                            uint32_t chain0, uint32_t iter, double* log_z);

/* Stepwise passes: the caller drives the steps of one pass, so that the islands of one
 * filter can be split over G processes, one GPU each (Section 2 lets the m islands of a
 * filter run in parallel; the interaction stages are the only coupling): every process
 * holds the whole filter's buffers, runs the island work of its own contiguous range of
 * CTAs (m/G islands), exchanges the step's CTA records and particle rows with the others
 * (an all-gather of airpf_step_regions), and runs the step's cascade over all records,
 * which every process then holds identically.  For one filter (B = 1), without records or
 * adaptive internal resampling, with per-step launches (AIRPF_LAUNCH_STEPS or
 * AIRPF_LAUNCH_STEPS_SPLIT); otherwise AIRPF_ERR_UNSUPPORTED.  Asynchronous on the context's
 * stream.  A pass:
 *   airpf_step_begin; for t = 1..T: airpf_step_islands(t, own range), exchange,
 *   airpf_step_cascade(t); airpf_step_end.
 * The result equals airpf_run's for the same (chain0, iter).  Split steps may defer the
 * exchange of the particle rows until after the cascade and skip it when the step's
 * interacting stages all lie inside one process's islands (airpf_step_levels): with
 * contiguous ranges of m/G islands, stage s pairs islands 2^(s-1) apart, so only the
 * top log2 G binary stages cross processes. */

/* Copies theta (d_theta_dim doubles) and y (T*dy) in and runs the pass's prologue. */
airpf_status airpf_step_begin(airpf_ctx* ctx, const double* d_theta, const double* d_y,
                              uint32_t chain0, uint32_t iter);

/* Island work of step t (1..T, Algorithm 1's weighting, internal resampling and mutation of
 * step t, and the cascade of step t-1 in fused steps) for CTAs cta0 .. cta0+ncta-1 of the
 * filter: ncta a power of 2 dividing cta0 (0: all CTAs).  The filter has m/G CTAs of G
 * islands (airpf_step_regions gives their records' sizes). */
airpf_status airpf_step_islands(airpf_ctx* ctx, int32_t t, int32_t cta0, int32_t ncta);

/* The cascade of step t (interaction stages, s*, log Z) over all CTA records: the cascade
 * kernel of split steps; fused steps run it at the next island launch (and, for t = T, in a
 * launch of their own here). */
airpf_status airpf_step_cascade(airpf_ctx* ctx, int32_t t);

/* Copies log Z^N_T (one double) to d_log_z. */
airpf_status airpf_step_end(airpf_ctx* ctx, double* d_log_z);

/* The device regions that step t's island launch writes and the other processes need, as
 * byte offsets into the context's workspace and sizes: the CTA records (exponents, block-sum
 * subtrees, sums of squares) and the particle rows of each state dimension.  Each region is
 * laid out by CTA (or island) in order, so CTA range [j n, (j+1) n) owns the j-th of
 * (regions bytes / n CTAs) equal parts.  offsets, bytes: arrays of at least 3 + dx entries;
 * *count receives the number of regions. */
airpf_status airpf_step_regions(airpf_ctx* ctx, int32_t t, size_t* offsets, size_t* bytes, int32_t* count);

/* Split steps: waits for the stream, then gives the number of binary interaction levels
 * of the last cascade (s* - 1 in binary stages; 0 if no stage interacted, log2 m if all
 * did).  The island CTAs of the next step read particle rows of islands at most
 * 2^levels - 1 apart.  Fused steps: AIRPF_ERR_UNSUPPORTED (their cascade runs inside the
 * next island launch, so the rows are exchanged every step). */
airpf_status airpf_step_levels(airpf_ctx* ctx, int32_t* levels);

/* Size of the device scratch of airpf_run_static: a fixed device array inside
 * the library, which CUDA allocates when the library's module loads on a device. */
#define AIRPF_STATIC_SCRATCH_BYTES ((size_t)32 << 20)

/* One AIRPF pass, as airpf_run, with no context, no workspace and no device
 * allocation of any kind.  No counterpart in the paper: it is for callers that
 * cannot allocate device memory where they need a likelihood estimate -- there
 * cudaMalloc/cudaFree would stall other work (cudaFree waits for the whole
 * device) or break the caller's own rule (a serving loop with a fixed memory
 * budget, a pool allocator that owns all device memory, a callback that must
 * not block) -- and that have no spare device buffer to lend as workspace.
 * The pass runs on a static scratch of AIRPF_STATIC_SCRATCH_BYTES per device;
 * nothing in it needs to start at zero (each pass writes every word it reads).
 *   cfg           as for airpf_create; record must be 0; launch AUTO, STEPS or
 *                 PERSISTENT_CTA, with the default tiling (ppt = islands_per_cta = 0);
 *                 PERSISTENT_GRID, STEPS_SPLIT, a tiling request, tau_int > 0, or a
 *                 step needing more than 227 KB of shared memory: AIRPF_ERR_UNSUPPORTED
 *   d_theta       [B * d_theta] device, read in place
 *   d_y           [T * dy] device, read in place
 *   d_model_data  LGSSM: device array A (dx*dx) then C (dy*dx); else NULL
 *   chain0, iter  as for airpf_run
 *   d_log_z       [B] out (device)
 *   stream        cudaStream_t as void*
 * A configuration whose scratch would exceed AIRPF_STATIC_SCRATCH_BYTES returns
 * AIRPF_ERR_WORKSPACE before any work (airpf_last_error(NULL) states both
 * sizes); give it a context with its own workspace instead.  The first call on
 * each device does a one-time set-up (it looks up the scratch address, which
 * also loads the library's module onto that device); make it before any stream
 * capture.  The address is kept for the life of the process: a cudaDeviceReset
 * (or any teardown of the device's primary context) voids it, so do not call
 * airpf_run_static on a device after resetting it.  Calls that overlap in time on one device (different streams, or
 * host threads without ordering between them) share the scratch and race:
 * order them on one stream or with events.  Asynchronous on `stream`; failures
 * leave their message for airpf_last_error(NULL). */
airpf_status airpf_run_static(const airpf_config* cfg, const double* d_theta, const double* d_y,
                              const double* d_model_data, uint32_t chain0, uint32_t iter,
                              double* d_log_z, void* stream);

/* Random-walk particle marginal Metropolis-Hastings, one chain per filter of
 * the batch (Andrieu et al. 2010; AIRPF is valid inside it by Theorem 1).
 * Proposal theta' = theta + step .* N(0, I); independent uniform priors on
 * [lo_d, hi_d] for every component with step_d > 0 (components with step_d = 0
 * stay fixed); a proposal outside the box or outside the model's parameter
 * domain is rejected without running its filter (its CTAs skip the pass).
 * Iteration j draws its proposal and acceptance uniform from kind-3 streams
 * with iter = iter0 + j (see the random-number convention above) and runs the
 * filter with that iter; u < exp(log Z' - log Z) accepts.
 *   d_y            [T * dy] observations (FP64)
 *   step, lo, hi   host arrays [d_theta]
 *   d_state_theta  [B * d_theta] in/out: current theta of each chain
 *   d_state_logz   [B] in/out: log Z of the current theta; NaN = not yet
 *                  estimated (estimated first with iter = 0xffffffff)
 *   chain0         chain of filter 0 (filter b is chain chain0 + b)
 *   iter0, iters   iterations iter0 .. iter0+iters-1 (iter0 + iters < 2^32 - 1);
 *                  a chain resumes by calling again with the next iter0
 *   d_theta_out    [iters * B * d_theta] out or NULL: chain state after
 *                  iteration j at row j*B + b
 *   d_logz_out     [iters * B] out or NULL
 *   d_n_accept     [B] in/out: accepted proposals (int32), added to
 * Asynchronous on the context's stream; the whole chain stays on the device.
 * Per iteration, and once more for the initial estimate, it enqueues two
 * one-thread-per-chain kernels around one filter pass. */
airpf_status airpf_pmmh(airpf_ctx* ctx, const double* d_y, const double* step, const double* lo,
                        const double* hi, double* d_state_theta, double* d_state_logz,
                        uint32_t chain0, uint32_t iter0, int32_t iters, double* d_theta_out,
                        double* d_logz_out, int32_t* d_n_accept);

/* ---- Batches of uneven size and the tiling autotuner ----
 * Chains whose (m, M) differ run as a group: one context per size class (its
 * chains are the filters of that context's batch, each with its own theta),
 * each context created on a stream of its own.  The group forks every member
 * stream from `stream` with an event, enqueues each member's work on its own
 * stream, and joins them back, so the classes' kernels run side by side and
 * the caller sees one asynchronous operation on `stream`.  The contexts stay
 * owned by the caller and must outlive the group. */
typedef struct airpf_group airpf_group;

airpf_status airpf_group_create(airpf_ctx* const* ctxs, int32_t n, void* stream, airpf_group** out);
airpf_status airpf_group_destroy(airpf_group* g);

/* airpf_run for every member i with d_theta[i], chain0[i], d_log_z[i] and the
 * shared observations d_y (record outputs are not taken here). */
airpf_status airpf_group_run(airpf_group* g, const double* const* d_theta, const double* d_y,
                             const uint32_t* chain0, uint32_t iter, double* const* d_log_z);

/* airpf_pmmh for every member i (state, chain0, outputs and acceptance
 * counters per member; d_theta_out and d_logz_out may be NULL, as may their
 * entries), same proposal and prior for all. */
airpf_status airpf_group_pmmh(airpf_group* g, const double* d_y, const double* step, const double* lo,
                              const double* hi, double* const* d_state_theta, double* const* d_state_logz,
                              const uint32_t* chain0, uint32_t iter0, int32_t iters,
                              double* const* d_theta_out, double* const* d_logz_out,
                              int32_t* const* d_n_accept);

/* PMMH with a Langevin proposal (the differentiation workload's sampler; the
 * paper's PMMH with a gradient-driven proposal): for a context created with
 * AIRPF_RECORD_GRAD, each iteration proposes
 *   theta'_d = theta_d + step_d^2 g_d(theta) / 2 + step_d eps_d,
 * g the Fisher-identity score of the chain's current estimate (airpf_grad),
 * runs the gradient pass at theta', and accepts iff
 *   log u < log Z' - log Z + log q(theta | theta') - log q(theta' | theta)
 * (q the proposal's normal density; uniform box priors [lo, hi] cancel inside
 * the box; a proposal outside the box or the model's domain is rejected).
 * eps and u come from the same kind-3 stream words as airpf_pmmh.
 *   d_state_grad  [B * d_theta] in/out: score at the current theta; set by the
 *                 initial estimate when d_state_logz is NaN
 * The other arguments as for airpf_pmmh.  Asynchronous. */
airpf_status airpf_pmmh_langevin(airpf_ctx* ctx, const double* d_y, const double* step, const double* lo,
                                 const double* hi, double* d_state_theta, double* d_state_logz,
                                 double* d_state_grad, uint32_t chain0, uint32_t iter0, int32_t iters,
                                 double* d_theta_out, double* d_logz_out, int32_t* d_n_accept);

/* airpf_sync of every member, then waits for `stream`. */
airpf_status airpf_group_sync(airpf_group* g);

/* Tiling autotuner (no counterpart in the paper).  Times `passes` passes of
 * each candidate tiling of cfg -- particles per thread {2, 4} x islands per
 * CTA {1, 2, 4, 8, 16} (up to 512 threads) x {STEPS, STEPS_SPLIT}, plus
 * PERSISTENT_CTA when a filter fits one CTA; candidates with the same actual
 * mapping are timed once -- after one warm-up pass each, with CUDA events on
 * `stream`, and returns in *best the configuration of the fastest (cfg with
 * launch, ppt and islands_per_cta set) and its milliseconds per pass.
 * d_workspace must hold airpf_workspace_bytes(cfg) rounded up to 256, plus
 * 8*B bytes (the timed passes' log Z).  Synchronises.  The tiling does not
 * change what a pass computes, only how fast. */
airpf_status airpf_autotune(const airpf_config* cfg, void* d_workspace, size_t workspace_bytes,
                            const double* model_data, const double* d_theta, const double* d_y,
                            int32_t passes, void* stream, airpf_config* best, float* best_ms);

/* Waits for the context's stream and reports device-side failures of the
 * work enqueued so far: AIRPF_ERR_TIMEOUT if a bounded grid-barrier wait ran
 * out (the results of that pass are invalid; the context stays usable),
 * AIRPF_ERR_CUDA for a CUDA error. */
airpf_status airpf_sync(airpf_ctx* ctx);

/* Gradient of log Z^N_T with respect to theta for each filter (AR1, SV, NGM, LGSSM;
 * a context created with AIRPF_RECORD_GRAD).  Runs the pass (as airpf_run,
 * writing d_log_z), then a backward pass over t = T..1 that needs the pass's
 * lineage, s*, island log-weights and the states kept every `ckpt` steps
 * (states in between are recomputed from the regenerated noise):
 *   d_grad   [B * d_theta] out or NULL: the adjoint gradient of log Z with the
 *            random numbers, ancestors, island choices and s* held fixed (the
 *            reparameterisation gradient; biased for the gradient of log Z
 *            itself, exact for the function a fixed lineage defines)
 *   d_score  [B * d_theta] out or NULL: the Fisher-identity score along the
 *            lineages, sum over particles of the final weight of their
 *            descendants times grad_theta log [f(x_t | parent) g(y_t | x_t)]
 *            (plus the prior's term), which estimates grad log Z consistently
 * At least one of them.  theta layouts as for the models above.  Asynchronous
 * on the context's stream. */
airpf_status airpf_grad(airpf_ctx* ctx, const double* d_theta, const double* d_y, uint32_t chain0,
                        uint32_t iter, double* d_log_z, double* d_grad, double* d_score);

/* Measurement aid, no counterpart in the paper.  For a context created with
 * AIRPF_RECORD_TIMING (which puts CUDA event-record nodes before and after each
 * kernel of steps 1..T into the pass's graph): waits for the stream and
 * returns the summed durations, in milliseconds, of the T island-step kernels
 * and of the T cascade kernels (0 when every CTA runs the cascade itself) of
 * the last airpf_run.  AIRPF_ERR_UNSUPPORTED
 * for a context without the flag. */
airpf_status airpf_kernel_times(airpf_ctx* ctx, double* step_ms, double* cascade_ms);

/* The airpf_launch mode the context resolved to (never AUTO). */
/* The output measures of the last airpf_run (the paper's output-measure equation,
 * Section 2): pi^N_{t,s} = sum_k W^k_{t,s} M^-1 sum_i delta(xi^{k,i}_{t,s}) / sum_k W^k_{t,s}
 * at s = 0 (the prediction filter: the mutated particles of step t with the island weights
 * before weighting with y_t) and s = 1 (the filter: the internally resampled particles with
 * the weights after it).  d_moments (device, caller-owned, B*T*2*2*dx doubles) receives
 * [b][t][s][0][d] = E[x_d] and [b][t][s][1][d] = E[x_d^2]; NaN where every island weight is
 * 0.  Needs a context created with AIRPF_RECORD_MOMENTS (else AIRPF_ERR_UNSUPPORTED);
 * asynchronous on the context's stream, after the run it describes. */
airpf_status airpf_moments(airpf_ctx* ctx, double* d_moments);

int32_t airpf_launch_mode(const airpf_ctx* ctx);

/* The context's island-to-thread mapping (no counterpart in the paper): threads per island,
 * particles per thread and islands per CTA, written to the three host int32 pointers.
 * AIRPF_ERR_ARG for a NULL context or pointer. */
airpf_status airpf_tiling(const airpf_ctx* ctx, int32_t* threads_per_island, int32_t* particles_per_thread,
                          int32_t* islands_per_cta);

/* Fault injection for tests of the failure path, no counterpart in the paper.
 * what = 1: in the next PERSISTENT_GRID pass, CTA 0 leaves before the first
 * grid barrier, so the other CTAs' bounded wait runs out after about a second
 * and airpf_sync returns AIRPF_ERR_TIMEOUT.  what = 0 clears it.  Returns
 * AIRPF_ERR_UNSUPPORTED for other launch modes. */
airpf_status airpf_debug_inject(airpf_ctx* ctx, int32_t what);

/* Test hook, no counterpart in the paper: d_y[i] = f(d_x[i]) for i < n as the FP64 path
 * computes f (table-driven double functions): fn = 0 the exponential, fn = 1 the natural
 * logarithm, fn = 2 and 3 sin(2 pi x) and cos(2 pi x) (the Box-Muller angle); of a 32-bit
 * word w = x (an integer 0 .. 2^32 - 1 given as a double): fn = 4 the uniform (w + 1/2) 2^-32,
 * fn = 5 its logarithm, fn = 6 and 7 the sine and cosine of 2 pi times it (the forms the
 * Box-Muller pairs use, reduced in integers).  Device arrays of n doubles, asynchronous on `stream` (a cudaStream_t, NULL for
 * the default stream).  AIRPF_ERR_ARG for another fn, n < 0 or a NULL array with n > 0. */
airpf_status airpf_debug_math(int32_t fn, const double* d_x, double* d_y, int64_t n, void* stream);

/* Number of model parameters for (model, dx); 0 for an unknown model. */
int32_t airpf_theta_dim(int32_t model, int32_t dx);

/* Kernels launched by the last airpf_run / airpf_pmmh call (for accounting). */
int64_t airpf_last_launch_count(const airpf_ctx* ctx);

/* Message of the last failure on this context (or of the last failed
 * airpf_create when ctx is NULL).  Never NULL. */
const char* airpf_last_error(const airpf_ctx* ctx);

/* Static string naming a status code. */
const char* airpf_status_string(airpf_status s);

#ifdef __cplusplus
}
#endif

#endif /* AIRPF_H */
