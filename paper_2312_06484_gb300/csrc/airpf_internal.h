// airpf_internal.h -- host/device parameter block of the AIRPF kernels and
// the launchers the C-ABI layer calls.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace airpf {

// split steps' group cascade: 2^kTailGroupLog CTA records per group (fewer when a
// filter has fewer CTAs)
constexpr int kTailGroupLog = 7;

// Per-run values the captured graph reads from device memory, so that one
// graph serves every (iter, chain0) and every PMMH iteration.
struct RunParams {
    uint32_t iter;
    uint32_t chain0;
};

// Everything the step kernel needs; passed by value.  Arrays are laid out
//   particles  X[b][d][k*M + i]   (structure of arrays, one island contiguous)
//   CTA records of the island weights, one per CTA j (islands j*G .. j*G+G-1):
//     pe[b][j]          largest binary exponent of the CTA's island weights
//     pt[b][j][2G]      the CTA's block-sum subtree, levels 0..g (g = log2 G),
//                       relative to 2^pe (double, or 64-bit fixed point)
//     pq[b][j][8]       per-level sums of squares of that subtree, levels 0..g-1
//   the cascade's result for step t+1: csum[b] (s*, largest exponent), cup[b]
//   (block sums of level s*-1 if above the CTAs), nsrc[b][k]
struct StepParams {
    int B, m, M, N, dx, dy, T, S, mode, model, fp64;
    double tau;
    double inv_M;                 // 1 / M
    float tau_f;                  // tau as float (FP32-mixed ENF test)
    float cdf_scale;              // 2^cdf_bits: fixed-point scale of the FP32-mixed CDF
    int cdf_bits;                 // 31 - ceil(log2 M)
    int G, tpi, ppt;              // islands per CTA, threads per island, particles per thread
    int lg_tpi;                   // log2 tpi
    int cta0, ncta, lg_ncta;      // island launches over CTAs cta0 .. cta0+ncta-1 of each filter (ncta 0: all)
    int theta_dim;
    uint32_t seed_lo, seed_hi;
    const RunParams* run;
    const double* theta;          // [B][theta_dim]
    const double* mdata;          // LGSSM: A then C
    const double* y;              // [T][dy]
    const int* active;            // [B] nonzero = run this filter (PMMH), or NULL
    void* mpar;                   // [B] model constants (written by the prologue)
    void* drift;                  // [T] per-step transition constant (NGM)
    unsigned* bar;                // [2] grid barrier: arrivals, generation
    unsigned* err;                // [1] nonzero after a timed-out wait
    int inject_stall;             // test hook (grid-persistent launch only)
    int pdl;                      // per-step launches: programmatic dependent launch
    int fused;                    // per-step launches: each CTA runs the previous step's cascade itself
    int split;                    // per-step launches with a group cascade kernel (NG x B CTAs)
    int wide;                     // fused steps: the instantiation with up to 128 registers a thread
                                  // (taken when the whole grid is one wave at its occupancy)
    void* utg;                    // [B][2NG] top tree of the last cascade (split steps)
    // split steps' group cascade: NG groups of 2^gs CTA records per filter; a ticket
    // per filter [B]; per group, double-buffered by step: exponent, block-sum subtree
    // of levels g .. g+gs [2^(gs+1)], sums of squares of levels 0 .. g+gs-1 [16]
    int NG, gs;
    unsigned* tick;
    int* ge[2];
    void* gtr[2];
    void* gqs[2];
    // gradient pass (record AIRPF_RECORD_GRAD): states x_t at checkpoints
    // (slot 0 = x_0, slot t/ckpt, and slot nck-1 = x_T when T is no multiple
    // of ckpt), the recomputed states between checkpoints, log W^k_{t,1}, the
    // island smoothing weights, the particle adjoints and descendant weights
    // (three rotating buffers each), and the two results
    int grad, ckpt, nck;
    void* xck;                    // [B][nck][dx][N]
    void* xblk;                   // [2][B][ckpt][N][dx]: blocks of even and odd index
    double* logw;                 // [B][T][m]
    // output measures (record AIRPF_RECORD_MOMENTS): per island and step, log W_{t,0} and
    // log W_{t,1}, and every warp's sums of x_d and x_d^2 over its mutated and its
    // internally resampled particles
    // adaptive internal resampling: on when tau_int > 0; lom holds log(M omega) of every
    // particle (0 after the island resampled), double-buffered like X
    int air;
    double tau_int;
    int rb;                       // radix bits: an r-ary stage is rb binary stages (1: binary)
    void* lom[2];                 // [B][N]
    int fmom, fm_nw;              // recording on; warps per island
    double* fw;                   // [B][T][m][2]
    double* fsum;                 // [B][T][m][fm_nw][4 dx]
    double* gpi[2];               // [B][m]
    void* xh[3];                  // [B][N][DX] particle adjoints (DX = 8 for the LGSSM, else 1)
    void* dh[3];                  // [B][N] descendant weights, the pass's precision
    double* gacc;                 // [B][m][2 kMaxTheta] the islands' running sums of the theta terms
    double* gout;                 // [B][theta_dim] adjoint gradient
    double* sout;                 // [B][theta_dim] Fisher score
    void* X[2];                   // particle stores, ping-pong by t & 1
    int P, g;                     // CTA records per filter (m / G) and log2 G
    int* pe[2];                   // CTA records, ping-pong by t & 1
    void* pt[2];
    void* pq[2];
    int* csum;                    // [B][4] last cascade: s*, largest exponent (INT_MIN: all zero)
    void* cup;                    // [B][P] upper-tree level s*-1 when it lies above the CTA level
    int* nsrc;                    // [B][m] inherited block of each island (written when s* > 1)
    int* ires[2];                 // internal ancestors of the last step (lineage), or NULL
    double* logz;                 // [B]
    double* trace;                // [B][T] or NULL
    double* enf;                  // [B][T][S+1] or NULL
    int* sstar;                   // [B][T] or NULL
    int* anc;                     // [B][T][N] or NULL
};

// Shared-memory bytes of one step launch.
size_t step_smem_bytes(const StepParams& p);

// Bytes of one filter's model constants.
size_t model_par_bytes();

// Sets kernel attributes (shared-memory opt-in); call outside stream capture.
cudaError_t prepare_step(const StepParams& p);

// Launches step t on `stream`: t = 0 the prologue (model constants), 1..T the
// island work of step t (each CTA publishes its record), T+1 the lineage of
// step T.
cudaError_t launch_step(const StepParams& p, int t, cudaStream_t stream);

// Launches the cascade of step t (one CTA per filter) on `stream`.
cudaError_t launch_cascade(const StepParams& p, int t, cudaStream_t stream);

// One launch running all T+1 steps: grid = cooperative launch over several
// CTAs per filter, otherwise one CTA per filter.  The prologue (t = 0 launch)
// must precede it.
cudaError_t launch_persistent(const StepParams& p, bool grid, cudaStream_t stream);

// Whether every CTA of the grid-persistent launch can be resident at once.
bool persistent_grid_fits(const StepParams& p);
// the output measures' moments of the last pass, out [B][T][2][2][dx]
cudaError_t launch_moments(const StepParams& p, double* out, cudaStream_t stream);
// can every CTA of a fused-steps grid be resident at once at the occupancy of
// the 128-register instantiation?
bool wide_fused_fits(const StepParams& p);

// Largest CTA of the one-CTA-per-filter launch.
int max_cta_threads();

// The backward pass of the gradient (after a recorded forward pass), enqueued
// on `stream`: every model but TOY (host_md: the LGSSM's A then C, row-major).
// Zeroes its accumulators first.
constexpr int kModelDataMax = 8 * 8 + 8 * 8;
// The backward pass, recorded into the capture of `stream`: the recomputation of the
// states of each block of ckpt steps runs on `aux` (forked from and joined back to
// `stream` through the kGradEvents events), one block ahead of the adjoint steps.
constexpr int kGradEvents = 5;
cudaError_t launch_grad_backward(const StepParams& p, const double* host_md, cudaStream_t stream, cudaStream_t aux,
                                 cudaEvent_t* ev);
bool grad_supported(int model);

// Writes the run parameters (one thread).
cudaError_t launch_set_run(RunParams* d_run, uint32_t iter, uint32_t chain0, cudaStream_t stream);

// Parameter block of the PMMH kernels (airpf_pmmh.cu); passed by value.
struct PmmhParams {
    int B, theta_dim, model, dx;
    uint32_t seed_lo, seed_hi, chain0;
    double step[16], lo[16], hi[16];     // random-walk scales and the prior box
    RunParams* run;                      // the pass's (iter, chain0)
    double* theta;                       // [B][theta_dim] the pass's parameters
    const double* logz;                  // [B] the pass's log Z
    int* active;                         // [B] which filters the pass runs
    double* state_theta;                 // [B][theta_dim] chain state
    double* state_logz;                  // [B]
    int* n_accept;                       // [B]
    double* theta_out;                   // [iters][B][theta_dim] or NULL
    double* logz_out;                    // [iters][B] or NULL
    // Langevin proposal: the score at the chain state and at the proposal, and
    // log q(proposal | state) up to its constant
    double* state_grad;                  // [B][theta_dim]
    const double* gprop;                 // [B][theta_dim]
    double* lqf;                         // [B]
};

// PMMH set-up of one pass (proposal, or the initial estimate of NaN log Z)
// and its conclusion (accept/reject, outputs of iteration j).
cudaError_t launch_pmmh_propose(const PmmhParams& q, uint32_t iter, int initial, cudaStream_t stream);
cudaError_t launch_pmmh_accept(const PmmhParams& q, uint32_t iter, int j, int initial, cudaStream_t stream);
cudaError_t launch_lmh_propose(const PmmhParams& q, uint32_t iter, int initial, cudaStream_t stream);
cudaError_t launch_lmh_accept(const PmmhParams& q, uint32_t iter, int j, int initial, cudaStream_t stream);

// Message for airpf_last_error(NULL) (calls without a context), printf-style.
void set_create_error(const char* fmt, ...);

}  // namespace airpf

struct airpf_ctx;
namespace airpf {
// The stream a context enqueues on (for the batch runner).
cudaStream_t ctx_stream(const airpf_ctx* ctx);

// Choose (tpi, ppt, G) for M particles per island and m islands per filter;
// want_ppt / want_g of 0 take the defaults.
void choose_mapping(int m, int M, int fp64, int want_ppt, int want_g, int* tpi, int* ppt, int* G);

}  // namespace airpf
