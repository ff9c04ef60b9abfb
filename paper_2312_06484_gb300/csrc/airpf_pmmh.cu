// airpf_pmmh.cu -- device side of particle marginal Metropolis-Hastings
// (Andrieu et al. 2010, the use of Z^N_T in Section 1.2; AIRPF qualifies by the
// unbiasedness of Theorem 1).  One chain per filter of the batch.  Between two
// filter passes the proposal, the prior-support test and the accept/reject
// decision run on the device, so a chain never leaves the GPU and an iteration
// costs two one-thread-per-chain kernels on top of the pass.
//
// Random streams (kind MH, t = 0, counter word 2 = the iteration):
//   proposal normals  unit = pair index q, sub 0: N(0,1) pair for components 2q, 2q+1
//   acceptance        unit 0, sub 1, word 0: u; accept iff log u < log Z' - log Z
// Uniform priors on a box cancel in the Metropolis-Hastings ratio, so inside
// the box the ratio is the ratio of the two likelihood estimates.
#include "airpf_device.cuh"
#include "airpf_internal.h"

namespace airpf {

// Domain of each model's parameters (theta layouts in the public header):
// positive scales and variances, a stationary SV volatility, probabilities in
// (0, 1), finite log noise scales for the LGSSM.
__device__ bool theta_in_domain(int model, int dx, const double* th)
{
    switch (model) {
    case AR1: return th[1] > 0.0 && th[2] > 0.0 && th[3] > 0.0;
    case SV: return fabs(th[1]) < 1.0 && th[2] > 0.0;
    case NGM: return th[0] > 0.0 && th[1] > 0.0 && th[2] > 0.0;
    case TOY: return th[0] > 0.0 && th[0] < 1.0 && th[1] > 0.0 && th[1] < 1.0;
    case LGSSM: return isfinite(th[dx]) && isfinite(th[dx + 1]);
    case CP: return th[0] >= 0.0 && th[0] <= 1.0 && th[1] > 0.0 && th[2] > 0.0;
    }
    return false;
}

// Pass set-up for every chain b: with initial != 0, the pass estimates log Z
// of the current theta of the chains whose log Z is NaN; otherwise it
// estimates log Z of the proposal, unless the proposal leaves the prior box
// or the model's domain.  active[b] = whether filter b runs.
__global__ void pmmh_propose_kernel(PmmhParams q, uint32_t iter, int initial)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) {
        q.run->iter = iter;
        q.run->chain0 = q.chain0;
    }
    if (b >= q.B) return;
    const int td = q.theta_dim;
    const double* cur = q.state_theta + (size_t)b * td;
    double* prop = q.theta + (size_t)b * td;
    int go;
    if (initial) {
        for (int d = 0; d < td; ++d) prop[d] = cur[d];
        go = isnan(q.state_logz[b]) ? 1 : 0;
    } else {
        const Stream st{q.seed_lo, q.seed_hi, iter, (q.chain0 + (uint32_t)b) << 8};
        bool inside = true;
        for (int pq = 0; 2 * pq < td; ++pq) {
            const U4 w = st.draw((uint32_t)pq, 0u, KIND_MH, 0u);
            double z[2];
            normal_pair(w.x, w.y, z[0], z[1]);
            for (int h = 0; h < 2; ++h) {
                const int d = 2 * pq + h;
                if (d >= td) break;
                prop[d] = cur[d] + q.step[d] * z[h];
                if (q.step[d] > 0.0 && !(prop[d] >= q.lo[d] && prop[d] <= q.hi[d])) inside = false;
            }
        }
        if (inside && !theta_in_domain(q.model, q.dx, prop)) inside = false;
        go = inside ? 1 : 0;
    }
    q.active[b] = go;
}

// After the pass: the initial estimate is stored, or the proposal accepted or
// rejected; iteration j's chain state goes to the optional outputs.
__global__ void pmmh_accept_kernel(PmmhParams q, uint32_t iter, int j, int initial)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= q.B) return;
    const int td = q.theta_dim;
    if (initial) {
        if (q.active[b]) q.state_logz[b] = q.logz[b];
        return;
    }
    double* cur = q.state_theta + (size_t)b * td;
    if (q.active[b]) {
        const Stream st{q.seed_lo, q.seed_hi, iter, (q.chain0 + (uint32_t)b) << 8};
        const U4 w = st.draw(0u, 0u, KIND_MH, 1u);
        const double lz = q.logz[b];
        if (log(unif_f64(w.x)) < lz - q.state_logz[b]) {
            const double* prop = q.theta + (size_t)b * td;
            for (int d = 0; d < td; ++d) cur[d] = prop[d];
            q.state_logz[b] = lz;
            q.n_accept[b] += 1;
        }
    }
    if (q.theta_out)
        for (int d = 0; d < td; ++d) q.theta_out[((size_t)j * q.B + b) * td + d] = cur[d];
    if (q.logz_out) q.logz_out[(size_t)j * q.B + b] = q.state_logz[b];
}

// Langevin proposal for every chain b (the score g of the current estimate
// drives it): theta'_d = theta_d + h_d^2 g_d / 2 + h_d eps_d, h_d = step[d]
// (h_d = 0 keeps theta_d); eps from the same stream words as the random walk.
// log q(theta' | theta) = -|eps|^2 / 2 (over the moving components, up to its
// constant) goes to lqf[b].  A proposal outside the prior box or the model's
// domain is marked inactive and the pass runs on the current theta instead.
// initial: the pass estimates log Z and the score at the current theta.
__global__ void lmh_propose_kernel(PmmhParams q, uint32_t iter, int initial)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= q.B) return;
    const int td = q.theta_dim;
    const double* cur = q.state_theta + (size_t)b * td;
    const double* g = q.state_grad + (size_t)b * td;
    double* prop = q.theta + (size_t)b * td;
    if (initial) {
        for (int d = 0; d < td; ++d) prop[d] = cur[d];
        q.active[b] = isnan(q.state_logz[b]) ? 1 : 0;
        return;
    }
    const Stream st{q.seed_lo, q.seed_hi, iter, (q.chain0 + (uint32_t)b) << 8};
    bool inside = true;
    double lqf = 0.0;
    for (int pq = 0; 2 * pq < td; ++pq) {
        const U4 w = st.draw((uint32_t)pq, 0u, KIND_MH, 0u);
        double z[2];
        normal_pair(w.x, w.y, z[0], z[1]);
        for (int h2 = 0; h2 < 2; ++h2) {
            const int d = 2 * pq + h2;
            if (d >= td) break;
            const double h = q.step[d];
            prop[d] = cur[d] + 0.5 * h * h * g[d] + h * z[h2];
            if (h > 0.0) {
                lqf -= 0.5 * z[h2] * z[h2];
                if (!(prop[d] >= q.lo[d] && prop[d] <= q.hi[d])) inside = false;
            }
        }
    }
    if (inside && !theta_in_domain(q.model, q.dx, prop)) inside = false;
    if (!inside)
        for (int d = 0; d < td; ++d) prop[d] = cur[d];
    q.active[b] = inside ? 1 : 0;
    q.lqf[b] = lqf;
}

// After the gradient pass at the proposals: the Metropolis-Hastings decision
// with log q(theta | theta') from the proposal's score, or (initial) the first
// estimate and score of chains whose log Z was NaN.
__global__ void lmh_accept_kernel(PmmhParams q, uint32_t iter, int j, int initial)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= q.B) return;
    const int td = q.theta_dim;
    double* cur = q.state_theta + (size_t)b * td;
    double* g = q.state_grad + (size_t)b * td;
    const double* gp = q.gprop + (size_t)b * td;
    if (initial) {
        if (q.active[b]) {
            q.state_logz[b] = q.logz[b];
            for (int d = 0; d < td; ++d) g[d] = gp[d];
        }
        return;
    }
    if (q.active[b]) {
        const double* prop = q.theta + (size_t)b * td;
        double lqr = 0.0;
        for (int d = 0; d < td; ++d) {
            const double h = q.step[d];
            if (h > 0.0) {
                const double e = (cur[d] - prop[d] - 0.5 * h * h * gp[d]) / h;
                lqr -= 0.5 * e * e;
            }
        }
        const Stream st{q.seed_lo, q.seed_hi, iter, (q.chain0 + (uint32_t)b) << 8};
        const U4 w = st.draw(0u, 0u, KIND_MH, 1u);
        const double lz = q.logz[b];
        if (log(unif_f64(w.x)) < lz - q.state_logz[b] + lqr - q.lqf[b]) {
            for (int d = 0; d < td; ++d) {
                cur[d] = prop[d];
                g[d] = gp[d];
            }
            q.state_logz[b] = lz;
            q.n_accept[b] += 1;
        }
    }
    if (q.theta_out)
        for (int d = 0; d < td; ++d) q.theta_out[((size_t)j * q.B + b) * td + d] = cur[d];
    if (q.logz_out) q.logz_out[(size_t)j * q.B + b] = q.state_logz[b];
}

cudaError_t launch_lmh_propose(const PmmhParams& q, uint32_t iter, int initial, cudaStream_t stream)
{
    lmh_propose_kernel<<<(q.B + 127) / 128, 128, 0, stream>>>(q, iter, initial);
    return cudaGetLastError();
}

cudaError_t launch_lmh_accept(const PmmhParams& q, uint32_t iter, int j, int initial, cudaStream_t stream)
{
    lmh_accept_kernel<<<(q.B + 127) / 128, 128, 0, stream>>>(q, iter, j, initial);
    return cudaGetLastError();
}

cudaError_t launch_pmmh_propose(const PmmhParams& q, uint32_t iter, int initial, cudaStream_t stream)
{
    pmmh_propose_kernel<<<(q.B + 127) / 128, 128, 0, stream>>>(q, iter, initial);
    return cudaGetLastError();
}

cudaError_t launch_pmmh_accept(const PmmhParams& q, uint32_t iter, int j, int initial, cudaStream_t stream)
{
    pmmh_accept_kernel<<<(q.B + 127) / 128, 128, 0, stream>>>(q, iter, j, initial);
    return cudaGetLastError();
}

}  // namespace airpf
