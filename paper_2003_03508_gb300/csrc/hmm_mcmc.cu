// Random-walk Metropolis-Hastings over the batched likelihood (hmm_mcmc_step).
//
// Section "Monte Carlo Markov Chains": a proposed state is accepted with
// probability min(1, likelihood x prior ratio). Section "Model priors" and
// Appendix A give the priors; they are read as: Dirichlet(alpha_P) on every
// row of P, Dirichlet(alpha_pi) on pi, Gamma(m^2/v, m/v) on p_k truncated to
// (0,1) (m = p_mean_lo for k < K/2, else p_mean_hi), 2x2 inverse-Wishart
// (df = iw_df, scale I) on Sigma_k, and uniform means on a box.
//
// The chains move in unconstrained coordinates theta (dimension K^2+6K-1):
// reference-logit rows of P (the diagonal is the reference), reference-logit
// pi (state 0 is the reference), logit p_k, the means, log sigma_x, log
// sigma_y, atanh rho. The log density of theta is the log prior plus the log
// Jacobian of theta -> parameters, evaluated in FP64.
//
// Random numbers are Philox4x32-10 (Salmon et al., SC 2011) keyed by the seed
// with counter (index/2, chain, iteration, 0) for the proposal normals
// (Box-Muller, cos/sin) and (index, chain, iteration, 1) for the acceptance
// uniform, so a run is reproducible and any draw can be recomputed.
//
// The t-walk (HMM_PROPOSAL_TWALK; Christen & Fox, Bayesian Analysis 2010, the
// sampler the paper uses) keeps a second point per chain and moves one of the
// two per iteration: a random coordinate subset (each coordinate with
// probability min(D, 4)/D, drawn again while empty) by the traverse (0.4918),
// walk (0.4918), blow (0.0082) or hop (0.0082) kernel, with the reference
// point the other one. Its draws use further Philox streams: side, kernel and
// beta uniforms (counter word 2), walk uniforms (3), blow/hop normals (4),
// subset attempt a (9 + a).
//
// One iteration = propose (+ transform) kernel, the batched likelihood, the
// accept kernel, and a one-thread kernel that advances the iteration counter
// kept in device memory. After a first, ordinary iteration the sampler
// captures one iteration in a CUDA graph and replays it.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hmm_internal.cuh"

struct hmm_mlp;
namespace hmm {
int mlp_dim(const hmm_mlp *m);
int mlp_hidden(const hmm_mlp *m);
float mlp_lambda(const hmm_mlp *m);
float mlp_drift(const hmm_mlp *m);
const float *mlp_scale(const hmm_mlp *m);
int mlp_eval(hmm_mlp *m, int B, const float *theta, float *x, float *a1, float *a2, float *out, cudaStream_t st);
size_t mlp_state_floats(const hmm_mlp *m);
cudaError_t mlp_state_io(hmm_mlp *m, float *host, float *lam, float *drift, bool save, cudaStream_t st);

namespace mcmc {

constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u, PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PH_W0;
            k1 += PH_W1;
        }
        const uint32_t hi0 = __umulhi(PH_M0, c[0]), lo0 = PH_M0 * c[0];
        const uint32_t hi1 = __umulhi(PH_M1, c[2]), lo1 = PH_M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0) + (1.0 / 33554432.0); }

__device__ double normal_draw(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t index) {
    uint32_t c[4] = {index / 2, chain, iter, 0u};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double rad = sqrt(-2.0 * log(u01(c[0])));
    const double ang = 6.283185307179586476925286766559 * u01(c[1]);
    return (index & 1) ? rad * sin(ang) : rad * cos(ang);
}

__device__ double uniform_draw(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t index) {
    uint32_t c[4] = {index, chain, iter, 1u};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return u01(c[0]);
}

// draws on a numbered stream (the fourth counter word): normals use the
// stream itself, uniforms stream + 1, as in the two functions above
__device__ double normal_draw_s(uint64_t seed, uint32_t stream, uint32_t chain, uint32_t iter, uint32_t index) {
    uint32_t c[4] = {index / 2, chain, iter, stream};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double rad = sqrt(-2.0 * log(u01(c[0])));
    const double ang = 6.283185307179586476925286766559 * u01(c[1]);
    return (index & 1) ? rad * sin(ang) : rad * cos(ang);
}

__device__ double uniform_draw_s(uint64_t seed, uint32_t stream, uint32_t chain, uint32_t iter, uint32_t index) {
    uint32_t c[4] = {index, chain, iter, stream + 1};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return u01(c[0]);
}

struct Prior {
    double alpha_P, alpha_pi, p_mean_lo, p_mean_hi, p_var, box[4], iw_df;
};

constexpr int TPB = 128;

__device__ double block_sum(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// theta (one chain, FP64 values in shared memory) -> parameters (FP32, the
// batched likelihood's layout) and the log density of theta. One CTA.
__device__ double transform(int K, const double *th, const Prior &pr, float *pi, float *P, float *p, float *mu,
                            float *cov, double *red) {
    double part = 0.0;
    // rows of P
    for (int i = threadIdx.x; i < K; i += TPB) {
        const double *z = th + (size_t)i * (K - 1);
        double mx = 0.0;
        for (int q = 0; q < K - 1; ++q) mx = fmax(mx, z[q]);
        double s = exp(-mx);
        for (int q = 0; q < K - 1; ++q) s += exp(z[q] - mx);
        const double lse = mx + log(s);
        for (int j = 0, q = 0; j < K; ++j) {
            const double zz = (j == i) ? 0.0 : z[q++];
            P[(size_t)i * K + j] = (float)exp(zz - lse);
            part += pr.alpha_P * (zz - lse);
        }
    }
    int o = K * (K - 1);
    // pi
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int k = 1; k < K; ++k) mx = fmax(mx, th[o + k - 1]);
        double s = exp(-mx);
        for (int k = 1; k < K; ++k) s += exp(th[o + k - 1] - mx);
        const double lse = mx + log(s);
        for (int k = 0; k < K; ++k) {
            const double zz = k == 0 ? 0.0 : th[o + k - 1];
            pi[k] = (float)exp(zz - lse);
            part += pr.alpha_pi * (zz - lse);
        }
    }
    o += K - 1;
    for (int k = threadIdx.x; k < K; k += TPB) {
        // p_k: logistic; truncated Gamma times the Jacobian p (1 - p)
        const double w = th[o + k];
        const double m = (k < K / 2) ? pr.p_mean_lo : pr.p_mean_hi;
        const double a = m * m / pr.p_var, b = m / pr.p_var;
        const double pk = 1.0 / (1.0 + exp(-w));
        p[k] = (float)pk;
        part += a * (-log1p(exp(-w))) - b * pk + (-log1p(exp(w)));
        // mean: uniform on the box
        const double x = th[o + K + 2 * k], y = th[o + K + 2 * k + 1];
        mu[2 * k] = (float)x;
        mu[2 * k + 1] = (float)y;
        if (x < pr.box[0] || x > pr.box[1] || y < pr.box[2] || y > pr.box[3]) part = -INFINITY;
        // covariance: inverse-Wishart(df, I) times the Jacobian 4 (1-rho^2) sx^3 sy^3
        const int oc = o + 3 * K;
        const double u = th[oc + 2 * k], v = th[oc + 2 * k + 1], r = th[oc + 2 * K + k];
        const double sx = exp(u), sy = exp(v), rho = tanh(r);
        const double sxx = sx * sx, syy = sy * sy, sxy = rho * sx * sy;
        cov[3 * k] = (float)sxx;
        cov[3 * k + 1] = (float)sxy;
        cov[3 * k + 2] = (float)syy;
        const double det = sxx * syy - sxy * sxy;
        part += -0.5 * (pr.iw_df + 3.0) * log(det) - 0.5 * (sxx + syy) / det;
        part += log(4.0) + log1p(-rho * rho) + 3.0 * u + 3.0 * v;
    }
    return block_sum(part, red);
}

struct Ctl {
    unsigned long long iter;   // absolute iteration counter
    unsigned long long iter0;  // counter at the start of the current hmm_mcmc_step call
    float *trace_lp;           // [n][C] log posterior trace of the current call, or null
    float *trace_theta;        // [n][C][D] state trace of the current call, or null
};

// theta -> parameters + log density, no proposal (initialisation / tests)
__global__ void __launch_bounds__(TPB) transform_kernel(int K, int D, const float *__restrict__ theta, Prior pr,
                                                        float *pi, float *P, float *p, float *mu, float *cov,
                                                        double *logprior) {
    extern __shared__ double sm[];
    double *th = sm;
    double *red = sm + D;
    const int c = blockIdx.x;
    for (int d = threadIdx.x; d < D; d += TPB) th[d] = theta[(size_t)c * D + d];
    __syncthreads();
    const double lp = transform(K, th, pr, pi + (size_t)c * K, P + (size_t)c * K * K, p + (size_t)c * K,
                                mu + (size_t)c * 2 * K, cov + (size_t)c * 3 * K, red);
    if (threadIdx.x == 0) logprior[c] = lp;
}

// theta' = theta + step * N(0, 1) (Philox), then theta' -> parameters + log density
__global__ void __launch_bounds__(TPB) propose_kernel(int K, int D, const float *__restrict__ theta,
                                                      const float *__restrict__ step, uint64_t seed,
                                                      const Ctl *__restrict__ ctl, Prior pr, float *theta_prop,
                                                      float *pi, float *P, float *p, float *mu, float *cov,
                                                      double *logprior) {
    extern __shared__ double sm[];
    double *th = sm;
    double *red = sm + D;
    const int c = blockIdx.x;
    const uint32_t it = (uint32_t)ctl->iter;
    for (int d = threadIdx.x; d < D; d += TPB) {
        const double z = normal_draw(seed, (uint32_t)c, it, (uint32_t)d);
        const float v = (float)((double)theta[(size_t)c * D + d] + (double)step[d] * z);
        theta_prop[(size_t)c * D + d] = v;
        th[d] = v;
    }
    __syncthreads();
    const double lp = transform(K, th, pr, pi + (size_t)c * K, P + (size_t)c * K * K, p + (size_t)c * K,
                                mu + (size_t)c * 2 * K, cov + (size_t)c * 3 * K, red);
    if (threadIdx.x == 0) logprior[c] = lp;
}

constexpr float FSIG_LO = -6.0f, FSIG_HI = 3.0f;  // same clamp as the network's training loss

// learned proposal: theta' = theta + lam s (gamma f_mu + exp(f_sig) z), z ~ N(0, I)
// (Philox); logq[c] = log q(theta' | theta) up to terms that cancel in the
// ratio; then theta' -> parameters + log density
__global__ void __launch_bounds__(TPB) propose_mlp_kernel(int K, int D, const float *__restrict__ theta,
                                                          const float *__restrict__ net, const float *__restrict__ scale,
                                                          float lam, float gam, uint64_t seed, const Ctl *__restrict__ ctl, Prior pr,
                                                          float *theta_prop, double *logq, float *pi, float *P,
                                                          float *p, float *mu, float *cov, double *logprior) {
    extern __shared__ double sm[];
    double *th = sm;
    double *red = sm + D;
    const int c = blockIdx.x;
    const uint32_t it = (uint32_t)ctl->iter;
    double lq = 0.0;
    for (int d = threadIdx.x; d < D; d += TPB) {
        const double z = normal_draw(seed, (uint32_t)c, it, (uint32_t)d);
        const float fmu = gam * net[(size_t)c * 2 * D + d];
        const float fs = fminf(fmaxf(net[(size_t)c * 2 * D + D + d], FSIG_LO), FSIG_HI);
        const double sd = (double)lam * scale[d] * exp((double)fs);
        const float v = (float)((double)theta[(size_t)c * D + d] + (double)lam * scale[d] * fmu + sd * z);
        theta_prop[(size_t)c * D + d] = v;
        th[d] = v;
        // density of the rounded proposal under q (standardised residual)
        const double r = ((double)v - theta[(size_t)c * D + d] - (double)lam * scale[d] * fmu) / sd;
        lq += -0.5 * r * r - log(sd);
    }
    const double lqs = block_sum(lq, red);
    if (threadIdx.x == 0) logq[c] = lqs;
    __syncthreads();
    const double lp = transform(K, th, pr, pi + (size_t)c * K, P + (size_t)c * K * K, p + (size_t)c * K,
                                mu + (size_t)c * 2 * K, cov + (size_t)c * 3 * K, red);
    if (threadIdx.x == 0) logprior[c] = lp;
}

// qcorr[c] = log q(theta | theta') - log q(theta' | theta), with the network
// evaluated at theta' (net_rev)
__global__ void __launch_bounds__(TPB) qcorr_kernel(int D, const float *__restrict__ theta,
                                                    const float *__restrict__ theta_prop,
                                                    const float *__restrict__ net_rev, const float *__restrict__ scale,
                                                    float lam, float gam, const double *__restrict__ logq_fwd,
                                                    double *qcorr) {
    __shared__ double red[TPB];
    const int c = blockIdx.x;
    double lq = 0.0;
    for (int d = threadIdx.x; d < D; d += TPB) {
        const float fmu = gam * net_rev[(size_t)c * 2 * D + d];
        const float fs = fminf(fmaxf(net_rev[(size_t)c * 2 * D + D + d], FSIG_LO), FSIG_HI);
        const double sd = (double)lam * scale[d] * exp((double)fs);
        const double r = ((double)theta[(size_t)c * D + d] - theta_prop[(size_t)c * D + d] -
                          (double)lam * scale[d] * fmu) / sd;
        lq += -0.5 * r * r - log(sd);
    }
    const double s = block_sum(lq, red);
    if (threadIdx.x == 0) qcorr[c] = s - logq_fwd[c];
}

// Metropolis-Hastings decision: accept when log u < (log L' + log pi') -
// (log L + log pi) + qcorr (qcorr = log q(theta|theta') - log q(theta'|theta),
// zero for the symmetric random walk).
__global__ void __launch_bounds__(TPB) accept_kernel(int D, uint64_t seed, const Ctl *__restrict__ ctl, float *theta,
                                                     const float *__restrict__ theta_prop, double *logpost,
                                                     double *loglik, double *logprior,
                                                     const double *__restrict__ loglik_prop,
                                                     const double *__restrict__ logprior_prop,
                                                     const double *__restrict__ qcorr,
                                                     unsigned long long *n_acc) {
    const int c = blockIdx.x;
    const uint32_t it = (uint32_t)ctl->iter;
    __shared__ int acc;
    if (threadIdx.x == 0) {
        const double lpp = loglik_prop[c] + logprior_prop[c];
        const double la = lpp - logpost[c] + (qcorr ? qcorr[c] : 0.0);
        const double u = uniform_draw(seed, (uint32_t)c, it, 0u);
        acc = (!isnan(lpp) && lpp > -INFINITY && log(u) < la) ? 1 : 0;
        if (acc) {
            logpost[c] = lpp;
            loglik[c] = loglik_prop[c];
            logprior[c] = logprior_prop[c];
            n_acc[c] += 1;
        }
    }
    __syncthreads();
    if (acc)
        for (int d = threadIdx.x; d < D; d += TPB) theta[(size_t)c * D + d] = theta_prop[(size_t)c * D + d];
    __syncthreads();
    const unsigned long long k = ctl->iter - ctl->iter0;
    if (ctl->trace_lp && threadIdx.x == 0) ctl->trace_lp[k * gridDim.x + c] = (float)logpost[c];
    if (ctl->trace_theta)
        for (int d = threadIdx.x; d < D; d += TPB)
            ctl->trace_theta[(k * gridDim.x + c) * D + d] = theta[(size_t)c * D + d];
}

// ---- t-walk ----
constexpr double TW_AW = 1.5, TW_AT = 6.0, TW_N1 = 4.0;
constexpr double TW_F_TRAVERSE = 0.4918, TW_F_WALK = 0.9836, TW_F_BLOW = 0.9918;
constexpr int TW_MAX_ATTEMPTS = 64;
enum { TW_TRAVERSE = 0, TW_WALK = 1, TW_BLOW = 2, TW_HOP = 3 };

__device__ double block_max(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// One t-walk proposal per chain (one CTA): picks the moving point, the
// kernel and the coordinate subset, writes the proposal theta' (float), the
// log of its acceptance factor besides the target ratio (W, -inf for a
// degenerate move), the side that moves, and theta' -> parameters + log
// density. Shared memory: theta' (D doubles), the reduction buffer, the
// subset (D bytes).
__global__ void __launch_bounds__(TPB) propose_twalk_kernel(int K, int D, const float *__restrict__ x,
                                                            const float *__restrict__ x2, uint64_t seed,
                                                            const Ctl *__restrict__ ctl, Prior pr, float *theta_prop,
                                                            double *W_out, int *side_out, float *pi, float *P,
                                                            float *p, float *mu, float *cov, double *logprior) {
    extern __shared__ double sm[];
    double *th = sm;
    double *red = sm + D;
    unsigned char *phi = reinterpret_cast<unsigned char *>(sm + D + TPB);
    __shared__ int s_side, s_kern;
    __shared__ double s_beta;
    const int c = blockIdx.x;
    const uint32_t it = (uint32_t)ctl->iter;
    if (threadIdx.x == 0) {
        s_side = uniform_draw_s(seed, 1, (uint32_t)c, it, 0) < 0.5 ? 0 : 1;
        const double uk = uniform_draw_s(seed, 1, (uint32_t)c, it, 1);
        s_kern = uk < TW_F_TRAVERSE ? TW_TRAVERSE : uk < TW_F_WALK ? TW_WALK : uk < TW_F_BLOW ? TW_BLOW : TW_HOP;
        const double u1 = uniform_draw_s(seed, 1, (uint32_t)c, it, 2), u2 = uniform_draw_s(seed, 1, (uint32_t)c, it, 3);
        s_beta = u1 < (TW_AT - 1.0) / (2.0 * TW_AT) ? pow(u2, 1.0 / (TW_AT + 1.0)) : pow(u2, 1.0 / (1.0 - TW_AT));
    }
    __syncthreads();
    const int side = s_side, kern = s_kern;
    const float *h = (side == 0 ? x : x2) + (size_t)c * D;
    const float *r = (side == 0 ? x2 : x) + (size_t)c * D;
    // the coordinate subset, drawn again while empty
    const double pphi = (D < TW_N1 ? (double)D : TW_N1) / (double)D;
    int m = 0;
    for (int a = 0; a < TW_MAX_ATTEMPTS && m == 0; ++a) {
        double cnt = 0.0;
        for (int d = threadIdx.x; d < D; d += TPB) {
            const unsigned char f = uniform_draw_s(seed, 8 + a, (uint32_t)c, it, (uint32_t)d) < pphi;
            phi[d] = f;
            cnt += f;
        }
        m = (int)block_sum(cnt, red);
    }
    if (m == 0) {  // practically unreachable: move every coordinate
        for (int d = threadIdx.x; d < D; d += TPB) phi[d] = 1;
        m = D;
    }
    __syncthreads();
    double w = 0.0;
    if (kern == TW_TRAVERSE) {
        const double beta = s_beta;
        for (int d = threadIdx.x; d < D; d += TPB) {
            const double hv = h[d], rv = r[d];
            th[d] = (double)(float)(phi[d] ? rv + beta * (rv - hv) : hv);
        }
        w = (m - 2) * log(beta);
    } else if (kern == TW_WALK) {
        for (int d = threadIdx.x; d < D; d += TPB) {
            const double hv = h[d], rv = r[d];
            double yv = hv;
            if (phi[d]) {
                const double u = uniform_draw_s(seed, 2, (uint32_t)c, it, (uint32_t)d);
                const double z = TW_AW / (1.0 + TW_AW) * (-1.0 + 2.0 * u + TW_AW * u * u);
                yv = hv + (hv - rv) * z;
            }
            th[d] = (double)(float)yv;
        }
    } else {
        double sf = 0.0;
        for (int d = threadIdx.x; d < D; d += TPB)
            if (phi[d]) sf = fmax(sf, fabs((double)r[d] - (double)h[d]));
        sf = block_max(sf, red);
        const bool blow = kern == TW_BLOW;
        if (!(sf > 0.0)) {
            w = -INFINITY;
            for (int d = threadIdx.x; d < D; d += TPB) th[d] = h[d];
        } else {
            const double sc = blow ? sf : sf / 3.0;
            for (int d = threadIdx.x; d < D; d += TPB)
                th[d] = (double)(float)(phi[d] ? (blow ? (double)r[d] : (double)h[d]) +
                                                     sc * normal_draw_s(seed, 4, (uint32_t)c, it, (uint32_t)d)
                                               : (double)h[d]);
            __syncthreads();
            // densities of the rounded proposal both ways (the 2 pi terms cancel)
            double sb = 0.0;
            for (int d = threadIdx.x; d < D; d += TPB)
                if (phi[d]) sb = fmax(sb, fabs((double)r[d] - th[d]));
            sb = block_max(sb, red);
            if (!(sb > 0.0)) {
                w = -INFINITY;
            } else {
                const double sfw = blow ? sf : sf / 3.0, sbw = blow ? sb : sb / 3.0;
                double q = 0.0;
                for (int d = threadIdx.x; d < D; d += TPB)
                    if (phi[d]) {
                        const double hv = h[d], yv = th[d], rv = r[d];
                        const double rb = blow ? (hv - rv) / sbw : (hv - yv) / sbw;  // reverse: x from y
                        const double rf = blow ? (yv - rv) / sfw : (yv - hv) / sfw;  // forward: y from x
                        q += -0.5 * rb * rb + 0.5 * rf * rf;
                    }
                q = block_sum(q, red);
                w = q - m * log(sbw) + m * log(sfw);
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < D; d += TPB) theta_prop[(size_t)c * D + d] = (float)th[d];
    if (threadIdx.x == 0) {
        W_out[c] = w;
        side_out[c] = side;
    }
    __syncthreads();
    const double lp = transform(K, th, pr, pi + (size_t)c * K, P + (size_t)c * K * K, p + (size_t)c * K,
                                mu + (size_t)c * 2 * K, cov + (size_t)c * 3 * K, red);
    if (threadIdx.x == 0) logprior[c] = lp;
}

// t-walk decision: accept when log u < (log L' + log pi') - (log L + log pi)
// of the moving point + W; the accepted proposal replaces that point. The
// traces record the first point.
__global__ void __launch_bounds__(TPB) accept_twalk_kernel(int D, uint64_t seed, const Ctl *__restrict__ ctl,
                                                           float *x, float *x2, const float *__restrict__ theta_prop,
                                                           double *logpost, double *loglik, double *logprior,
                                                           double *logpost2, double *loglik2, double *logprior2,
                                                           const double *__restrict__ loglik_prop,
                                                           const double *__restrict__ logprior_prop,
                                                           const double *__restrict__ W, const int *__restrict__ side,
                                                           unsigned long long *n_acc) {
    const int c = blockIdx.x;
    const uint32_t it = (uint32_t)ctl->iter;
    __shared__ int acc;
    const int sd = side[c];
    if (threadIdx.x == 0) {
        const double lpp = loglik_prop[c] + logprior_prop[c];
        const double cur = sd == 0 ? logpost[c] : logpost2[c];
        const double la = lpp - cur + W[c];
        const double u = uniform_draw(seed, (uint32_t)c, it, 0u);
        acc = (!isnan(lpp) && lpp > -INFINITY && W[c] > -INFINITY && log(u) < la) ? 1 : 0;
        if (acc) {
            if (sd == 0) {
                logpost[c] = lpp;
                loglik[c] = loglik_prop[c];
                logprior[c] = logprior_prop[c];
            } else {
                logpost2[c] = lpp;
                loglik2[c] = loglik_prop[c];
                logprior2[c] = logprior_prop[c];
            }
            n_acc[c] += 1;
        }
    }
    __syncthreads();
    if (acc) {
        float *dst = (sd == 0 ? x : x2) + (size_t)c * D;
        for (int d = threadIdx.x; d < D; d += TPB) dst[d] = theta_prop[(size_t)c * D + d];
    }
    __syncthreads();
    const unsigned long long k = ctl->iter - ctl->iter0;
    if (ctl->trace_lp && threadIdx.x == 0) ctl->trace_lp[k * gridDim.x + c] = (float)logpost[c];
    if (ctl->trace_theta)
        for (int d = threadIdx.x; d < D; d += TPB)
            ctl->trace_theta[(k * gridDim.x + c) * D + d] = x[(size_t)c * D + d];
}

__global__ void advance_kernel(Ctl *ctl) { ctl->iter += 1; }

// largest |FP32-SIMT value - stored value| over the chains. The stored values
// (the ones the Metropolis-Hastings rule compares) are left as they are, so
// every acceptance ratio stays within the sampler's own precision.
__global__ void recheck_kernel(int C, const double *ll32, const double *loglik, double *maxdiff) {
    __shared__ double red[128];
    double m = 0.0;
    for (int c = threadIdx.x; c < C; c += 128) {
        const double d = fabs(ll32[c] - loglik[c]);
        if (!isnan(d)) m = fmax(m, d);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *maxdiff = red[0];
}

__global__ void sum_kernel(int C, const double *a, const double *b, double *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) out[c] = a[c] + b[c];
}

}  // namespace mcmc
}  // namespace hmm

using namespace hmm;
using namespace hmm::mcmc;

struct hmm_sampler {
    hmm_ctx *lik = nullptr;  // private context: its workspace never moves under the graph
    hmm_ctx *lik32 = nullptr;  // FP32-SIMT recheck of the current states (own workspace)
    double *loglik32 = nullptr;
    double *recheck_maxdiff = nullptr;
    int C = 0, K = 0, D = 0;
    uint64_t seed = 0;
    Prior prior{};
    hmm_opts opts{};
    int n_seg = 0;
    int64_t *offs = nullptr;  // host copy
    const float *xy = nullptr;
    const uint8_t *tremor = nullptr;
    // device state
    float *theta = nullptr, *theta_prop = nullptr, *step = nullptr;
    float *pi = nullptr, *P = nullptr, *p = nullptr, *mu = nullptr, *cov = nullptr;
    double *logpost = nullptr, *loglik = nullptr, *logprior = nullptr, *loglik_prop = nullptr,
           *logprior_prop = nullptr;
    unsigned long long *n_acc = nullptr;
    Ctl *ctl = nullptr;
    unsigned long long iter_host = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches_per_iter = 0;
    int graph_failed = 0;
    // learned proposal (HMM_PROPOSAL_MLP): network and its buffers
    int kind = HMM_PROPOSAL_RW;
    hmm_mlp *mlp = nullptr;
    float *mx = nullptr, *ma1 = nullptr, *ma2 = nullptr, *net_f = nullptr, *net_r = nullptr;
    double *logq = nullptr, *qcorr = nullptr;
    // t-walk (HMM_PROPOSAL_TWALK): the second point of every chain
    float *theta2 = nullptr;
    double *logpost2 = nullptr, *loglik2 = nullptr, *logprior2 = nullptr, *tw_W = nullptr;
    int *tw_side = nullptr;
    // iterations run on the sampler's own stream (the legacy default stream
    // cannot be captured), ordered against the caller's stream by events
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

static Prior to_prior(const hmm_prior *p, int K) {
    Prior r{};
    if (p) {
        r.alpha_P = p->alpha_P;
        r.alpha_pi = p->alpha_pi;
        r.p_mean_lo = p->p_mean_lo;
        r.p_mean_hi = p->p_mean_hi;
        r.p_var = p->p_var;
        for (int i = 0; i < 4; ++i) r.box[i] = p->box[i];
        r.iw_df = p->iw_df;
    } else {
        r.alpha_P = 0.01;
        r.alpha_pi = 1.0;
        r.p_mean_lo = 0.1;
        r.p_mean_hi = 0.9;
        r.p_var = 0.001;
        r.box[0] = 0;
        r.box[1] = 300;
        r.box[2] = 0;
        r.box[3] = 150;
        r.iw_df = K;
    }
    return r;
}

static size_t smem_for(int D) { return sizeof(double) * ((size_t)D + TPB); }
static size_t smem_twalk(int D) { return smem_for(D) + (size_t)D + 16; }

extern "C" {

int32_t hmm_theta_dim(int32_t K) { return K * K + 6 * K - 1; }

void hmm_prior_default(hmm_prior *p, int32_t K) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->alpha_P = 0.01f;
    p->alpha_pi = 1.0f;
    p->p_mean_lo = 0.1f;
    p->p_mean_hi = 0.9f;
    p->p_var = 0.001f;
    p->box[0] = 0.f;
    p->box[1] = 300.f;
    p->box[2] = 0.f;
    p->box[3] = 150.f;
    p->iw_df = (float)K;
}

int hmm_theta_to_params(int32_t n, int32_t K, const float *theta, const hmm_prior *prior, float *pi, float *P,
                        float *p_tremor, float *mu, float *cov, double *logprior, void *stream) {
    if (n < 1 || K < 2 || K > 80 || !theta || !pi || !P || !p_tremor || !mu || !cov || !logprior)
        return HMM_EINVAL;
    const int D = hmm_theta_dim(K);
    const Prior pr = to_prior(prior, K);
    transform_kernel<<<n, TPB, smem_for(D), (cudaStream_t)stream>>>(K, D, theta, pr, pi, P, p_tremor, mu, cov,
                                                                     logprior);
    return cudaGetLastError() == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

int hmm_sampler_destroy(hmm_sampler *s) {
    if (!s) return HMM_OK;
    if (s->own) cudaStreamSynchronize(s->own);
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    if (s->own) cudaStreamDestroy(s->own);
    void *bufs[] = {s->theta, s->theta_prop, s->step, s->pi, s->P, s->p, s->mu, s->cov, s->logpost, s->loglik,
                    s->logprior, s->loglik_prop, s->logprior_prop, s->n_acc, s->ctl, s->loglik32,
                    s->recheck_maxdiff, s->mx, s->ma1, s->ma2, s->net_f, s->net_r, s->logq, s->qcorr,
                    s->theta2, s->logpost2, s->loglik2, s->logprior2, s->tw_W, s->tw_side};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete[] s->offs;
    if (s->lik) hmm_destroy(s->lik);
    if (s->lik32) hmm_destroy(s->lik32);
    delete s;
    return HMM_OK;
}

int hmm_sampler_create(hmm_sampler **out, int device, int32_t n_chains, int32_t K, const hmm_prior *prior,
                       const float *theta0, const float *step, uint64_t seed, int32_t n_seg,
                       const int64_t *seg_offsets, const float *xy, const uint8_t *tremor, const hmm_opts *opts,
                       void *stream) {
    if (!out) return HMM_EINVAL;
    *out = nullptr;
    if (n_chains < 1 || K < 2 || K > 80 || !theta0 || !step || n_seg < 1 || !seg_offsets) return HMM_EINVAL;
    hmm_sampler *s = new (std::nothrow) hmm_sampler();
    if (!s) return HMM_ENOMEM;
    int rc = hmm_create(&s->lik, device);
    if (rc) {
        delete s;
        return rc;
    }
    const int C = n_chains, D = hmm_theta_dim(K);
    s->C = C;
    s->K = K;
    s->D = D;
    s->seed = seed;
    s->prior = to_prior(prior, K);
    if (opts) s->opts = *opts; else hmm_opts_default(&s->opts);
    s->n_seg = n_seg;
    s->offs = new int64_t[n_seg + 1];
    memcpy(s->offs, seg_offsets, sizeof(int64_t) * (n_seg + 1));
    s->xy = xy;
    s->tremor = tremor;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void **)&s->theta, sizeof(float) * C * D);
    alloc((void **)&s->theta_prop, sizeof(float) * C * D);
    alloc((void **)&s->step, sizeof(float) * D);
    alloc((void **)&s->pi, sizeof(float) * C * K);
    alloc((void **)&s->P, sizeof(float) * C * K * K);
    alloc((void **)&s->p, sizeof(float) * C * K);
    alloc((void **)&s->mu, sizeof(float) * C * 2 * K);
    alloc((void **)&s->cov, sizeof(float) * C * 3 * K);
    alloc((void **)&s->logpost, sizeof(double) * C);
    alloc((void **)&s->loglik, sizeof(double) * C);
    alloc((void **)&s->logprior, sizeof(double) * C);
    alloc((void **)&s->loglik_prop, sizeof(double) * C);
    alloc((void **)&s->logprior_prop, sizeof(double) * C);
    alloc((void **)&s->n_acc, sizeof(unsigned long long) * C);
    alloc((void **)&s->ctl, sizeof(Ctl));
    alloc((void **)&s->loglik32, sizeof(double) * C);
    alloc((void **)&s->recheck_maxdiff, sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hmm_sampler_destroy(s);
        return HMM_ENOMEM;
    }
    Ctl c0{};
    e = cudaMemcpyAsync(s->theta, theta0, sizeof(float) * C * D, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->step, step, sizeof(float) * D, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->n_acc, 0, sizeof(unsigned long long) * C, st);
    // no recheck yet: the FP32 report reads NaN (all bits set)
    if (e == cudaSuccess) e = cudaMemsetAsync(s->loglik32, 0xff, sizeof(double) * C, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->recheck_maxdiff, 0xff, sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->ctl, &c0, sizeof(Ctl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hmm_sampler_destroy(s);
        return HMM_ECUDA;
    }
    // initial state: parameters, log prior, log likelihood, log posterior
    transform_kernel<<<C, TPB, smem_for(D), st>>>(K, D, s->theta, s->prior, s->pi, s->P, s->p, s->mu, s->cov,
                                                   s->logprior);
    rc = hmm_loglik_batched(s->lik, C, K, s->pi, s->P, s->p, s->mu, s->cov, n_seg, s->offs, xy, tremor, &s->opts,
                            s->loglik, stream);
    if (rc == HMM_OK) {
        sum_kernel<<<(C + 127) / 128, 128, 0, st>>>(C, s->loglik, s->logprior, s->logpost);
        if (cudaGetLastError() != cudaSuccess) rc = HMM_ECUDA;
    }
    if (rc != HMM_OK) {
        hmm_sampler_destroy(s);
        return rc;
    }
    *out = s;
    return HMM_OK;
}

static int recheck(hmm_sampler *s, cudaStream_t st);

// one iteration's launches (also what the graph captures)
static int iteration(hmm_sampler *s, cudaStream_t st) {
    const int C = s->C, K = s->K, D = s->D;
    int extra = 0;
    if (s->kind == HMM_PROPOSAL_MLP) {
        const float lam = mlp_lambda(s->mlp);
        const float *scale = mlp_scale(s->mlp);
        if (mlp_eval(s->mlp, C, s->theta, s->mx, s->ma1, s->ma2, s->net_f, st)) return HMM_ECUDA;
        const float gam = mlp_drift(s->mlp);
        propose_mlp_kernel<<<C, TPB, smem_for(D), st>>>(K, D, s->theta, s->net_f, scale, lam, gam, s->seed, s->ctl,
                                                         s->prior, s->theta_prop, s->logq, s->pi, s->P, s->p, s->mu,
                                                         s->cov, s->logprior_prop);
        if (mlp_eval(s->mlp, C, s->theta_prop, s->mx, s->ma1, s->ma2, s->net_r, st)) return HMM_ECUDA;
        qcorr_kernel<<<C, TPB, 0, st>>>(D, s->theta, s->theta_prop, s->net_r, scale, lam, gam, s->logq, s->qcorr);
        extra = 2 * 4 + 1;  // two network evaluations (standardise + 3 GEMMs) and the q ratio
    } else if (s->kind == HMM_PROPOSAL_TWALK) {
        propose_twalk_kernel<<<C, TPB, smem_twalk(D), st>>>(K, D, s->theta, s->theta2, s->seed, s->ctl, s->prior,
                                                             s->theta_prop, s->tw_W, s->tw_side, s->pi, s->P, s->p,
                                                             s->mu, s->cov, s->logprior_prop);
    } else {
        propose_kernel<<<C, TPB, smem_for(D), st>>>(K, D, s->theta, s->step, s->seed, s->ctl, s->prior,
                                                     s->theta_prop, s->pi, s->P, s->p, s->mu, s->cov,
                                                     s->logprior_prop);
    }
    if (cudaGetLastError() != cudaSuccess) return HMM_ECUDA;
    int rc = hmm_loglik_batched(s->lik, C, K, s->pi, s->P, s->p, s->mu, s->cov, s->n_seg, s->offs, s->xy,
                                s->tremor, &s->opts, s->loglik_prop, st);
    if (rc) return rc;
    s->launches_per_iter = hmm_last_launch_count(s->lik) + 3 + extra;
    if (s->kind == HMM_PROPOSAL_TWALK)
        accept_twalk_kernel<<<C, TPB, 0, st>>>(D, s->seed, s->ctl, s->theta, s->theta2, s->theta_prop, s->logpost,
                                               s->loglik, s->logprior, s->logpost2, s->loglik2, s->logprior2,
                                               s->loglik_prop, s->logprior_prop, s->tw_W, s->tw_side, s->n_acc);
    else
        accept_kernel<<<C, TPB, 0, st>>>(D, s->seed, s->ctl, s->theta, s->theta_prop, s->logpost, s->loglik,
                                         s->logprior, s->loglik_prop, s->logprior_prop,
                                         s->kind == HMM_PROPOSAL_MLP ? s->qcorr : nullptr, s->n_acc);
    advance_kernel<<<1, 1, 0, st>>>(s->ctl);
    return cudaGetLastError() == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

static int mcmc_step_own(hmm_sampler *s, int32_t n_iter, float *trace_logpost, float *trace_theta,
                         cudaStream_t st);

int hmm_mcmc_step(hmm_sampler *s, int32_t n_iter, float *trace_logpost, float *trace_theta, void *stream) {
    if (!s || n_iter < 0) return HMM_EINVAL;
    if (n_iter == 0) return HMM_OK;
    cudaStream_t user = (cudaStream_t)stream;
    if (cudaEventRecord(s->ev_in, user) != cudaSuccess || cudaStreamWaitEvent(s->own, s->ev_in, 0) != cudaSuccess)
        return HMM_ECUDA;
    const int rc = mcmc_step_own(s, n_iter, trace_logpost, trace_theta, s->own);
    if (cudaEventRecord(s->ev_out, s->own) != cudaSuccess || cudaStreamWaitEvent(user, s->ev_out, 0) != cudaSuccess)
        return rc ? rc : HMM_ECUDA;
    return rc;
}

static int mcmc_step_own(hmm_sampler *s, int32_t n_iter, float *trace_logpost, float *trace_theta,
                         cudaStream_t st) {
    // per-call control block: trace destinations and the first iteration index
    Ctl c{};
    c.iter = s->iter_host;
    c.iter0 = s->iter_host;
    c.trace_lp = trace_logpost;
    c.trace_theta = trace_theta;
    cudaError_t e = cudaMemcpyAsync(s->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // &c is a stack object
    if (e != cudaSuccess) return HMM_ECUDA;
    int done = 0;
    if (!s->exec && s->graph_failed) {
        for (; done < n_iter; ++done) {
            int rc = iteration(s, st);
            if (rc) return rc;
        }
        s->iter_host += n_iter;
        if (s->opts.recheck_fp32 && s->opts.precision != HMM_PREC_FP32_SIMT) return recheck(s, st);
        return HMM_OK;
    }
    if (!s->exec) {
        // first iteration runs directly (sizes the workspace, uploads the plan),
        // the second is captured once and replayed from then on
        int rc = iteration(s, st);
        if (rc) return rc;
        ++done;
        if (done < n_iter) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                rc = iteration(s, st);
                e = cudaStreamEndCapture(st, &g);
                if (rc == HMM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&s->exec, g, 0);
                if (e == cudaSuccess) s->graph = g; else if (g) cudaGraphDestroy(g);
            }
            if (e != cudaSuccess || rc != HMM_OK) {
                cudaGetLastError();
                if (s->exec) {
                    cudaGraphExecDestroy(s->exec);
                    s->exec = nullptr;
                }
                // fall back to direct launches for the rest of this call
                s->graph_failed = 1;
                for (; done < n_iter; ++done) {
                    rc = iteration(s, st);
                    if (rc) return rc;
                }
                s->iter_host += n_iter;
                if (s->opts.recheck_fp32 && s->opts.precision != HMM_PREC_FP32_SIMT) return recheck(s, st);
                return HMM_OK;
            }
        }
    }
    for (; done < n_iter; ++done) {
        e = cudaGraphLaunch(s->exec, st);
        if (e != cudaSuccess) return HMM_ECUDA;
    }
    s->iter_host += n_iter;
    if (s->opts.recheck_fp32 && s->opts.precision != HMM_PREC_FP32_SIMT) return recheck(s, st);
    return HMM_OK;
}

// FP32-SIMT re-evaluation of every chain's current state, i.e. of the last
// proposal each chain accepted, into the sampler's FP32 report (loglik32) and
// the largest difference from the stored values. It never feeds back into the
// chains: their stored log likelihoods, and so every later acceptance ratio,
// stay in the sampler's precision.
static int recheck(hmm_sampler *s, cudaStream_t st) {
    if (!s->lik32) {
        int dev = 0;
        cudaGetDevice(&dev);
        int rc = hmm_create(&s->lik32, dev);
        if (rc) return rc;
    }
    const int C = s->C, K = s->K, D = s->D;
    transform_kernel<<<C, TPB, smem_for(D), st>>>(K, D, s->theta, s->prior, s->pi, s->P, s->p, s->mu, s->cov,
                                                   s->logprior_prop);
    hmm_opts o = s->opts;
    o.precision = HMM_PREC_FP32_SIMT;
    o.chunk_len = 0;
    o.recheck_fp32 = 0;
    int rc = hmm_loglik_batched(s->lik32, C, K, s->pi, s->P, s->p, s->mu, s->cov, s->n_seg, s->offs, s->xy,
                                s->tremor, &o, s->loglik32, st);
    if (rc) return rc;
    recheck_kernel<<<1, 128, 0, st>>>(C, s->loglik32, s->loglik, s->recheck_maxdiff);
    return cudaGetLastError() == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

static int copy_fp32_report(hmm_sampler *s, double *loglik_fp32_out, double *max_abs_diff_dev, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (loglik_fp32_out)
        e = cudaMemcpyAsync(loglik_fp32_out, s->loglik32, sizeof(double) * s->C, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && max_abs_diff_dev)
        e = cudaMemcpyAsync(max_abs_diff_dev, s->recheck_maxdiff, sizeof(double), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

int hmm_sampler_recheck(hmm_sampler *s, double *loglik_fp32_out, double *max_abs_diff_dev, void *stream) {
    if (!s) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = recheck(s, st);
    if (rc) return rc;
    return copy_fp32_report(s, loglik_fp32_out, max_abs_diff_dev, st);
}

int hmm_sampler_fp32_report(hmm_sampler *s, double *loglik_fp32_out, double *max_abs_diff_dev, void *stream) {
    if (!s) return HMM_EINVAL;
    return copy_fp32_report(s, loglik_fp32_out, max_abs_diff_dev, (cudaStream_t)stream);
}

int hmm_sampler_state(hmm_sampler *s, float *theta_out, double *logpost_out, double *loglik_out,
                      unsigned long long *n_accept_out, void *stream) {
    if (!s) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (theta_out) e = cudaMemcpyAsync(theta_out, s->theta, sizeof(float) * s->C * s->D, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && logpost_out)
        e = cudaMemcpyAsync(logpost_out, s->logpost, sizeof(double) * s->C, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && loglik_out)
        e = cudaMemcpyAsync(loglik_out, s->loglik, sizeof(double) * s->C, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && n_accept_out)
        e = cudaMemcpyAsync(n_accept_out, s->n_acc, sizeof(unsigned long long) * s->C, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

int hmm_sampler_set_twalk(hmm_sampler *s, const float *theta2, void *stream) {
    if (!s || !theta2) return HMM_EINVAL;
    const int C = s->C, K = s->K, D = s->D;
    cudaStream_t st = (cudaStream_t)stream;
    if (!s->theta2) {
        cudaError_t e = cudaMalloc(&s->theta2, sizeof(float) * C * D);
        if (e == cudaSuccess) e = cudaMalloc(&s->logpost2, sizeof(double) * C);
        if (e == cudaSuccess) e = cudaMalloc(&s->loglik2, sizeof(double) * C);
        if (e == cudaSuccess) e = cudaMalloc(&s->logprior2, sizeof(double) * C);
        if (e == cudaSuccess) e = cudaMalloc(&s->tw_W, sizeof(double) * C);
        if (e == cudaSuccess) e = cudaMalloc(&s->tw_side, sizeof(int) * C);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return HMM_ENOMEM;
        }
    }
    // the sampler's own stream may be replaying iterations: order after them
    if (s->own && cudaStreamSynchronize(s->own) != cudaSuccess) return HMM_ECUDA;
    if (cudaMemcpyAsync(s->theta2, theta2, sizeof(float) * C * D, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return HMM_ECUDA;
    // the second point's parameters, log prior, log likelihood, log posterior
    // (the parameter buffers are scratch between iterations)
    transform_kernel<<<C, TPB, smem_for(D), st>>>(K, D, s->theta2, s->prior, s->pi, s->P, s->p, s->mu, s->cov,
                                                   s->logprior2);
    if (cudaGetLastError() != cudaSuccess) return HMM_ECUDA;
    int rc = hmm_loglik_batched(s->lik, C, K, s->pi, s->P, s->p, s->mu, s->cov, s->n_seg, s->offs, s->xy,
                                s->tremor, &s->opts, s->loglik2, stream);
    if (rc) return rc;
    sum_kernel<<<(C + 127) / 128, 128, 0, st>>>(C, s->loglik2, s->logprior2, s->logpost2);
    if (cudaGetLastError() != cudaSuccess) return HMM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HMM_ECUDA;
    return hmm_sampler_set_proposal(s, HMM_PROPOSAL_TWALK, nullptr);
}

int hmm_sampler_twalk_state(hmm_sampler *s, float *theta2_out, double *logpost2_out, void *stream) {
    if (!s || !s->theta2) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (theta2_out)
        e = cudaMemcpyAsync(theta2_out, s->theta2, sizeof(float) * s->C * s->D, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && logpost2_out)
        e = cudaMemcpyAsync(logpost2_out, s->logpost2, sizeof(double) * s->C, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

int hmm_sampler_set_proposal(hmm_sampler *s, int32_t kind, hmm_mlp *mlp) {
    if (!s) return HMM_EINVAL;
    if (kind != HMM_PROPOSAL_RW && kind != HMM_PROPOSAL_MLP && kind != HMM_PROPOSAL_TWALK) return HMM_EINVAL;
    if (kind == HMM_PROPOSAL_TWALK && !s->theta2) return HMM_EINVAL;  // hmm_sampler_set_twalk first
    if (kind == HMM_PROPOSAL_MLP) {
        if (!mlp || mlp_dim(mlp) != s->D) return HMM_EINVAL;
        if (!s->mx) {
            const int C = s->C, D = s->D, H = mlp_hidden(mlp);
            cudaError_t e = cudaMalloc(&s->mx, sizeof(float) * C * D);
            if (e == cudaSuccess) e = cudaMalloc(&s->ma1, sizeof(float) * C * H);
            if (e == cudaSuccess) e = cudaMalloc(&s->ma2, sizeof(float) * C * H);
            if (e == cudaSuccess) e = cudaMalloc(&s->net_f, sizeof(float) * C * 2 * D);
            if (e == cudaSuccess) e = cudaMalloc(&s->net_r, sizeof(float) * C * 2 * D);
            if (e == cudaSuccess) e = cudaMalloc(&s->logq, sizeof(double) * C);
            if (e == cudaSuccess) e = cudaMalloc(&s->qcorr, sizeof(double) * C);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return HMM_ENOMEM;
            }
        } else if (mlp_hidden(mlp) != mlp_hidden(s->mlp ? s->mlp : mlp)) {
            return HMM_EINVAL;  // buffers were sized for another hidden width
        }
    }
    // the captured iteration no longer matches: capture again on the next call
    if (s->own) cudaStreamSynchronize(s->own);
    if (s->exec) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    if (s->graph) {
        cudaGraphDestroy(s->graph);
        s->graph = nullptr;
    }
    s->graph_failed = 0;
    s->kind = kind;
    s->mlp = kind == HMM_PROPOSAL_MLP ? mlp : nullptr;
    return HMM_OK;
}

// ---- checkpoints ----
//
// File layout (native byte order): the 8-byte tag "HMMSMP01"; int32 C, K, D,
// proposal kind, has second points, network d, network hidden width, n_seg;
// int64 total observations; uint64 seed, iteration counter; float step[D];
// float theta[C][D]; double logpost[C], loglik[C], logprior[C]; uint64
// accepted[C]; double FP32 report[C] and its largest difference; then, with
// second points, float theta2[C][D] and double logpost2/loglik2/logprior2[C];
// then, for the learned proposal, the network state (parameters, mean,
// in_scale, scale) and float lam, drift.

static const char CKPT_TAG[8] = {'H', 'M', 'M', 'S', 'M', 'P', '0', '1'};

struct CkptHead {
    int32_t C, K, D, kind, has2, mlp_d, mlp_h, n_seg;
    int64_t T_total;
    uint64_t seed, iter;
};

namespace {

struct Blob {
    void *dev;
    size_t bytes;
};

std::vector<Blob> ckpt_blobs(hmm_sampler *s, bool with2) {
    const size_t C = s->C, D = s->D;
    std::vector<Blob> b = {{s->step, sizeof(float) * D},          {s->theta, sizeof(float) * C * D},
                           {s->logpost, sizeof(double) * C},      {s->loglik, sizeof(double) * C},
                           {s->logprior, sizeof(double) * C},     {s->n_acc, sizeof(unsigned long long) * C},
                           {s->loglik32, sizeof(double) * C},     {s->recheck_maxdiff, sizeof(double)}};
    if (with2) {
        b.push_back({s->theta2, sizeof(float) * C * D});
        b.push_back({s->logpost2, sizeof(double) * C});
        b.push_back({s->loglik2, sizeof(double) * C});
        b.push_back({s->logprior2, sizeof(double) * C});
    }
    return b;
}

void drop_graph(hmm_sampler *s) {
    if (s->exec) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    if (s->graph) {
        cudaGraphDestroy(s->graph);
        s->graph = nullptr;
    }
    s->graph_failed = 0;
}

}  // namespace

int hmm_sampler_save(hmm_sampler *s, const char *path, void *stream) {
    if (!s || !path) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // iterations replay on the sampler's own stream: the state is final after it
    if (s->own && cudaStreamSynchronize(s->own) != cudaSuccess) return HMM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HMM_ECUDA;
    CkptHead h{};
    h.C = s->C;
    h.K = s->K;
    h.D = s->D;
    h.kind = s->kind;
    h.has2 = s->theta2 ? 1 : 0;
    h.mlp_d = s->kind == HMM_PROPOSAL_MLP ? mlp_dim(s->mlp) : 0;
    h.mlp_h = s->kind == HMM_PROPOSAL_MLP ? mlp_hidden(s->mlp) : 0;
    h.n_seg = s->n_seg;
    h.T_total = s->offs[s->n_seg];
    h.seed = s->seed;
    h.iter = s->iter_host;
    std::vector<char> buf(sizeof(CKPT_TAG) + sizeof(h));
    memcpy(buf.data(), CKPT_TAG, sizeof(CKPT_TAG));
    memcpy(buf.data() + sizeof(CKPT_TAG), &h, sizeof(h));
    for (const Blob &b : ckpt_blobs(s, h.has2)) {
        const size_t o = buf.size();
        buf.resize(o + b.bytes);
        if (cudaMemcpyAsync(buf.data() + o, b.dev, b.bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HMM_ECUDA;
    }
    if (h.kind == HMM_PROPOSAL_MLP) {
        const size_t nf = mlp_state_floats(s->mlp);
        const size_t o = buf.size();
        buf.resize(o + sizeof(float) * (nf + 2));
        float *f = reinterpret_cast<float *>(buf.data() + o);
        if (mlp_state_io(s->mlp, f, f + nf, f + nf + 1, true, st) != cudaSuccess) return HMM_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return HMM_ECUDA;
    FILE *fp = fopen(path, "wb");
    if (!fp) return HMM_EINVAL;
    const bool ok = fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    const bool closed = fclose(fp) == 0;
    return ok && closed ? HMM_OK : HMM_EINVAL;
}

int hmm_sampler_load(hmm_sampler *s, const char *path, void *stream) {
    if (!s || !path) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    FILE *fp = fopen(path, "rb");
    if (!fp) return HMM_EINVAL;
    std::vector<char> buf;
    char chunk[1 << 16];
    size_t n;
    while ((n = fread(chunk, 1, sizeof(chunk), fp)) > 0) buf.insert(buf.end(), chunk, chunk + n);
    fclose(fp);
    CkptHead h{};
    if (buf.size() < sizeof(CKPT_TAG) + sizeof(h) || memcmp(buf.data(), CKPT_TAG, sizeof(CKPT_TAG)) != 0)
        return HMM_EINVAL;
    memcpy(&h, buf.data() + sizeof(CKPT_TAG), sizeof(h));
    // the sampler must have been created for the same chains and data
    if (h.C != s->C || h.K != s->K || h.D != s->D || h.n_seg != s->n_seg || h.T_total != s->offs[s->n_seg])
        return HMM_EINVAL;
    if (h.kind != HMM_PROPOSAL_RW && h.kind != HMM_PROPOSAL_MLP && h.kind != HMM_PROPOSAL_TWALK) return HMM_EINVAL;
    if (h.kind == HMM_PROPOSAL_TWALK && !h.has2) return HMM_EINVAL;
    // the learned proposal is restored into the network the sampler uses now
    if (h.kind == HMM_PROPOSAL_MLP &&
        (s->kind != HMM_PROPOSAL_MLP || !s->mlp || mlp_dim(s->mlp) != h.mlp_d || mlp_hidden(s->mlp) != h.mlp_h))
        return HMM_EINVAL;
    size_t need = sizeof(CKPT_TAG) + sizeof(h);
    if (h.has2 && !s->theta2) {
        const int C = s->C, D = s->D;
        cudaError_t e = cudaMalloc(&s->theta2, sizeof(float) * C * D);
        if (e == cudaSuccess) e = cudaMalloc(&s->logpost2, sizeof(double) * C);
        if (e == cudaSuccess) e = cudaMalloc(&s->loglik2, sizeof(double) * C);
        if (e == cudaSuccess) e = cudaMalloc(&s->logprior2, sizeof(double) * C);
        if (e == cudaSuccess) e = cudaMalloc(&s->tw_W, sizeof(double) * C);
        if (e == cudaSuccess) e = cudaMalloc(&s->tw_side, sizeof(int) * C);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return HMM_ENOMEM;
        }
    }
    const std::vector<Blob> blobs = ckpt_blobs(s, h.has2);
    for (const Blob &b : blobs) need += b.bytes;
    const size_t nf = h.kind == HMM_PROPOSAL_MLP ? mlp_state_floats(s->mlp) : 0;
    if (h.kind == HMM_PROPOSAL_MLP) need += sizeof(float) * (nf + 2);
    if (buf.size() != need) return HMM_EINVAL;
    if (s->own && cudaStreamSynchronize(s->own) != cudaSuccess) return HMM_ECUDA;
    size_t o = sizeof(CKPT_TAG) + sizeof(h);
    for (const Blob &b : blobs) {
        if (cudaMemcpyAsync(b.dev, buf.data() + o, b.bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return HMM_ECUDA;
        o += b.bytes;
    }
    if (h.kind == HMM_PROPOSAL_MLP) {
        float *f = reinterpret_cast<float *>(buf.data() + o);
        if (mlp_state_io(s->mlp, f, f + nf, f + nf + 1, false, st) != cudaSuccess) return HMM_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return HMM_ECUDA;
    // the seed and the proposal kind are kernel arguments of the captured iteration
    drop_graph(s);
    s->seed = h.seed;
    s->iter_host = h.iter;
    s->kind = h.kind;
    if (h.kind != HMM_PROPOSAL_MLP) s->mlp = nullptr;
    return HMM_OK;
}

int hmm_sampler_launches_per_iter(const hmm_sampler *s) { return s ? s->launches_per_iter : -1; }

int hmm_sampler_graph_active(const hmm_sampler *s) { return s ? (s->exec != nullptr ? 1 : 0) : -1; }

}  // extern "C"
