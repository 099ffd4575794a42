// Gradient of log L and the EM (Baum-Welch) update from the hidden chain's
// expected sufficient statistics (hmm_loglik_grad, hmm_em_step).
//
// The statistics come from the chunked forward-backward pass of
// hmm_expected_stats: N (expected transition counts), G0 (posterior of the
// first state), Gs, Gr (posterior mass over all steps and over tremor
// steps) and the gamma-weighted moments Sx, Sy, Sxx, Sxy, Syy of the tremor
// locations. The complete-data log likelihood of the model of Section 2,
//     log p(s, o) = log v0[s_0] + sum_{t>=1} log P[s_{t-1}, s_t] + sum_t log e_{s_t}(o_t),
// with the emissions of Eq. "emission-matrix", has a gradient whose posterior
// expectation is the gradient of log L (the Fisher identity):
//     d/dP_ij    = N_ij / P_ij
//     d/dp_k     = Gr_k / p_k - (Gs_k - Gr_k) / (1 - p_k)
//     d/dmu_k    = Sigma_k^-1 (S_k - Gr_k mu_k)
//     d/dSigma_k = 1/2 Sigma_k^-1 (Q_k - Gr_k Sigma_k) Sigma_k^-1,
//     Q_k = sum over tremor steps of gamma_t(k) (o_t - mu_k)(o_t - mu_k)^T,
// and d/dpi_k = G0_k / pi_k when pi is the law of the first state; with the
// transition-first convention v0 = P^T pi, so r_j = G0_j / v0_j gives
// d/dpi_i = sum_j P_ij r_j and adds pi_i r_j to d/dP_ij. P and pi are
// differentiated as free entries (the simplex constraint belongs to whatever
// parameterisation the caller uses); Sigma as (sxx, sxy, syy), sxy entering
// both off-diagonal entries. Terms whose expected count is zero contribute
// zero. Everything here is FP64, one CTA.
//
// The M-step maximises the expected complete-data log likelihood:
// P_ij = N_ij / sum_j N_ij, pi = G0, p_k = Gr_k / Gs_k, mu_k = S_k / Gr_k,
// Sigma_k = Q_k / Gr_k; a row or state with no expected count keeps its
// previous value.
#include "hmm_internal.cuh"

namespace hmm {
namespace {

constexpr int GT = 256;

struct StatsView {
    const double *N, *G0, *Gs, *Gr, *Sx, *Sy, *Sxx, *Sxy, *Syy;
    __device__ StatsView(const double *s, int K)
        : N(s), G0(s + K * K), Gs(G0 + K), Gr(Gs + K), Sx(Gr + K), Sy(Sx + K), Sxx(Sy + K), Sxy(Sxx + K),
          Syy(Sxy + K) {}
};

__device__ __forceinline__ double ratio(double num, double den) { return num != 0.0 ? num / den : 0.0; }

__global__ void __launch_bounds__(GT) fisher_grad_kernel(int K, int init_mode, const float *__restrict__ pi,
                                                         const float *__restrict__ P, const float *__restrict__ p,
                                                         const float *__restrict__ mu, const float *__restrict__ cov,
                                                         const double *__restrict__ stats, double *__restrict__ grad) {
    const StatsView st(stats, K);
    double *dpi = grad, *dP = grad + K, *dp = dP + K * K, *dmu = dp + K, *dcov = dmu + 2 * K;
    // transition-first: r_j = G0_j / v0_j, v0 = P^T pi
    extern __shared__ double r[];
    for (int j = threadIdx.x; j < K; j += GT) {
        if (init_mode == HMM_INIT_TRANSITION_FIRST) {
            double v0 = 0.0;
            for (int i = 0; i < K; ++i) v0 += (double)pi[i] * (double)P[i * K + j];
            r[j] = ratio(st.G0[j], v0);
        } else {
            r[j] = 0.0;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += GT) {
        const int i = e / K, j = e % K;
        double g = ratio(st.N[e], (double)P[e]);
        if (init_mode == HMM_INIT_TRANSITION_FIRST) g += (double)pi[i] * r[j];
        dP[e] = g;
    }
    for (int k = threadIdx.x; k < K; k += GT) {
        if (init_mode == HMM_INIT_TRANSITION_FIRST) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += (double)P[k * K + j] * r[j];
            dpi[k] = s;
        } else {
            dpi[k] = ratio(st.G0[k], (double)pi[k]);
        }
        const double pk = p[k], gr = st.Gr[k], gn = st.Gs[k] - st.Gr[k];
        dp[k] = ratio(gr, pk) - ratio(gn, 1.0 - pk);
        // Sigma^-1 of (sxx, sxy, syy)
        const double a = cov[3 * k], b = cov[3 * k + 1], c = cov[3 * k + 2];
        const double det = a * c - b * b;
        const double l00 = c / det, l01 = -b / det, l11 = a / det;
        const double mx = mu[2 * k], my = mu[2 * k + 1];
        const double s1x = st.Sx[k], s1y = st.Sy[k];
        // Q = s2 - m s1^T - s1 m^T + g m m^T
        const double q00 = st.Sxx[k] - 2.0 * mx * s1x + gr * mx * mx;
        const double q01 = st.Sxy[k] - mx * s1y - s1x * my + gr * mx * my;
        const double q11 = st.Syy[k] - 2.0 * my * s1y + gr * my * my;
        const double ux = s1x - gr * mx, uy = s1y - gr * my;
        dmu[2 * k] = l00 * ux + l01 * uy;
        dmu[2 * k + 1] = l01 * ux + l11 * uy;
        // dS = 1/2 Lam (Q - g S) Lam
        const double m00 = q00 - gr * a, m01 = q01 - gr * b, m11 = q11 - gr * c;
        const double t00 = l00 * m00 + l01 * m01, t01 = l00 * m01 + l01 * m11;
        const double t10 = l01 * m00 + l11 * m01, t11 = l01 * m01 + l11 * m11;
        const double d00 = 0.5 * (t00 * l00 + t01 * l01);
        const double d01 = 0.5 * (t00 * l01 + t01 * l11);
        const double d11 = 0.5 * (t10 * l01 + t11 * l11);
        dcov[3 * k] = d00;
        dcov[3 * k + 1] = 2.0 * d01;
        dcov[3 * k + 2] = d11;
    }
}

__global__ void __launch_bounds__(GT) em_mstep_kernel(int K, const float *__restrict__ pi, const float *__restrict__ P,
                                                      const float *__restrict__ p, const float *__restrict__ mu,
                                                      const float *__restrict__ cov, const double *__restrict__ stats,
                                                      float *pi_out, float *P_out, float *p_out, float *mu_out,
                                                      float *cov_out) {
    const StatsView st(stats, K);
    __shared__ double g0sum;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += st.G0[k];
        g0sum = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += GT) {
        double rs = 0.0;
        for (int j = 0; j < K; ++j) rs += st.N[i * K + j];
        for (int j = 0; j < K; ++j) P_out[i * K + j] = rs > 0.0 ? (float)(st.N[i * K + j] / rs) : P[i * K + j];
        pi_out[i] = g0sum > 0.0 ? (float)(st.G0[i] / g0sum) : pi[i];
        const double g = st.Gr[i], gs = st.Gs[i];
        p_out[i] = gs > 0.0 ? (float)(g / gs) : p[i];
        if (g > 0.0) {
            const double mx = st.Sx[i] / g, my = st.Sy[i] / g;
            mu_out[2 * i] = (float)mx;
            mu_out[2 * i + 1] = (float)my;
            cov_out[3 * i] = (float)(st.Sxx[i] / g - mx * mx);
            cov_out[3 * i + 1] = (float)(st.Sxy[i] / g - mx * my);
            cov_out[3 * i + 2] = (float)(st.Syy[i] / g - my * my);
        } else {
            mu_out[2 * i] = mu[2 * i];
            mu_out[2 * i + 1] = mu[2 * i + 1];
            for (int c = 0; c < 3; ++c) cov_out[3 * i + c] = cov[3 * i + c];
        }
    }
}

}  // namespace

cudaError_t launch_fisher_grad(int K, int init_mode, const float *pi, const float *P, const float *p, const float *mu,
                               const float *cov, const double *stats, double *grad, cudaStream_t st) {
    fisher_grad_kernel<<<1, GT, sizeof(double) * K, st>>>(K, init_mode, pi, P, p, mu, cov, stats, grad);
    return cudaGetLastError();
}

cudaError_t launch_em_mstep(int K, const float *pi, const float *P, const float *p, const float *mu, const float *cov,
                            const double *stats, float *pi_out, float *P_out, float *p_out, float *mu_out,
                            float *cov_out, cudaStream_t st) {
    em_mstep_kernel<<<1, GT, 0, st>>>(K, pi, P, p, mu, cov, stats, pi_out, P_out, p_out, mu_out, cov_out);
    return cudaGetLastError();
}

}  // namespace hmm
