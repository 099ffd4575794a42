/*
 * CPU oracle for the MCMC layer -- TEST INFRASTRUCTURE ONLY (loaded by the
 * tests, smoke() and the benchmark's CPU leg, never by the product path).
 *
 * Section "Monte Carlo Markov Chains": states are accepted or rejected by the
 * ratio of likelihood x prior at the proposed and current states.
 * Section "Model priors" and Appendix A: symmetric Dirichlet(0.01) on the
 * transition matrix, Gamma priors on the tremor probabilities (half with
 * mean 0.1, half with mean 0.9, variance 0.001), uniform means on a box
 * containing the data, inverse-Wishart covariances with df = K.
 *
 * Readings (the printed Appendix A formulas are garbled):
 *   - Dirichlet(alpha) on every row of P (normaliser Gamma(n a)/Gamma(a)^n);
 *     Dirichlet(1) (flat) on pi.
 *   - Gamma(shape m^2/v, rate m/v) on p_k truncated to (0, 1): m = 0.1 for
 *     k < K/2, else 0.9; v = 0.001.
 *   - the inverse-Wishart is the 2 x 2 one, nu = K, scale I_2.
 *   - mu_k uniform on the box [x0, x1] x [y0, y1].
 * Densities are evaluated up to additive constants that do not depend on the
 * parameters (they cancel in the acceptance ratio).
 *
 * Unconstrained coordinates theta (the order of the vector):
 *   P   : K*(K-1) reference logits, row i, columns j != i in increasing j;
 *         P_ij = exp(z_ij) / (1 + sum_{l != i} exp(z_il)), P_ii = 1 / (same)
 *   pi  : K-1 reference logits for states 1..K-1 (state 0 is the reference)
 *   p   : K logits, p_k = 1 / (1 + exp(-w_k))
 *   mu  : 2K (x_k, y_k)
 *   sig : 2K (log sigma_x, log sigma_y)
 *   rho : K  (atanh rho)
 * dimension K^2 + 6K - 1.
 *
 * Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written from its
 * published definition. Uniforms in (0, 1): (x >> 8) * 2^-24 + 2^-25.
 * Normals: Box-Muller on a pair of such uniforms, cos branch.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

/* ctr[4] in, out[4] out, key[2] */
void oracle_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0) + (1.0 / 33554432.0); }

/*
 * Random numbers of one (stream, chain, iteration): counter
 * (index/2, chain, iteration, stream) with key (seed_lo, seed_hi);
 * normal number `index` uses the words of counter index/2 (Box-Muller pair,
 * cos for even index, sin for odd). Uniform `index` uses word 0 of counter
 * (index, chain, iteration, stream + 1).
 */
double oracle_normal(uint64_t seed, uint32_t stream, uint32_t chain, uint32_t iter, uint32_t index)
{
    uint32_t ctr[4] = {index / 2, chain, iter, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    oracle_philox4x32_10(ctr, key, o);
    double a = u01(o[0]), b = u01(o[1]);
    double rad = sqrt(-2.0 * log(a));
    double ang = 6.283185307179586476925286766559 * b;
    return (index & 1) ? rad * sin(ang) : rad * cos(ang);
}

double oracle_uniform(uint64_t seed, uint32_t stream, uint32_t chain, uint32_t iter, uint32_t index)
{
    uint32_t ctr[4] = {index, chain, iter, stream + 1};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    oracle_philox4x32_10(ctr, key, o);
    return u01(o[0]);
}

int oracle_theta_dim(int K) { return K * K + 6 * K - 1; }

typedef struct {
    double alpha_P, alpha_pi;      /* Dirichlet concentrations (rows of P, pi) */
    double p_mean_lo, p_mean_hi;   /* Gamma means for k < K/2 and k >= K/2     */
    double p_var;                  /* Gamma variance                           */
    double box[4];                 /* x0, x1, y0, y1 for the uniform means      */
    double iw_df;                  /* inverse-Wishart degrees of freedom        */
} oracle_prior;

/*
 * theta -> (pi, P, p, mu, cov) in double, and the log prior density plus the
 * log Jacobian of the map (the log density of theta, up to a constant).
 * Returns -INFINITY if a mean lies outside the box.
 */
double oracle_theta_to_params(int K, const double *th, const oracle_prior *pr, double *pi,
                              double *P, double *p, double *mu, double *cov)
{
    double lp = 0.0;
    int o = 0;
    /* rows of P: reference-logit softmax; density of the logits under a
     * Dirichlet(alpha) row with its Jacobian prod_j P_ij: alpha sum_j log P_ij */
    for (int i = 0; i < K; ++i) {
        double mx = 0.0;  /* reference logit is 0 */
        for (int j = 0, q = o; j < K; ++j) if (j != i) { if (th[q] > mx) mx = th[q]; ++q; }
        double s = exp(-mx);
        for (int j = 0, q = o; j < K; ++j) if (j != i) { s += exp(th[q] - mx); ++q; }
        double lse = mx + log(s);
        for (int j = 0, q = o; j < K; ++j) {
            double z = (j == i) ? 0.0 : th[q++];
            P[i * K + j] = exp(z - lse);
            lp += pr->alpha_P * (z - lse);
        }
        o += K - 1;
    }
    /* pi: reference logit for state 0 */
    {
        double mx = 0.0;
        for (int k = 1; k < K; ++k) if (th[o + k - 1] > mx) mx = th[o + k - 1];
        double s = exp(-mx);
        for (int k = 1; k < K; ++k) s += exp(th[o + k - 1] - mx);
        double lse = mx + log(s);
        for (int k = 0; k < K; ++k) {
            double z = k == 0 ? 0.0 : th[o + k - 1];
            pi[k] = exp(z - lse);
            lp += pr->alpha_pi * (z - lse);
        }
        o += K - 1;
    }
    /* p_k: logistic; Gamma(a, b) truncated to (0,1) times Jacobian p (1 - p):
     * a log p - b p + log(1 - p) */
    for (int k = 0; k < K; ++k) {
        double w = th[o + k];
        double m = (k < K / 2) ? pr->p_mean_lo : pr->p_mean_hi;
        double a = m * m / pr->p_var, b = m / pr->p_var;
        double lpk = -log1p(exp(-w));          /* log p     */
        double l1p = -log1p(exp(w));           /* log (1-p) */
        p[k] = 1.0 / (1.0 + exp(-w));
        lp += a * lpk - b * p[k] + l1p;
    }
    o += K;
    /* means: uniform on the box */
    for (int k = 0; k < K; ++k) {
        double x = th[o + 2 * k], y = th[o + 2 * k + 1];
        mu[2 * k] = x;
        mu[2 * k + 1] = y;
        if (x < pr->box[0] || x > pr->box[1] || y < pr->box[2] || y > pr->box[3]) lp = -INFINITY;
    }
    o += 2 * K;
    /* covariances: (log sx, log sy, atanh rho); 2x2 inverse-Wishart(nu, I)
     * density |S|^(-(nu+3)/2) exp(-tr(S^-1)/2) times the Jacobian
     * 4 (1 - rho^2) sx^3 sy^3 */
    for (int k = 0; k < K; ++k) {
        double u = th[o + 2 * k], v = th[o + 2 * k + 1], r = th[o + 2 * K + k];
        double sx = exp(u), sy = exp(v), rho = tanh(r);
        double sxx = sx * sx, syy = sy * sy, sxy = rho * sx * sy;
        cov[3 * k] = sxx;
        cov[3 * k + 1] = sxy;
        cov[3 * k + 2] = syy;
        double det = sxx * syy - sxy * sxy;
        double tr_inv = (sxx + syy) / det;
        lp += -0.5 * (pr->iw_df + 3.0) * log(det) - 0.5 * tr_inv;
        lp += log(4.0) + log1p(-rho * rho) + 3.0 * u + 3.0 * v;
    }
    return lp;
}
