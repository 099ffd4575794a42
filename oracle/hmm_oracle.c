/*
 * CPU oracle for the tremor-HMM log-likelihood -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this file's library. The product path never calls it, and it shares
 * no code, header, table or constant with the CUDA sources.
 *
 * Everything is plain, serial and in double precision (long double for the
 * two cross-checks), written to be checked against the paper by eye:
 *
 *   Section 2, Eq. "emission-matrix": the diagonal emission matrix P(x) has
 *     entries p_k * phi(x | mu_k, Sigma_k) for a tremor observed at x in R^2
 *     and 1 - p_k for "no tremor"; phi is the bivariate normal density.
 *   Section 2, Eq. "likelihood func": L = delta^T Gamma P(x_0) ... Gamma P(x_N) 1.
 *   Algorithm 1 (the Forward algorithm on a CPU): v <- delta^T; per
 *     observation v <- v Gamma, v <- v P(x_k); return v 1.
 *   Section "Step 3" (last paragraph): log L is computed with scale
 *     coefficients so nothing underflows.
 *
 * Readings of the paper used here (each is also listed in the design notes):
 *   - init_mode 0 ("emit first", the default): L = pi^T D_1 P D_2 ... P D_T 1,
 *     i.e. pi is the distribution of the first hidden state.
 *   - init_mode 1 ("transition first", Eq. "likelihood func" and Algorithm 1
 *     as printed): pi is replaced by P^T pi before the first emission.
 *   - The two emission cases are "tremor at x" (first line) and "no tremor"
 *     (second line); the case labels are missing from the printed equation.
 *   - Sigma_k is the full 2x2 covariance, passed as (sxx, sxy, syy).
 *   - The scaling of Algorithm 1 is the textbook one: after each step the
 *     forward vector is divided by its sum c_t and log L accumulates
 *     m_t + log c_t, where m_t = max_k log e_k(o_t) keeps exp() in range.
 *   - A zero likelihood returns -INFINITY.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* log e_k(o) for every state k (Eq. "emission-matrix"), natural log. */
static void log_emissions(int K, const float *p, const float *mu, const float *cov,
                          int tremor, double x, double y, double *out)
{
    for (int k = 0; k < K; ++k) {
        double pk = (double)p[k];
        if (!tremor) {
            out[k] = log(1.0 - pk);
            continue;
        }
        double sxx = cov[3 * k + 0], sxy = cov[3 * k + 1], syy = cov[3 * k + 2];
        double det = sxx * syy - sxy * sxy;
        double dx = x - (double)mu[2 * k + 0];
        double dy = y - (double)mu[2 * k + 1];
        /* (o - mu)^T Sigma^{-1} (o - mu) with Sigma^{-1} = adj(Sigma) / det */
        double q = (syy * dx * dx - 2.0 * sxy * dx * dy + sxx * dy * dy) / det;
        out[k] = log(pk) - log(ORACLE_TWO_PI) - 0.5 * log(det) - 0.5 * q;
    }
}

void oracle_log_emission(int K, const float *p, const float *mu, const float *cov,
                         int tremor, double x, double y, double *out)
{
    log_emissions(K, p, mu, cov, tremor, x, y, out);
}

/* Initial distribution actually used at the first observation. */
static void initial_vector(int K, const float *pi, const float *P, int init_mode, double *v)
{
    if (init_mode == 1) {           /* delta^T Gamma: one transition first */
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
            for (int i = 0; i < K; ++i) s += (double)pi[i] * (double)P[i * K + j];
            v[j] = s;
        }
    } else {
        for (int j = 0; j < K; ++j) v[j] = (double)pi[j];
    }
}

static double max_of(int K, const double *a)
{
    double m = -INFINITY;
    for (int k = 0; k < K; ++k) if (a[k] > m) m = a[k];
    return m;
}

/*
 * Scaled forward recursion (Algorithm 1 with scale coefficients), FP64.
 * log L is accumulated with Kahan compensation.
 */
double oracle_loglik(int K, const float *pi, const float *P, const float *p,
                     const float *mu, const float *cov, int64_t T, const float *xy,
                     const uint8_t *tremor, int init_mode)
{
    double *alpha = (double *)malloc(sizeof(double) * K);
    double *beta = (double *)malloc(sizeof(double) * K);
    double *le = (double *)malloc(sizeof(double) * K);
    initial_vector(K, pi, P, init_mode, alpha);
    double logL = 0.0, comp = 0.0;
    if (T == 0) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += alpha[k];
        free(alpha); free(beta); free(le);
        return log(s);
    }
    for (int64_t t = 0; t < T; ++t) {
        log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);
        if (t == 0) {
            for (int k = 0; k < K; ++k) beta[k] = alpha[k];
        } else {
            for (int j = 0; j < K; ++j) {
                double s = 0.0;
                for (int i = 0; i < K; ++i) s += alpha[i] * (double)P[i * K + j];
                beta[j] = s;
            }
        }
        double m = max_of(K, le);
        if (m == -INFINITY) { logL = -INFINITY; break; }
        double c = 0.0;
        for (int k = 0; k < K; ++k) {
            alpha[k] = beta[k] * exp(le[k] - m);
            c += alpha[k];
        }
        if (!(c > 0.0)) { logL = -INFINITY; break; }
        for (int k = 0; k < K; ++k) alpha[k] /= c;
        /* Kahan-compensated logL += m + log(c) */
        double term = m + log(c);
        double yk = term - comp;
        double tk = logL + yk;
        comp = (tk - logL) - yk;
        logL = tk;
    }
    free(alpha); free(beta); free(le);
    return logL;
}

/*
 * Independent cross-check: the scaled backward recursion
 *   b_T = 1,  b_t[i] = sum_j P_ij e_j(o_{t+1}) b_{t+1}[j],
 *   L = sum_k pi_k e_k(o_1) b_1[k].
 */
double oracle_loglik_backward(int K, const float *pi, const float *P, const float *p,
                              const float *mu, const float *cov, int64_t T, const float *xy,
                              const uint8_t *tremor, int init_mode)
{
    double *b = (double *)malloc(sizeof(double) * K);
    double *nb = (double *)malloc(sizeof(double) * K);
    double *le = (double *)malloc(sizeof(double) * K);
    double *v0 = (double *)malloc(sizeof(double) * K);
    initial_vector(K, pi, P, init_mode, v0);
    double logS = 0.0;
    if (T == 0) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += v0[k];
        free(b); free(nb); free(le); free(v0);
        return log(s);
    }
    for (int k = 0; k < K; ++k) b[k] = 1.0;
    for (int64_t t = T - 1; t >= 1; --t) {
        log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);
        double m = max_of(K, le);
        if (m == -INFINITY) { logS = -INFINITY; break; }
        double mx = 0.0;
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += (double)P[i * K + j] * exp(le[j] - m) * b[j];
            nb[i] = s;
            if (s > mx) mx = s;
        }
        if (!(mx > 0.0)) { logS = -INFINITY; break; }
        for (int i = 0; i < K; ++i) b[i] = nb[i] / mx;
        logS += m + log(mx);
    }
    double out;
    if (logS == -INFINITY) {
        out = -INFINITY;
    } else {
        log_emissions(K, p, mu, cov, tremor[0], xy[0], xy[1], le);
        double m = max_of(K, le);
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += v0[k] * exp(le[k] - m) * b[k];
        out = (m == -INFINITY || !(s > 0.0)) ? -INFINITY : logS + m + log(s);
    }
    free(b); free(nb); free(le); free(v0);
    return out;
}

/* The same forward recursion carried in long double (rounding cross-check). */
double oracle_loglik_ld(int K, const float *pi, const float *P, const float *p,
                        const float *mu, const float *cov, int64_t T, const float *xy,
                        const uint8_t *tremor, int init_mode)
{
    long double *alpha = (long double *)malloc(sizeof(long double) * K);
    long double *beta = (long double *)malloc(sizeof(long double) * K);
    long double *le = (long double *)malloc(sizeof(long double) * K);
    if (init_mode == 1) {
        for (int j = 0; j < K; ++j) {
            long double s = 0.0L;
            for (int i = 0; i < K; ++i) s += (long double)pi[i] * (long double)P[i * K + j];
            alpha[j] = s;
        }
    } else {
        for (int j = 0; j < K; ++j) alpha[j] = (long double)pi[j];
    }
    long double logL = 0.0L;
    if (T == 0) {
        long double s = 0.0L;
        for (int k = 0; k < K; ++k) s += alpha[k];
        free(alpha); free(beta); free(le);
        return (double)logl(s);
    }
    for (int64_t t = 0; t < T; ++t) {
        long double x = xy[2 * t], y = xy[2 * t + 1];
        for (int k = 0; k < K; ++k) {
            long double pk = p[k];
            if (!tremor[t]) { le[k] = logl(1.0L - pk); continue; }
            long double sxx = cov[3 * k], sxy = cov[3 * k + 1], syy = cov[3 * k + 2];
            long double det = sxx * syy - sxy * sxy;
            long double dx = x - (long double)mu[2 * k], dy = y - (long double)mu[2 * k + 1];
            long double q = (syy * dx * dx - 2.0L * sxy * dx * dy + sxx * dy * dy) / det;
            le[k] = logl(pk) - logl(2.0L * 3.14159265358979323846264338327950288L)
                    - 0.5L * logl(det) - 0.5L * q;
        }
        if (t == 0) {
            for (int k = 0; k < K; ++k) beta[k] = alpha[k];
        } else {
            for (int j = 0; j < K; ++j) {
                long double s = 0.0L;
                for (int i = 0; i < K; ++i) s += alpha[i] * (long double)P[i * K + j];
                beta[j] = s;
            }
        }
        long double m = -INFINITY;
        for (int k = 0; k < K; ++k) if (le[k] > m) m = le[k];
        if (m == -INFINITY) { logL = -INFINITY; break; }
        long double c = 0.0L;
        for (int k = 0; k < K; ++k) { alpha[k] = beta[k] * expl(le[k] - m); c += alpha[k]; }
        if (!(c > 0.0L)) { logL = -INFINITY; break; }
        for (int k = 0; k < K; ++k) alpha[k] /= c;
        logL += m + logl(c);
    }
    free(alpha); free(beta); free(le);
    return (double)logL;
}

/*
 * Brute force over all K^T hidden paths (tiny inputs only):
 *   L = sum_{s_1..s_T} pi_{s_1} e_{s_1}(o_1) prod_{t>=2} P_{s_{t-1} s_t} e_{s_t}(o_t).
 * Emissions are evaluated once in double and summed in long double.
 * Returns NAN if K^T exceeds 2^26.
 */
double oracle_loglik_bruteforce(int K, const float *pi, const float *P, const float *p,
                                const float *mu, const float *cov, int64_t T, const float *xy,
                                const uint8_t *tremor, int init_mode)
{
    double npaths = pow((double)K, (double)T);
    if (npaths > 67108864.0) return NAN;
    double *v0 = (double *)malloc(sizeof(double) * K);
    initial_vector(K, pi, P, init_mode, v0);
    if (T == 0) {
        long double s = 0.0L;
        for (int k = 0; k < K; ++k) s += v0[k];
        free(v0);
        return (double)logl(s);
    }
    double *e = (double *)malloc(sizeof(double) * K * (size_t)T);
    for (int64_t t = 0; t < T; ++t) {
        log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], e + (size_t)t * K);
        for (int k = 0; k < K; ++k) e[(size_t)t * K + k] = exp(e[(size_t)t * K + k]);
    }
    int *s = (int *)calloc((size_t)T, sizeof(int));
    long double total = 0.0L;
    for (;;) {
        long double w = (long double)v0[s[0]] * e[s[0]];
        for (int64_t t = 1; t < T; ++t)
            w *= (long double)P[s[t - 1] * K + s[t]] * e[(size_t)t * K + s[t]];
        total += w;
        int64_t d = T - 1;               /* odometer increment over the path */
        while (d >= 0 && ++s[d] == K) { s[d] = 0; --d; }
        if (d < 0) break;
    }
    free(v0); free(e); free(s);
    return total > 0.0L ? (double)logl(total) : -INFINITY;
}

/* ---------- many proposals x many segments, threads over proposals ---------- */

typedef struct {
    int n_prop, K, n_seg, init_mode;
    const float *pi, *P, *p, *mu, *cov, *xy;
    const uint8_t *tremor;
    const int64_t *offs;
    double *out;
    int next;
    pthread_mutex_t lock;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = (batch_job *)arg;
    int K = j->K;
    for (;;) {
        pthread_mutex_lock(&j->lock);
        int q = j->next++;
        pthread_mutex_unlock(&j->lock);
        if (q >= j->n_prop) break;
        double acc = 0.0;
        for (int s = 0; s < j->n_seg; ++s) {
            int64_t a = j->offs[s], b = j->offs[s + 1];
            acc += oracle_loglik(K, j->pi + (size_t)q * K, j->P + (size_t)q * K * K,
                                 j->p + (size_t)q * K, j->mu + (size_t)q * 2 * K,
                                 j->cov + (size_t)q * 3 * K, b - a, j->xy + 2 * a,
                                 j->tremor + a, j->init_mode);
        }
        j->out[q] = acc;
    }
    return NULL;
}

/*
 * out[q] = sum over segments s of log L(proposal q | segment s); each segment
 * is an independent sequence starting from pi. n_threads <= 0 means 1.
 */
void oracle_loglik_batched(int n_prop, int K, const float *pi, const float *P,
                           const float *p, const float *mu, const float *cov, int n_seg,
                           const int64_t *offsets, const float *xy, const uint8_t *tremor,
                           int init_mode, double *out, int n_threads)
{
    batch_job j;
    j.n_prop = n_prop; j.K = K; j.n_seg = n_seg; j.init_mode = init_mode;
    j.pi = pi; j.P = P; j.p = p; j.mu = mu; j.cov = cov; j.xy = xy; j.tremor = tremor;
    j.offs = offsets; j.out = out; j.next = 0;
    pthread_mutex_init(&j.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, batch_worker, &j);
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&j.lock);
}

/*
 * Posterior state probabilities gamma_t(k) = P(s_t = k | o_1..o_T), the
 * smoothing step that follows the likelihood (the forward-backward
 * algorithm; Rabiner, Proc. IEEE 1989, Section III-A). The forward
 * vectors are normalised every step and stored in `gamma` (T x K); the
 * backward recursion
 *   b_T = 1,  b_t[i] = sum_j P_ij e_j(o_{t+1}) b_{t+1}[j]
 * runs with its own per-step normalisation (any positive factor per step
 * cancels), and gamma_t = alpha_t * b_t / sum_k alpha_t(k) b_t(k).
 * Returns log L; for a zero likelihood gamma is set to NaN and -inf
 * returned.
 */
double oracle_posterior(int K, const float *pi, const float *P, const float *p, const float *mu,
                        const float *cov, int64_t T, const float *xy, const uint8_t *tremor, int init_mode,
                        double *gamma)
{
    double *alpha = (double *)malloc(sizeof(double) * K);
    double *beta = (double *)malloc(sizeof(double) * K);
    double *nb = (double *)malloc(sizeof(double) * K);
    double *le = (double *)malloc(sizeof(double) * K);
    initial_vector(K, pi, P, init_mode, alpha);
    double logL = 0.0;
    int zero = 0;
    for (int64_t t = 0; t < T && !zero; ++t) {
        log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);
        if (t == 0) {
            for (int k = 0; k < K; ++k) beta[k] = alpha[k];
        } else {
            for (int j = 0; j < K; ++j) {
                double s = 0.0;
                for (int i = 0; i < K; ++i) s += alpha[i] * (double)P[i * K + j];
                beta[j] = s;
            }
        }
        double m = max_of(K, le), c = 0.0;
        if (m == -INFINITY) { zero = 1; break; }
        for (int k = 0; k < K; ++k) {
            alpha[k] = beta[k] * exp(le[k] - m);
            c += alpha[k];
        }
        if (!(c > 0.0)) { zero = 1; break; }
        for (int k = 0; k < K; ++k) {
            alpha[k] /= c;
            gamma[t * K + k] = alpha[k];
        }
        logL += m + log(c);
    }
    if (zero) {
        for (int64_t i = 0; i < T * K; ++i) gamma[i] = NAN;
        free(alpha); free(beta); free(nb); free(le);
        return -INFINITY;
    }
    for (int k = 0; k < K; ++k) beta[k] = 1.0;
    for (int64_t t = T - 1; t >= 0; --t) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += gamma[t * K + k] * beta[k];
        for (int k = 0; k < K; ++k) gamma[t * K + k] = gamma[t * K + k] * beta[k] / s;
        if (t == 0) break;
        log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);
        double m = max_of(K, le), n = 0.0;
        for (int i = 0; i < K; ++i) {
            double v = 0.0;
            for (int j = 0; j < K; ++j) v += (double)P[i * K + j] * exp(le[j] - m) * beta[j];
            nb[i] = v;
            if (v > n) n = v;
        }
        for (int i = 0; i < K; ++i) beta[i] = nb[i] / n;
    }
    free(alpha); free(beta); free(nb); free(le);
    return logL;
}

/*
 * Expected sufficient statistics of the hidden chain given the observations
 * (the E-step of EM, Baum-Welch; Rabiner 1989, Section III-C), written to
 * `stats` (K*K + 8*K doubles, in this order):
 *   N[i][j] = sum_{t>=1} P(s_{t-1}=i, s_t=j | o)   expected transitions
 *   G0[k]   = P(s_0 = k | o)
 *   Gs[k]   = sum_t gamma_t(k)
 *   Gr[k]   = sum_t gamma_t(k) [tremor at t]
 *   Sx[k], Sy[k]            = sum_t gamma_t(k) [tremor] x_t, y_t
 *   Sxx[k], Sxy[k], Syy[k]  = sum_t gamma_t(k) [tremor] x_t^2, x_t y_t, y_t^2
 * With the Fisher identity (the gradient of log L is the posterior
 * expectation of the gradient of the complete-data log likelihood) these
 * give d log L / d(pi, P, p, mu, Sigma). Returns log L.
 */
double oracle_expected_stats(int K, const float *pi, const float *P, const float *p, const float *mu,
                             const float *cov, int64_t T, const float *xy, const uint8_t *tremor, int init_mode,
                             double *stats)
{
    double *gam = (double *)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1) * K);
    double *fwd = (double *)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1) * K);
    double *beta = (double *)malloc(sizeof(double) * K);
    double *nb = (double *)malloc(sizeof(double) * K);
    double *le = (double *)malloc(sizeof(double) * K);
    double *w = (double *)malloc(sizeof(double) * K);
    double *N = stats, *G0 = stats + K * K, *Gs = G0 + K, *Gr = Gs + K, *Sx = Gr + K, *Sy = Sx + K;
    double *Sxx = Sy + K, *Sxy = Sxx + K, *Syy = Sxy + K;
    memset(stats, 0, sizeof(double) * (size_t)(K * K + 8 * K));
    /* forward vectors (normalised) via the posterior routine's recursion */
    double logL = oracle_posterior(K, pi, P, p, mu, cov, T, xy, tremor, init_mode, gam);
    if (!(logL > -INFINITY) || T == 0) {
        free(gam); free(fwd); free(beta); free(nb); free(le); free(w);
        return logL;
    }
    /* forward vectors again, kept for the pairwise terms */
    {
        double *a = (double *)malloc(sizeof(double) * K);
        initial_vector(K, pi, P, init_mode, a);
        for (int64_t t = 0; t < T; ++t) {
            log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);
            double m = max_of(K, le), c = 0.0;
            for (int j = 0; j < K; ++j) {
                double s;
                if (t == 0) {
                    s = a[j];
                } else {
                    s = 0.0;
                    for (int i = 0; i < K; ++i) s += fwd[(t - 1) * K + i] * (double)P[i * K + j];
                }
                w[j] = s * exp(le[j] - m);
                c += w[j];
            }
            for (int j = 0; j < K; ++j) fwd[t * K + j] = w[j] / c;
        }
        free(a);
    }
    /* backward pass: pairwise posteriors xi_t(i,j) ∝ f_{t-1}(i) P_ij e_j(o_t) b_t(j) */
    for (int k = 0; k < K; ++k) beta[k] = 1.0;
    for (int64_t t = T - 1; t >= 1; --t) {
        log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);
        double m = max_of(K, le), z = 0.0;
        for (int j = 0; j < K; ++j) w[j] = exp(le[j] - m) * beta[j];
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) z += fwd[(t - 1) * K + i] * (double)P[i * K + j] * w[j];
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) N[i * K + j] += fwd[(t - 1) * K + i] * (double)P[i * K + j] * w[j] / z;
        double n = 0.0;
        for (int i = 0; i < K; ++i) {
            double v = 0.0;
            for (int j = 0; j < K; ++j) v += (double)P[i * K + j] * w[j];
            nb[i] = v;
            if (v > n) n = v;
        }
        for (int i = 0; i < K; ++i) beta[i] = nb[i] / n;
    }
    for (int64_t t = 0; t < T; ++t) {
        const int tr = tremor[t] != 0;
        const double x = xy[2 * t], y = xy[2 * t + 1];
        for (int k = 0; k < K; ++k) {
            const double g = gam[t * K + k];
            if (t == 0) G0[k] = g;
            Gs[k] += g;
            if (tr) {
                Gr[k] += g;
                Sx[k] += g * x;
                Sy[k] += g * y;
                Sxx[k] += g * x * x;
                Sxy[k] += g * x * y;
                Syy[k] += g * y * y;
            }
        }
    }
    free(gam); free(fwd); free(beta); free(nb); free(le); free(w);
    return logL;
}

/*
 * The most probable hidden path (Viterbi; Rabiner 1989, Section III-B), in
 * the natural-log domain: delta_0(k) = log v0_k + log e_k(o_0),
 * delta_t(j) = max_i [delta_{t-1}(i) + log P_ij] + log e_j(o_t), with the
 * smallest maximising i kept as the back-pointer, the path ending in the
 * smallest maximising state. Writes path[T]; returns the path's log joint
 * probability log p(s, o) (-inf when every path has probability zero).
 */
double oracle_viterbi(int K, const float *pi, const float *P, const float *p, const float *mu,
                      const float *cov, int64_t T, const float *xy, const uint8_t *tremor, int init_mode,
                      int32_t *path)
{
    if (T == 0) return 0.0;
    double *d = (double *)malloc(sizeof(double) * K);
    double *nd = (double *)malloc(sizeof(double) * K);
    double *le = (double *)malloc(sizeof(double) * K);
    int32_t *bp = (int32_t *)malloc(sizeof(int32_t) * (size_t)T * K);
    initial_vector(K, pi, P, init_mode, d);
    log_emissions(K, p, mu, cov, tremor[0], xy[0], xy[1], le);
    for (int k = 0; k < K; ++k) d[k] = log(d[k]) + le[k];
    for (int64_t t = 1; t < T; ++t) {
        log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);
        for (int j = 0; j < K; ++j) {
            double best = -INFINITY;
            int arg = 0;
            for (int i = 0; i < K; ++i) {
                double v = d[i] + log((double)P[i * K + j]);
                if (v > best) { best = v; arg = i; }
            }
            nd[j] = best + le[j];
            bp[t * K + j] = arg;
        }
        memcpy(d, nd, sizeof(double) * K);
    }
    double best = -INFINITY;
    int arg = 0;
    for (int k = 0; k < K; ++k)
        if (d[k] > best) { best = d[k]; arg = k; }
    path[T - 1] = arg;
    for (int64_t t = T - 1; t >= 1; --t) path[t - 1] = bp[t * K + path[t]];
    free(d); free(nd); free(le); free(bp);
    return best;
}

/* log p(s, o) of a given hidden path (the joint probability of path and data) */
double oracle_path_logjoint(int K, const float *pi, const float *P, const float *p, const float *mu,
                            const float *cov, int64_t T, const float *xy, const uint8_t *tremor, int init_mode,
                            const int32_t *path)
{
    if (T == 0) return 0.0;
    double *v0 = (double *)malloc(sizeof(double) * K);
    double *le = (double *)malloc(sizeof(double) * K);
    initial_vector(K, pi, P, init_mode, v0);
    log_emissions(K, p, mu, cov, tremor[0], xy[0], xy[1], le);
    double s = log(v0[path[0]]) + le[path[0]];
    for (int64_t t = 1; t < T; ++t) {
        log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);
        s += log((double)P[path[t - 1] * K + path[t]]) + le[path[t]];
    }
    free(v0); free(le);
    return s;
}
