/*
 * CPU oracle for the t-walk proposal -- TEST INFRASTRUCTURE ONLY (loaded by
 * the tests, never by the product path).
 *
 * The paper samples its posterior with the t-walk (Section "Monte Carlo
 * Markov Chains"; Christen & Fox, "A general purpose sampling algorithm for
 * continuous distributions (the t-walk)", Bayesian Analysis 5(2), 2010).
 * The t-walk keeps two points (x, x') in the parameter space. Each
 * iteration moves one of them, chosen with probability 1/2, with the other
 * as reference; a random subset phi of the coordinates (each with
 * probability min(n, n1)/n, drawn again while empty) is moved by one of
 * four kernels:
 *   traverse (prob 0.4918): y = r + beta (r - h), beta from the density
 *            (a_t - 1)(a_t + 1)/(2 a_t) beta^(a_t) on (0, 1] and the same
 *            constant times beta^(-a_t) above 1 (so g(beta) = g(1/beta));
 *            acceptance factor beta^(n_phi - 2);
 *   walk     (prob 0.4918): y = h + (h - r) z, z from the density
 *            proportional to 1/sqrt(1 + z) on [-a_w/(1+a_w), a_w]; symmetric;
 *   blow     (prob 0.0082): y = r + sigma z, z ~ N(0, I), sigma the largest
 *            |r_j - h_j| over phi; acceptance uses the proposal densities
 *            both ways (the reverse move's sigma is computed from y);
 *   hop      (prob 0.0082): y = h + (sigma / 3) z, likewise.
 * Here h is the point being moved and r the reference; coordinates outside
 * phi are unchanged. Parameters a_w = 1.5, a_t = 6, n1 = 4.
 *
 * Random numbers are Philox draws (mcmc_oracle.c) with these counter
 * streams (the fourth counter word): side, kernel and beta uniforms 2;
 * walk uniforms 3; blow/hop normals 4; subset attempt a uses 9 + a.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

double oracle_normal(uint64_t seed, uint32_t stream, uint32_t chain, uint32_t iter, uint32_t index);
double oracle_uniform(uint64_t seed, uint32_t stream, uint32_t chain, uint32_t iter, uint32_t index);

#define TW_AW 1.5
#define TW_AT 6.0
#define TW_N1 4.0
#define TW_F_TRAVERSE 0.4918
#define TW_F_WALK 0.9836
#define TW_F_BLOW 0.9918
#define TW_MAX_ATTEMPTS 64

enum { TW_TRAVERSE = 0, TW_WALK = 1, TW_BLOW = 2, TW_HOP = 3 };

/* log density of the coordinates phi of w under N(centre, s^2 I), without
 * the 2 pi term (it cancels in the ratio of forward and reverse moves) */
static double lnorm_phi(int n, const unsigned char *phi, const double *w, const double *centre, double s)
{
    double q = 0.0;
    int m = 0;
    for (int j = 0; j < n; ++j)
        if (phi[j]) {
            double d = (w[j] - centre[j]) / s;
            q += d * d;
            ++m;
        }
    return -0.5 * q - m * log(s);
}

static double sigma_phi(int n, const unsigned char *phi, const double *a, const double *b)
{
    double s = 0.0;
    for (int j = 0; j < n; ++j)
        if (phi[j]) s = fmax(s, fabs(a[j] - b[j]));
    return s;
}

/*
 * One t-walk proposal for chain `chain` at iteration `iter`.
 * x, xp: the two current points (n floats). Outputs: *side (0: x moves with
 * reference x', 1: x' moves with reference x), *kernel, *nphi, y (n floats,
 * the proposal for the moving point, rounded to float), *W (log of the
 * acceptance factor besides the target ratio; -inf for a degenerate move).
 * The scratch buffer `work` holds 6 n doubles (the last n as n bytes).
 */
static void twalk_propose_f(int n, const float *x, const float *xp, uint64_t seed, uint32_t chain,
                            uint32_t iter, const double *F, int *side, int *kernel, int *nphi, float *y, double *W,
                            double *work)
{
    double *h = work, *r = work + n, *yd = work + 2 * n, *yr = work + 3 * n;
    unsigned char *phi = (unsigned char *)(work + 5 * n);
    *side = oracle_uniform(seed, 1, chain, iter, 0) < 0.5 ? 0 : 1;
    const float *hf = *side == 0 ? x : xp, *rf = *side == 0 ? xp : x;
    for (int j = 0; j < n; ++j) {
        h[j] = hf[j];
        r[j] = rf[j];
    }
    const double uk = oracle_uniform(seed, 1, chain, iter, 1);
    *kernel = uk < F[0] ? TW_TRAVERSE : uk < F[1] ? TW_WALK : uk < F[2] ? TW_BLOW : TW_HOP;
    /* the subset phi: independent coordinates, drawn again while empty */
    const double pphi = (n < TW_N1 ? n : TW_N1) / (double)n;
    int m = 0;
    for (int a = 0; a < TW_MAX_ATTEMPTS && m == 0; ++a) {
        m = 0;
        for (int j = 0; j < n; ++j) {
            phi[j] = oracle_uniform(seed, 8 + a, chain, iter, j) < pphi;
            m += phi[j];
        }
    }
    if (m == 0) { /* practically unreachable: move every coordinate */
        for (int j = 0; j < n; ++j) phi[j] = 1;
        m = n;
    }
    *nphi = m;
    double w = 0.0;
    memcpy(yd, h, sizeof(double) * n);
    if (*kernel == TW_TRAVERSE) {
        const double u1 = oracle_uniform(seed, 1, chain, iter, 2), u2 = oracle_uniform(seed, 1, chain, iter, 3);
        const double beta = u1 < (TW_AT - 1.0) / (2.0 * TW_AT) ? pow(u2, 1.0 / (TW_AT + 1.0))
                                                                : pow(u2, 1.0 / (1.0 - TW_AT));
        for (int j = 0; j < n; ++j)
            if (phi[j]) yd[j] = r[j] + beta * (r[j] - h[j]);
        w = (m - 2) * log(beta);
    } else if (*kernel == TW_WALK) {
        for (int j = 0; j < n; ++j)
            if (phi[j]) {
                const double u = oracle_uniform(seed, 2, chain, iter, j);
                const double z = TW_AW / (1.0 + TW_AW) * (-1.0 + 2.0 * u + TW_AW * u * u);
                yd[j] = h[j] + (h[j] - r[j]) * z;
            }
    } else {
        const double sig = sigma_phi(n, phi, r, h);
        if (!(sig > 0.0)) {
            w = -INFINITY;
        } else {
            const int blow = *kernel == TW_BLOW;
            const double s = blow ? sig : sig / 3.0;
            for (int j = 0; j < n; ++j)
                if (phi[j]) yd[j] = (blow ? r[j] : h[j]) + s * oracle_normal(seed, 4, chain, iter, j);
        }
    }
    for (int j = 0; j < n; ++j) {
        y[j] = (float)yd[j];
        yr[j] = y[j];
    }
    if ((*kernel == TW_BLOW || *kernel == TW_HOP) && w == 0.0) {
        /* densities of the rounded proposal both ways */
        const int blow = *kernel == TW_BLOW;
        const double sf = sigma_phi(n, phi, r, h), sb = sigma_phi(n, phi, r, yr);
        if (!(sb > 0.0)) {
            w = -INFINITY;
        } else if (blow) {
            w = lnorm_phi(n, phi, h, r, sb) - lnorm_phi(n, phi, yr, r, sf);
        } else {
            w = lnorm_phi(n, phi, h, yr, sb / 3.0) - lnorm_phi(n, phi, yr, h, sf / 3.0);
        }
    }
    *W = w;
}

void oracle_twalk_propose(int n, const float *x, const float *xp, uint64_t seed, uint32_t chain, uint32_t iter,
                          int *side, int *kernel, int *nphi, float *y, double *W, double *work)
{
    static const double F[3] = {TW_F_TRAVERSE, TW_F_WALK, TW_F_BLOW};
    twalk_propose_f(n, x, xp, seed, chain, iter, F, side, kernel, nphi, y, W, work);
}

/*
 * A whole t-walk run on the standard normal target in n dimensions (a pin:
 * the sampler must reproduce its moments). x0, xp0: starting points;
 * F: the cumulative kernel probabilities (traverse, + walk, + blow; the
 * default is the published mixture, and a run may use one kernel alone);
 * samples: n_iter x n floats (the x point after every iteration);
 * work: 6 n doubles followed by 3 n floats.
 */
void oracle_twalk_gauss_run(int n, int n_iter, uint64_t seed, const double *F, const float *x0, const float *xp0,
                            float *samples, double *work)
{
    float *x = (float *)(work + 6 * n), *xp = x + n, *y = xp + n;
    memcpy(x, x0, sizeof(float) * n);
    memcpy(xp, xp0, sizeof(float) * n);
    double lx = 0.0, lxp = 0.0;
    for (int j = 0; j < n; ++j) {
        lx -= 0.5 * (double)x[j] * x[j];
        lxp -= 0.5 * (double)xp[j] * xp[j];
    }
    for (int it = 0; it < n_iter; ++it) {
        int side, kernel, m;
        double W;
        twalk_propose_f(n, x, xp, seed, 0, (uint32_t)it, F, &side, &kernel, &m, y, &W, work);
        double ly = 0.0;
        for (int j = 0; j < n; ++j) ly -= 0.5 * (double)y[j] * y[j];
        const double lcur = side == 0 ? lx : lxp;
        const double u = oracle_uniform(seed, 0, 0, (uint32_t)it, 0);
        if (W > -INFINITY && log(u) < ly - lcur + W) {
            if (side == 0) {
                memcpy(x, y, sizeof(float) * n);
                lx = ly;
            } else {
                memcpy(xp, y, sizeof(float) * n);
                lxp = ly;
            }
        }
        memcpy(samples + (size_t)it * n, x, sizeof(float) * n);
    }
}
