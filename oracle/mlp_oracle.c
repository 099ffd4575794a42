/*
 * CPU oracle for the learned proposal's network -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain FP64 loops, no blocking: the forward pass, the training loss and its
 * gradient by backpropagation written out layer by layer, and one Adam step
 * (Kingma & Ba, "Adam: a method for stochastic optimization", ICLR 2015,
 * Algorithm 1, with bias correction).
 *
 * Network: x = (theta - mean) / in_scale; h1 = relu(W1 x + b1);
 * h2 = relu(W2 h1 + b2); out = W3 h2 + b3 = (f_mu [d], f_sig [d]).
 * Loss over B pairs (theta_b, y_b): mean_b sum_i ( r_i^2 / (2 e^{2 s_i}) + s_i ),
 * r = (y - theta) / scale - f_mu, s = clamp(f_sig, -6, 3).
 * Parameter layout: W1 [H][d], b1 [H], W2 [H][H], b2 [H], W3 [2d][H], b3 [2d].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* forward for one row; h1, h2 (H each) and out (2d) are written */
static void fwd_row(int d, int H, const double *p, const double *x, double *h1, double *h2, double *out)
{
    const double *W1 = p, *b1 = W1 + (size_t)H * d, *W2 = b1 + H, *b2 = W2 + (size_t)H * H;
    const double *W3 = b2 + H, *b3 = W3 + (size_t)2 * d * H;
    for (int j = 0; j < H; ++j) {
        double s = b1[j];
        for (int i = 0; i < d; ++i) s += W1[(size_t)j * d + i] * x[i];
        h1[j] = s > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < H; ++j) {
        double s = b2[j];
        for (int i = 0; i < H; ++i) s += W2[(size_t)j * H + i] * h1[i];
        h2[j] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < 2 * d; ++o) {
        double s = b3[o];
        for (int i = 0; i < H; ++i) s += W3[(size_t)o * H + i] * h2[i];
        out[o] = s;
    }
}

void oracle_mlp_forward(int d, int H, const double *params, const double *mean, const double *in_scale, int B,
                        const double *theta, double *out)
{
    double *x = (double *)malloc(sizeof(double) * d);
    double *h1 = (double *)malloc(sizeof(double) * H), *h2 = (double *)malloc(sizeof(double) * H);
    for (int b = 0; b < B; ++b) {
        for (int i = 0; i < d; ++i) x[i] = (theta[(size_t)b * d + i] - mean[i]) / in_scale[i];
        fwd_row(d, H, params, x, h1, h2, out + (size_t)b * 2 * d);
    }
    free(x); free(h1); free(h2);
}

/* loss (returned) and its gradient wrt every parameter (grad, same layout) */
double oracle_mlp_loss_grad(int d, int H, const double *params, const double *mean, const double *in_scale,
                            const double *scale, int B, const double *theta, const double *y, double *grad)
{
    size_t np = (size_t)H * d + H + (size_t)H * H + H + (size_t)2 * d * H + 2 * d;
    memset(grad, 0, sizeof(double) * np);
    const double *W2 = params + (size_t)H * d + H, *W3 = W2 + (size_t)H * H + H;
    double *gW1 = grad, *gb1 = gW1 + (size_t)H * d, *gW2 = gb1 + H, *gb2 = gW2 + (size_t)H * H;
    double *gW3 = gb2 + H, *gb3 = gW3 + (size_t)2 * d * H;
    double *x = (double *)malloc(sizeof(double) * d);
    double *h1 = (double *)malloc(sizeof(double) * H), *h2 = (double *)malloc(sizeof(double) * H);
    double *out = (double *)malloc(sizeof(double) * 2 * d), *dout = (double *)malloc(sizeof(double) * 2 * d);
    double *dh1 = (double *)malloc(sizeof(double) * H), *dh2 = (double *)malloc(sizeof(double) * H);
    double loss = 0.0;
    for (int b = 0; b < B; ++b) {
        const double *th = theta + (size_t)b * d, *yy = y + (size_t)b * d;
        for (int i = 0; i < d; ++i) x[i] = (th[i] - mean[i]) / in_scale[i];
        fwd_row(d, H, params, x, h1, h2, out);
        /* d loss / d out */
        for (int i = 0; i < d; ++i) {
            double raw = out[d + i];
            double s = clampd(raw, -6.0, 3.0);
            double r = (yy[i] - th[i]) / scale[i] - out[i];
            double inv = exp(-2.0 * s);
            loss += 0.5 * r * r * inv + s;
            dout[i] = -r * inv / B;
            dout[d + i] = (raw > -6.0 && raw < 3.0) ? (1.0 - r * r * inv) / B : 0.0;
        }
        /* layer 3 */
        for (int o = 0; o < 2 * d; ++o) {
            gb3[o] += dout[o];
            for (int i = 0; i < H; ++i) gW3[(size_t)o * H + i] += dout[o] * h2[i];
        }
        for (int i = 0; i < H; ++i) {
            double s = 0.0;
            for (int o = 0; o < 2 * d; ++o) s += dout[o] * W3[(size_t)o * H + i];
            dh2[i] = h2[i] > 0.0 ? s : 0.0;
        }
        /* layer 2 */
        for (int j = 0; j < H; ++j) {
            gb2[j] += dh2[j];
            for (int i = 0; i < H; ++i) gW2[(size_t)j * H + i] += dh2[j] * h1[i];
        }
        for (int i = 0; i < H; ++i) {
            double s = 0.0;
            for (int j = 0; j < H; ++j) s += dh2[j] * W2[(size_t)j * H + i];
            dh1[i] = h1[i] > 0.0 ? s : 0.0;
        }
        /* layer 1 */
        for (int j = 0; j < H; ++j) {
            gb1[j] += dh1[j];
            for (int i = 0; i < d; ++i) gW1[(size_t)j * d + i] += dh1[j] * x[i];
        }
    }
    free(x); free(h1); free(h2); free(out); free(dout); free(dh1); free(dh2);
    return loss / B;
}

/* Adam (Algorithm 1 of Kingma & Ba) for step t >= 1 */
void oracle_adam_step(size_t n, double *p, const double *g, double *m, double *v, int t, double lr, double b1,
                      double b2, double eps)
{
    for (size_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / (1.0 - pow(b1, t));
        double vh = v[i] / (1.0 - pow(b2, t));
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
