// Learned Metropolis-Hastings proposal: a small MLP trained on the random
// walk's own history, with hand-written forward, backward and Adam kernels.
//
// The network maps the standardised state x = (theta - m) / s_in (d inputs)
// through two ReLU layers of H units to 2d outputs (f_mu, f_sig):
//     h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), (f_mu, f_sig) = W3 h2 + b3.
// The proposal is the Gaussian
//     q(theta' | theta) = N(theta + lam s gamma f_mu, diag((lam s exp(f_sig))^2)),
// with f_sig clamped to [-6, 3] (part of the definition of q). It is
// evaluable in both directions, so Metropolis-Hastings with the correction
// log q(theta | theta') - log q(theta' | theta) keeps the posterior exact
// (Section "Monte Carlo Markov Chains": the likelihood x prior ratio still
// decides; the network only proposes).
//
// Training maximises log q(theta_{t+lag} | theta_t) over pairs drawn from a
// random-walk trace: per pair, with r = (y - theta) / s - f_mu and
// sig = exp(f_sig), the loss is sum_i (r_i^2 / (2 sig_i^2) + f_sig,i) (the
// terms that do not depend on the network dropped). Optimiser: Adam
// (Kingma & Ba, ICLR 2015) with bias correction.
//
// All GEMMs are FP32 SIMT tiles: the network costs about 1 MFLOP per chain
// and iteration, against ~10^10 for one likelihood evaluation.
#include <cmath>
#include <cstring>
#include <new>

#include "hmm_internal.cuh"

namespace hmm {
namespace mlp {

constexpr float FSIG_LO = -6.0f, FSIG_HI = 3.0f;

// C[m][n] = alpha * sum_k A(m,k) B(k,n) (+ bias[n]) (relu), beta C + ...
// A(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]
constexpr int TILE = 32;

template <bool TA, bool TB>
__global__ void __launch_bounds__(TILE * 8) gemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                         const float *__restrict__ B, int ldb, float *__restrict__ C,
                                                         int ldc, const float *__restrict__ bias, int relu,
                                                         float beta) {
    __shared__ float sA[TILE][TILE + 1];
    __shared__ float sB[TILE][TILE + 1];
    const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;  // 32 x 8 threads, 4 rows each
    const int m0 = blockIdx.y * TILE, n0 = blockIdx.x * TILE;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += TILE) {
        for (int r = ty; r < TILE; r += 8) {
            const int m = m0 + r, k = k0 + tx;
            sA[r][tx] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
            const int kk = k0 + r, n = n0 + tx;
            sB[r][tx] = (kk < K && n < N) ? (TB ? B[(size_t)n * ldb + kk] : B[(size_t)kk * ldb + n]) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < TILE; ++k) {
            const float b = sB[k][tx];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = fmaf(sA[ty + 8 * i][k], b, acc[i]);
        }
        __syncthreads();
    }
    const int n = n0 + tx;
    if (n >= N) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 8 * i;
        if (m >= M) continue;
        float v = acc[i];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.f);
        float *c = C + (size_t)m * ldc + n;
        *c = beta != 0.f ? beta * *c + v : v;
    }
}

static cudaError_t gemm(bool ta, bool tb, int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                        float *C, int ldc, const float *bias, int relu, float beta, cudaStream_t st) {
    dim3 grid((N + TILE - 1) / TILE, (M + TILE - 1) / TILE), block(TILE * 8);
    if (!ta && !tb) gemm_kernel<false, false><<<grid, block, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, beta);
    else if (!ta && tb) gemm_kernel<false, true><<<grid, block, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, beta);
    else if (ta && !tb) gemm_kernel<true, false><<<grid, block, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, beta);
    else gemm_kernel<true, true><<<grid, block, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, beta);
    return cudaGetLastError();
}

// x = (theta - m) / s
__global__ void standardise_kernel(int B, int d, const float *theta, const float *mean, const float *scale,
                                   float *x) {
    const size_t n = (size_t)B * d;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % d);
        x[i] = (theta[i] - mean[c]) / scale[c];
    }
}

__device__ __forceinline__ float clamp_sig(float v) { return fminf(fmaxf(v, FSIG_LO), FSIG_HI); }

// per-pair loss and gradient wrt the network outputs (mean over the batch)
__global__ void loss_grad_kernel(int B, int d, const float *theta, const float *y, const float *scale,
                                 const float *out, float *dout, double *loss_per_row) {
    const int b = blockIdx.x;
    double part = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        const float fmu = out[(size_t)b * 2 * d + i];
        const float raw = out[(size_t)b * 2 * d + d + i];
        const float fs = clamp_sig(raw);
        const float r = (y[(size_t)b * d + i] - theta[(size_t)b * d + i]) / scale[i] - fmu;
        const float inv = expf(-2.0f * fs);
        const float z2 = r * r * inv;
        part += 0.5 * (double)z2 + (double)fs;
        dout[(size_t)b * 2 * d + i] = -r * inv / (float)B;
        const bool inside = raw > FSIG_LO && raw < FSIG_HI;
        dout[(size_t)b * 2 * d + d + i] = inside ? (1.0f - z2) / (float)B : 0.0f;
    }
    __shared__ double red[128];
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_per_row[b] = red[0];
}

__global__ void mean_kernel(int B, const double *v, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < B; i += 256) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / B;
}

// dZ = dA * (Z > 0) in place on dA (the forward kept post-activation A; A > 0 iff Z > 0)
__global__ void relu_back_kernel(size_t n, const float *act, float *grad) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(act[i] > 0.f)) grad[i] = 0.f;
}

// db[n] = sum_b dZ[b][n]
__global__ void colsum_kernel(int B, int N, const float *dz, float *db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dz[(size_t)b * N + n];
    db[n] = s;
}

__global__ void adam_kernel(size_t n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2,
                            float eps, float bc1, float bc2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// Philox-based initialisation: uniform(-a, a) with a = sqrt(6 / fan_in) (He/Kaiming uniform for ReLU)
__global__ void init_kernel(size_t n, float *w, float a, uint64_t seed, uint32_t stream) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)i, (uint32_t)(i >> 32), stream, 0x4d4c5000u};
        uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
        for (int r = 0; r < 10; ++r) {
            if (r > 0) {
                k0 += 0x9E3779B9u;
                k1 += 0xBB67AE85u;
            }
            const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
            const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
            const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
            c[0] = n0;
            c[1] = lo1;
            c[2] = n2;
            c[3] = lo0;
        }
        const float u = (float)(c[0] >> 8) * (1.0f / 16777216.0f);
        w[i] = a * (2.0f * u - 1.0f);
    }
}

}  // namespace mlp
}  // namespace hmm

using namespace hmm;
using namespace hmm::mlp;

struct hmm_mlp {
    int d = 0, H = 0;
    size_t n_params = 0;
    float *params = nullptr;  // W1 [H][d], b1 [H], W2 [H][H], b2 [H], W3 [2d][H], b3 [2d]
    float *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    float *mean = nullptr, *in_scale = nullptr;  // input standardisation x = (theta - mean) / in_scale
    float *scale = nullptr;                      // proposal / training scale s (displacement units)
    float lam = 1.0f;
    float drift = 1.0f;  // gamma: the proposal mean is theta + lam s gamma f_mu
    long long adam_t = 0;
    // activations for a batch of up to cap rows
    int cap = 0;
    float *x = nullptr, *a1 = nullptr, *a2 = nullptr, *out = nullptr, *dout = nullptr, *d1 = nullptr, *d2 = nullptr;
    double *rowloss = nullptr;

    float *W1() { return params; }
    float *b1() { return params + (size_t)H * d; }
    float *W2() { return b1() + H; }
    float *b2() { return W2() + (size_t)H * H; }
    float *W3() { return b2() + H; }
    float *b3() { return W3() + (size_t)2 * d * H; }
};

static size_t mlp_nparams(int d, int H) { return (size_t)H * d + H + (size_t)H * H + H + (size_t)2 * d * H + 2 * d; }

static int ensure_batch(hmm_mlp *m, int B) {
    if (B <= m->cap) return HMM_OK;
    float *bufs[] = {m->x, m->a1, m->a2, m->out, m->dout, m->d1, m->d2};
    for (float *b : bufs)
        if (b) cudaFree(b);
    if (m->rowloss) cudaFree(m->rowloss);
    m->x = m->a1 = m->a2 = m->out = m->dout = m->d1 = m->d2 = nullptr;
    m->rowloss = nullptr;
    const int d = m->d, H = m->H;
    cudaError_t e = cudaMalloc(&m->x, sizeof(float) * B * d);
    if (e == cudaSuccess) e = cudaMalloc(&m->a1, sizeof(float) * B * H);
    if (e == cudaSuccess) e = cudaMalloc(&m->a2, sizeof(float) * B * H);
    if (e == cudaSuccess) e = cudaMalloc(&m->out, sizeof(float) * B * 2 * d);
    if (e == cudaSuccess) e = cudaMalloc(&m->dout, sizeof(float) * B * 2 * d);
    if (e == cudaSuccess) e = cudaMalloc(&m->d1, sizeof(float) * B * H);
    if (e == cudaSuccess) e = cudaMalloc(&m->d2, sizeof(float) * B * H);
    if (e == cudaSuccess) e = cudaMalloc(&m->rowloss, sizeof(double) * B);
    if (e != cudaSuccess) {
        cudaGetLastError();
        m->cap = 0;
        return HMM_ENOMEM;
    }
    m->cap = B;
    return HMM_OK;
}

// forward of B standardised rows x into out, through the given activation buffers
static cudaError_t forward_ext(hmm_mlp *m, int B, const float *x, float *a1, float *a2, float *out, cudaStream_t st) {
    const int d = m->d, H = m->H;
    cudaError_t e = gemm(false, true, B, H, d, x, d, m->W1(), d, a1, H, m->b1(), 1, 0.f, st);
    if (e == cudaSuccess) e = gemm(false, true, B, H, H, a1, H, m->W2(), H, a2, H, m->b2(), 1, 0.f, st);
    if (e == cudaSuccess) e = gemm(false, true, B, 2 * d, H, a2, H, m->W3(), H, out, 2 * d, m->b3(), 0, 0.f, st);
    return e;
}

// forward of B standardised rows (m->x) into m->out; activations kept for backward
static cudaError_t forward(hmm_mlp *m, int B, cudaStream_t st) { return forward_ext(m, B, m->x, m->a1, m->a2, m->out, st); }

// gradients of the loss wrt every parameter from dout (m->grads, same layout)
static cudaError_t backward(hmm_mlp *m, int B, cudaStream_t st) {
    const int d = m->d, H = m->H;
    float *g = m->grads;
    float *gW1 = g, *gb1 = gW1 + (size_t)H * d, *gW2 = gb1 + H, *gb2 = gW2 + (size_t)H * H, *gW3 = gb2 + H,
          *gb3 = gW3 + (size_t)2 * d * H;
    // layer 3: dW3 = dout^T a2, db3 = colsum dout, d2 = dout W3 (then relu')
    cudaError_t e = gemm(true, false, 2 * d, H, B, m->dout, 2 * d, m->a2, H, gW3, H, nullptr, 0, 0.f, st);
    if (e == cudaSuccess) {
        colsum_kernel<<<(2 * d + 127) / 128, 128, 0, st>>>(B, 2 * d, m->dout, gb3);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = gemm(false, false, B, H, 2 * d, m->dout, 2 * d, m->W3(), H, m->d2, H, nullptr, 0, 0.f, st);
    if (e == cudaSuccess) {
        relu_back_kernel<<<256, 256, 0, st>>>((size_t)B * H, m->a2, m->d2);
        e = gemm(true, false, H, H, B, m->d2, H, m->a1, H, gW2, H, nullptr, 0, 0.f, st);
    }
    if (e == cudaSuccess) {
        colsum_kernel<<<(H + 127) / 128, 128, 0, st>>>(B, H, m->d2, gb2);
        e = gemm(false, false, B, H, H, m->d2, H, m->W2(), H, m->d1, H, nullptr, 0, 0.f, st);
    }
    if (e == cudaSuccess) {
        relu_back_kernel<<<256, 256, 0, st>>>((size_t)B * H, m->a1, m->d1);
        e = gemm(true, false, H, d, B, m->d1, H, m->x, d, gW1, d, nullptr, 0, 0.f, st);
    }
    if (e == cudaSuccess) {
        colsum_kernel<<<(H + 127) / 128, 128, 0, st>>>(B, H, m->d1, gb1);
        e = cudaGetLastError();
    }
    return e;
}

static int loss_and_grad(hmm_mlp *m, int B, const float *theta, const float *y, double *loss_dev, cudaStream_t st) {
    int rc = ensure_batch(m, B);
    if (rc) return rc;
    standardise_kernel<<<256, 256, 0, st>>>(B, m->d, theta, m->mean, m->in_scale, m->x);
    cudaError_t e = forward(m, B, st);
    if (e == cudaSuccess) {
        loss_grad_kernel<<<B, 128, 0, st>>>(B, m->d, theta, y, m->scale, m->out, m->dout, m->rowloss);
        mean_kernel<<<1, 256, 0, st>>>(B, m->rowloss, loss_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward(m, B, st);
    return e == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

extern "C" {

int hmm_mlp_create(hmm_mlp **out, int32_t d, int32_t hidden, uint64_t seed, void *stream) {
    if (!out || d < 1 || hidden < 1) return HMM_EINVAL;
    *out = nullptr;
    hmm_mlp *m = new (std::nothrow) hmm_mlp();
    if (!m) return HMM_ENOMEM;
    m->d = d;
    m->H = hidden;
    m->n_params = mlp_nparams(d, hidden);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&m->params, sizeof(float) * m->n_params);
    if (e == cudaSuccess) e = cudaMalloc(&m->grads, sizeof(float) * m->n_params);
    if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, sizeof(float) * m->n_params);
    if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, sizeof(float) * m->n_params);
    if (e == cudaSuccess) e = cudaMalloc(&m->mean, sizeof(float) * d);
    if (e == cudaSuccess) e = cudaMalloc(&m->scale, sizeof(float) * d);
    if (e == cudaSuccess) e = cudaMalloc(&m->in_scale, sizeof(float) * d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return HMM_ENOMEM;
    }
    // He-uniform weights, zero biases; the last layer starts small so the
    // untrained proposal is a narrow random walk
    cudaMemsetAsync(m->params, 0, sizeof(float) * m->n_params, st);
    init_kernel<<<256, 256, 0, st>>>((size_t)hidden * d, m->W1(), sqrtf(6.0f / d), seed, 1);
    init_kernel<<<256, 256, 0, st>>>((size_t)hidden * hidden, m->W2(), sqrtf(6.0f / hidden), seed, 2);
    init_kernel<<<256, 256, 0, st>>>((size_t)2 * d * hidden, m->W3(), 0.01f * sqrtf(6.0f / hidden), seed, 3);
    cudaMemsetAsync(m->adam_m, 0, sizeof(float) * m->n_params, st);
    cudaMemsetAsync(m->adam_v, 0, sizeof(float) * m->n_params, st);
    // identity standardisation until set
    float *ones = new float[d];
    for (int i = 0; i < d; ++i) ones[i] = 1.0f;
    cudaMemsetAsync(m->mean, 0, sizeof(float) * d, st);
    e = cudaMemcpyAsync(m->scale, ones, sizeof(float) * d, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->in_scale, ones, sizeof(float) * d, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    delete[] ones;
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return HMM_ECUDA;
    }
    *out = m;
    return HMM_OK;
}

int hmm_mlp_destroy(hmm_mlp *m) {
    if (!m) return HMM_OK;
    float *bufs[] = {m->params, m->grads, m->adam_m, m->adam_v, m->mean, m->scale, m->in_scale, m->x, m->a1, m->a2,
                     m->out, m->dout, m->d1, m->d2};
    for (float *b : bufs)
        if (b) cudaFree(b);
    if (m->rowloss) cudaFree(m->rowloss);
    delete m;
    return HMM_OK;
}

int64_t hmm_mlp_num_params(const hmm_mlp *m) { return m ? (int64_t)m->n_params : -1; }

int hmm_mlp_params(hmm_mlp *m, float *params_dev, int set, void *stream) {
    if (!m || !params_dev) return HMM_EINVAL;
    cudaError_t e = set ? cudaMemcpyAsync(m->params, params_dev, sizeof(float) * m->n_params, cudaMemcpyDeviceToDevice,
                                          (cudaStream_t)stream)
                        : cudaMemcpyAsync(params_dev, m->params, sizeof(float) * m->n_params, cudaMemcpyDeviceToDevice,
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

int hmm_mlp_set_scaling(hmm_mlp *m, const float *mean_dev, const float *in_scale_dev, const float *scale_dev,
                        float lam, void *stream) {
    if (!m || !mean_dev || !in_scale_dev || !scale_dev || !(lam > 0.f)) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(m->mean, mean_dev, sizeof(float) * m->d, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->in_scale, in_scale_dev, sizeof(float) * m->d, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->scale, scale_dev, sizeof(float) * m->d, cudaMemcpyDeviceToDevice, st);
    m->lam = lam;
    return e == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

int hmm_mlp_forward(hmm_mlp *m, int32_t B, const float *theta, float *out_dev, void *stream) {
    if (!m || B < 1 || !theta || !out_dev) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_batch(m, B);
    if (rc) return rc;
    standardise_kernel<<<256, 256, 0, st>>>(B, m->d, theta, m->mean, m->in_scale, m->x);
    cudaError_t e = forward(m, B, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_dev, m->out, sizeof(float) * B * 2 * m->d, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

int hmm_mlp_loss_grad(hmm_mlp *m, int32_t B, const float *theta, const float *y, double *loss_dev,
                      float *grads_dev, void *stream) {
    if (!m || B < 1 || !theta || !y || !loss_dev) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = loss_and_grad(m, B, theta, y, loss_dev, st);
    if (rc) return rc;
    if (grads_dev &&
        cudaMemcpyAsync(grads_dev, m->grads, sizeof(float) * m->n_params, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return HMM_ECUDA;
    return HMM_OK;
}

int hmm_mlp_adam_step(hmm_mlp *m, float lr, float beta1, float beta2, float eps, void *stream) {
    if (!m) return HMM_EINVAL;
    m->adam_t += 1;
    const float bc1 = 1.0f - powf(beta1, (float)m->adam_t), bc2 = 1.0f - powf(beta2, (float)m->adam_t);
    adam_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(m->n_params, m->params, m->grads, m->adam_m, m->adam_v, lr,
                                                        beta1, beta2, eps, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

}  // extern "C"

// ---- used by the sampler (hmm_mcmc.cu) ----
namespace hmm {

int mlp_dim(const hmm_mlp *m) { return m->d; }
float mlp_lambda(const hmm_mlp *m) { return m->lam; }
float mlp_drift(const hmm_mlp *m) { return m->drift; }
const float *mlp_scale(const hmm_mlp *m) { return m->scale; }

int mlp_hidden(const hmm_mlp *m) { return m->H; }
const float *mlp_mean(const hmm_mlp *m) { return m->mean; }

// What a proposal built on the network depends on (sampler checkpoints):
// the parameters, the input standardisation (mean, in_scale), the scale,
// lam and the drift factor; n_params + 3d floats plus the two scalars.
size_t mlp_state_floats(const hmm_mlp *m) { return m->n_params + 3 * (size_t)m->d; }

cudaError_t mlp_state_io(hmm_mlp *m, float *host, float *lam, float *drift, bool save, cudaStream_t st) {
    float *dev[4] = {m->params, m->mean, m->in_scale, m->scale};
    const size_t n[4] = {m->n_params, (size_t)m->d, (size_t)m->d, (size_t)m->d};
    cudaError_t e = cudaSuccess;
    size_t o = 0;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
        e = save ? cudaMemcpyAsync(host + o, dev[i], sizeof(float) * n[i], cudaMemcpyDeviceToHost, st)
                 : cudaMemcpyAsync(dev[i], host + o, sizeof(float) * n[i], cudaMemcpyHostToDevice, st);
        o += n[i];
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (save) {
        *lam = m->lam;
        *drift = m->drift;
    } else if (e == cudaSuccess) {
        m->lam = *lam;
        m->drift = *drift;
    }
    return e;
}

// network outputs for B states into out (B x 2d) through caller-owned buffers
// x [B][d], a1 and a2 [B][H] (their addresses stay fixed under a CUDA graph)
int mlp_eval(hmm_mlp *m, int B, const float *theta, float *x, float *a1, float *a2, float *out, cudaStream_t st) {
    standardise_kernel<<<256, 256, 0, st>>>(B, m->d, theta, m->mean, m->in_scale, x);
    return forward_ext(m, B, x, a1, a2, out, st) == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

}  // namespace hmm

// ---- training loop and data statistics (all on the device) ----
namespace hmm {
namespace mlp {

// rows idx[b] = Philox(seed, step, b) mod n of X and Y into Xb, Yb
__global__ void gather_pairs_kernel(int B, int d, int n, const float *X, const float *Y, uint64_t seed, uint32_t step,
                                    float *Xb, float *Yb) {
    const int b = blockIdx.x;
    uint32_t c[4] = {(uint32_t)b, step, 0x7261696eu, 0u};
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    const uint64_t wide = ((uint64_t)c[0] << 32) | c[1];
    const int row = (int)(wide % (uint64_t)n);
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        Xb[(size_t)b * d + i] = X[(size_t)row * d + i];
        Yb[(size_t)b * d + i] = Y[(size_t)row * d + i];
    }
}

// per-column mean and standard deviation of X, and standard deviation of Y - X (FP64)
__global__ void pair_stats_kernel(int n, int d, const float *X, const float *Y, float *mean, float *in_scale,
                                  float *scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double sx = 0.0, sd = 0.0;
    for (int r = 0; r < n; ++r) {
        sx += X[(size_t)r * d + i];
        sd += (double)Y[(size_t)r * d + i] - X[(size_t)r * d + i];
    }
    const double mx = sx / n, md = sd / n;
    double v = 0.0, vx = 0.0;
    for (int r = 0; r < n; ++r) {
        const double e = (double)Y[(size_t)r * d + i] - X[(size_t)r * d + i] - md;
        const double ex = (double)X[(size_t)r * d + i] - mx;
        v += e * e;
        vx += ex * ex;
    }
    mean[i] = (float)mx;
    scale[i] = (float)fmax(sqrt(v / fmax(1.0, n - 1.0)), 1e-6);
    in_scale[i] = (float)fmax(sqrt(vx / fmax(1.0, n - 1.0)), 1e-6);
}

}  // namespace mlp
}  // namespace hmm

extern "C" {

int hmm_mlp_fit_scaling(hmm_mlp *m, int32_t n, const float *X, const float *Y, float lam, void *stream) {
    if (!m || n < 2 || !X || !Y || !(lam > 0.f)) return HMM_EINVAL;
    pair_stats_kernel<<<(m->d + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n, m->d, X, Y, m->mean, m->in_scale,
                                                                              m->scale);
    m->lam = lam;
    return cudaGetLastError() == cudaSuccess ? HMM_OK : HMM_ECUDA;
}

int hmm_mlp_set_lambda(hmm_mlp *m, float lam, float drift) {
    if (!m || !(lam > 0.f) || !(drift >= 0.f)) return HMM_EINVAL;
    m->lam = lam;
    m->drift = drift;
    return HMM_OK;
}

int hmm_mlp_train(hmm_mlp *m, int32_t n, const float *X, const float *Y, int32_t n_steps, int32_t batch, float lr,
                  uint64_t seed, double *loss_trace, void *stream) {
    if (!m || n < 1 || !X || !Y || n_steps < 0 || batch < 1 || !(lr > 0.f)) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int d = m->d;
    float *Xb = nullptr, *Yb = nullptr;
    double *loss = nullptr;
    cudaError_t e = cudaMalloc(&Xb, sizeof(float) * batch * d);
    if (e == cudaSuccess) e = cudaMalloc(&Yb, sizeof(float) * batch * d);
    if (e == cudaSuccess) e = cudaMalloc(&loss, sizeof(double));
    int rc = e == cudaSuccess ? HMM_OK : HMM_ENOMEM;
    for (int s = 0; s < n_steps && rc == HMM_OK; ++s) {
        gather_pairs_kernel<<<batch, 128, 0, st>>>(batch, d, n, X, Y, seed, (uint32_t)s, Xb, Yb);
        rc = loss_and_grad(m, batch, Xb, Yb, loss, st);
        if (rc == HMM_OK) rc = hmm_mlp_adam_step(m, lr, 0.9f, 0.999f, 1e-8f, stream);
        if (rc == HMM_OK && loss_trace &&
            cudaMemcpyAsync(loss_trace + s, loss, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = HMM_ECUDA;
    }
    cudaStreamSynchronize(st);  // the minibatch buffers are freed below
    if (Xb) cudaFree(Xb);
    if (Yb) cudaFree(Yb);
    if (loss) cudaFree(loss);
    return rc;
}

}  // extern "C"
