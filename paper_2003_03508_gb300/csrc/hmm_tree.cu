// Combining the chunk products (Section "Step 3": the products the compute
// units return are combined into the likelihood, with the scale coefficients
// carried along so nothing underflows).
//
// tree_level: one CTA multiplies up to TREE_GROUP consecutive products of one
//   (proposal, segment) in order, X <- X * Y, keeping a power-of-two exponent
//   per row: with X = diag(2^ex) X~ and Y = diag(2^ey) Y~,
//     row i of X Y = 2^(ex_i + m_i) sum_k (X~_ik 2^(ey_k - m_i)) Y~_k,
//     m_i = max over the k with X~_ik > 0 of (ey_k + exponent of X~_ik),
//   so every term of row i is at most 2 and the largest is at least 1; a term
//   that falls below the float range next to it is negligible in that row's
//   sum. The alignment is per row of the result: rows of Y can differ in
//   scale by far more than the float range (a reducible P), and a row of the
//   result may draw only on the small ones. Every row of the result is then
//   renormalised to [1, 2). Exponents are int64 (exact). The grouping is
//   fixed by the chunk count, so the result does not depend on scheduling.
// final: per proposal, per segment in order, the head vector
//   h_k = pi0_k e_k(x_0) (pi0 = pi, or P^T pi for the transition-first form)
//   is formed in FP64 and combined with the segment's product:
//     log L_s = M + log sum_j sum_i exp(log h_i + ex_i ln 2 - M) X~_ij.
//   The per-segment values are summed in segment order in FP64.
#include <climits>
#include <math.h>

#include "hmm_internal.cuh"

namespace hmm {

constexpr int TREE_THREADS = 256;

template <bool E32>
__global__ void __launch_bounds__(TREE_THREADS)
tree_level_kernel(int KP, int level, const TreeGroup *__restrict__ groups, LevelPtrs lv,
                  unsigned *__restrict__ status) {
    extern __shared__ __align__(16) float smem[];
    float *X = smem;
    float *Y = X + KP * KP;
    long long *ex = reinterpret_cast<long long *>(Y + KP * KP);
    long long *ey = ex + KP;
    long long *mrow = ey + KP;  // m_i of the current product

    const int q = blockIdx.y;
    const TreeGroup g = groups[blockIdx.x];
    const size_t nin = (size_t)lv.n[level];
    const float *Ain = lv.A[level] + (size_t)q * nin * KP * KP;
    const size_t nout = (size_t)lv.n[level + 1];
    float *Aout = lv.A[level + 1] + (size_t)q * nout * KP * KP;
    long long *eout = reinterpret_cast<long long *>(lv.e[level + 1]) + (size_t)q * nout * KP;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = TREE_THREADS / 32;

    auto load_e = [&](size_t m, int k) -> long long {
        if (E32) {
            int32_t v = reinterpret_cast<const int32_t *>(lv.e[level])[((size_t)q * nin + m) * KP + k];
            return v == ZERO_ROW_EXP32 ? ZERO_ROW_EXP64 : (long long)v;
        }
        return reinterpret_cast<const long long *>(lv.e[level])[((size_t)q * nin + m) * KP + k];
    };

    for (int idx = tid; idx < KP * KP; idx += TREE_THREADS) X[idx] = Ain[(size_t)g.src * KP * KP + idx];
    for (int k = tid; k < KP; k += TREE_THREADS) ex[k] = load_e(g.src, k);
    bool bad = false;
    for (int m = 1; m < g.cnt; ++m) {
        const size_t src = (size_t)g.src + m;
        for (int k = tid; k < KP; k += TREE_THREADS) ey[k] = load_e(src, k);
        for (int idx = tid; idx < KP * KP; idx += TREE_THREADS) Y[idx] = Ain[src * KP * KP + idx];
        __syncthreads();
        // per row of X (warp per row): m_i, then X~_ik <- X~_ik 2^(ey_k - m_i)
        for (int i = warp; i < KP; i += nwarps) {
            long long mm = LLONG_MIN;
            for (int k = lane; k < KP; k += 32) {
                const float x = X[i * KP + k];
                if (x > 0.0f && ey[k] != ZERO_ROW_EXP64) {
                    const long long v = ey[k] + float_exponent(x);
                    mm = v > mm ? v : mm;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                long long other = __shfl_xor_sync(0xffffffffu, mm, o);
                mm = other > mm ? other : mm;
            }
            for (int k = lane; k < KP; k += 32) {
                const float x = X[i * KP + k];
                float w = 0.0f;
                if (mm != LLONG_MIN && x > 0.0f && ey[k] != ZERO_ROW_EXP64) {
                    long long dd = ey[k] - mm;  // <= 127: x 2^dd <= 2
                    dd = dd < -400 ? -400 : dd;
                    w = ldexpf(x, (int)dd);
                }
                X[i * KP + k] = w;
            }
            if (lane == 0) mrow[i] = mm;
        }
        __syncthreads();
        // Z = X * Y, each thread a strided set of entries, held in registers
        float z[(80 * 80 + TREE_THREADS - 1) / TREE_THREADS];
        int nz = 0;
        if (KP == 32) {
            // the same entries (row tid/32 + 8n, column tid%32) and the same k
            // order, with each Y element loaded once for the thread's four rows
            // and X read as 16-byte words (the same row across the warp)
            const int j = tid & 31, r = tid >> 5;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < 32; k += 4) {
                const float y0 = Y[k * 32 + j], y1 = Y[(k + 1) * 32 + j], y2 = Y[(k + 2) * 32 + j],
                            y3 = Y[(k + 3) * 32 + j];
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    const float4 x = *reinterpret_cast<const float4 *>(X + (r + 8 * n) * 32 + k);
                    acc[n] = fmaf(x.w, y3, fmaf(x.z, y2, fmaf(x.y, y1, fmaf(x.x, y0, acc[n]))));
                }
            }
#pragma unroll
            for (int n = 0; n < 4; ++n) z[n] = acc[n];
        } else {
            for (int idx = tid; idx < KP * KP; idx += TREE_THREADS, ++nz) {
                int i = idx / KP, j = idx % KP;
                float acc = 0.0f;
                for (int k = 0; k < KP; ++k) acc = fmaf(X[i * KP + k], Y[k * KP + j], acc);
                z[nz] = acc;
            }
        }
        __syncthreads();
        nz = 0;
        for (int idx = tid; idx < KP * KP; idx += TREE_THREADS, ++nz) X[idx] = z[nz];
        __syncthreads();
        // renormalise each row to [1, 2) (warp per row)
        for (int i = warp; i < KP; i += nwarps) {
            float mx = 0.0f;
            for (int j = lane; j < KP; j += 32) mx = fmaxf(mx, X[i * KP + j]);
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (mx > 0.0f) {
                if (!isfinite(mx)) bad = true;
                int r = float_exponent(mx);
                r = r < -126 ? -126 : (r > 126 ? 126 : r);
                float s = pow2f(-r);
                for (int j = lane; j < KP; j += 32) X[i * KP + j] *= s;
                if (lane == 0) ex[i] += mrow[i] + r;
            } else if (lane == 0) {
                ex[i] = ZERO_ROW_EXP64;
            }
        }
        __syncthreads();
    }
    for (int idx = tid; idx < KP * KP; idx += TREE_THREADS) Aout[(size_t)g.dst * KP * KP + idx] = X[idx];
    for (int k = tid; k < KP; k += TREE_THREADS) eout[(size_t)g.dst * KP + k] = ex[k];
    if (bad) atomicOr(status, ST_ENUMERIC);
}

cudaError_t launch_tree_level(int n_prop, int KP, int level, int n_groups, const TreeGroup *groups,
                              const LevelPtrs &lv, unsigned *status, cudaStream_t st) {
    if (n_groups == 0) return cudaSuccess;
    size_t smem = (size_t)2 * KP * KP * sizeof(float) + 3 * KP * sizeof(long long);
    dim3 grid(n_groups, n_prop);
    if (level == 0) {
        cudaFuncSetAttribute(tree_level_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tree_level_kernel<true><<<grid, TREE_THREADS, smem, st>>>(KP, level, groups, lv, status);
    } else {
        cudaFuncSetAttribute(tree_level_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tree_level_kernel<false><<<grid, TREE_THREADS, smem, st>>>(KP, level, groups, lv, status);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- final

constexpr int FINAL_THREADS = 128;

__device__ double block_sum_fixed(double v, double *red) {
    // deterministic: fixed pairing in shared memory
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = FINAL_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = FINAL_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(FINAL_THREADS)
final_kernel(int K, int KP, int init_mode, int n_seg, const SegFinal *__restrict__ segs,
             const float2 *__restrict__ head, LevelPtrs lv, const float *__restrict__ pi,
             const float *__restrict__ P, const float *__restrict__ p, const float *__restrict__ mu,
             const float *__restrict__ cov, const int *__restrict__ prop_bad,
             const int *__restrict__ obs_bad, double *__restrict__ out) {
    __shared__ double red[FINAL_THREADS];
    __shared__ double lpi0[80];   // log of the initial vector
    __shared__ double w[80];      // log h_i + ex_i ln 2
    const int q = blockIdx.x;
    const int tid = threadIdx.x;
    pi += (size_t)q * K;
    P += (size_t)q * K * K;
    p += (size_t)q * K;
    mu += (size_t)q * 2 * K;
    cov += (size_t)q * 3 * K;
    const double LN2 = 0.69314718055994530942;
    const double LOG_2PI = 1.8378770664093454836;

    for (int j = tid; j < K; j += FINAL_THREADS) {
        double v;
        if (init_mode == HMM_INIT_TRANSITION_FIRST) {
            v = 0.0;
            for (int i = 0; i < K; ++i) v += (double)pi[i] * (double)P[i * K + j];
        } else {
            v = pi[j];
        }
        lpi0[j] = log(v);
    }
    __syncthreads();
    double total = 0.0;
    for (int s = 0; s < n_seg; ++s) {
        const SegFinal sf = segs[s];
        double ll;
        if (sf.T == 0) {
            double a = 0.0;
            for (int k = tid; k < K; k += FINAL_THREADS) a += exp(lpi0[k]);
            ll = log(block_sum_fixed(a, red));
        } else {
            const float2 o = head[s];
            const bool tremor = !isnan(o.x);
            for (int k = tid; k < K; k += FINAL_THREADS) {
                double pk = p[k];
                double le;
                if (!tremor) {
                    le = log(1.0 - pk);
                } else {
                    double sxx = cov[3 * k], sxy = cov[3 * k + 1], syy = cov[3 * k + 2];
                    double det = sxx * syy - sxy * sxy;
                    double dx = (double)o.x - mu[2 * k], dy = (double)o.y - mu[2 * k + 1];
                    double qf = (syy * dx * dx - 2.0 * sxy * dx * dy + sxx * dy * dy) / det;
                    le = log(pk) - LOG_2PI - 0.5 * log(det) - 0.5 * qf;
                }
                double lh = lpi0[k] + le;
                if (sf.level >= 0) {
                    long long e;
                    if (sf.level == 0) {
                        int32_t e32 = reinterpret_cast<const int32_t *>(lv.e[0])[((size_t)q * lv.n[0] + sf.idx) * KP + k];
                        e = e32 == ZERO_ROW_EXP32 ? ZERO_ROW_EXP64 : (long long)e32;
                    } else
                        e = reinterpret_cast<const long long *>(lv.e[sf.level])[((size_t)q * lv.n[sf.level] + sf.idx) * KP + k];
                    lh += (double)e * LN2;
                }
                w[k] = lh;
            }
            __syncthreads();
            double mloc = -INFINITY;
            for (int k = tid; k < K; k += FINAL_THREADS) mloc = fmax(mloc, w[k]);
            const double M = block_max(mloc, red);
            double acc = 0.0;
            if (M > -INFINITY) {
                for (int k = tid; k < K; k += FINAL_THREADS) w[k] = exp(w[k] - M);
                __syncthreads();
                if (sf.level < 0) {
                    for (int k = tid; k < K; k += FINAL_THREADS) acc += w[k];
                } else {
                    const float *X = lv.A[sf.level] + ((size_t)q * lv.n[sf.level] + sf.idx) * KP * KP;
                    for (int j = tid; j < K; j += FINAL_THREADS) {
                        double v = 0.0;
                        for (int i = 0; i < K; ++i) v = fma(w[i], (double)X[i * KP + j], v);
                        acc += v;
                    }
                }
            }
            const double S = block_sum_fixed(acc, red);
            ll = (M > -INFINITY && S > 0.0) ? M + log(S) : -INFINITY;
        }
        total += ll;
        __syncthreads();
    }
    if (tid == 0) out[q] = (prop_bad[q] || *obs_bad) ? NAN : total;
}

cudaError_t launch_final(int n_prop, int K, int init_mode, int n_seg, const SegFinal *segs,
                         const float2 *head, const LevelPtrs &lv, int KP, const float *pi,
                         const float *P, const float *p, const float *mu, const float *cov,
                         const int *prop_bad, const int *obs_bad, double *out, cudaStream_t st) {
    final_kernel<<<n_prop, FINAL_THREADS, 0, st>>>(K, KP, init_mode, n_seg, segs, head, lv, pi, P, p,
                                                   mu, cov, prop_bad, obs_bad, out);
    return cudaGetLastError();
}

}  // namespace hmm
