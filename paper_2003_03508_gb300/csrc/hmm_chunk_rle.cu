// Run-length shortcut for the chunk products (FP32 on the CUDA cores).
//
// A step without a tremor always has the same matrix, M_0 = P D_0 with
// D_0 = diag(1 - p_k) (Eq. "emission-matrix", no-tremor case), so a run of
// n such steps contributes M_0^n. Writing n in binary, M_0^n is the product
// of the powers M_0^(2^b) over the set bits b of n: popcount(n) matrix
// products instead of n. This is not part of the paper's algorithm; it
// changes the amount of arithmetic (not the result, up to rounding), so its
// throughput is reported apart from the roofline of the chunk kernels.
//
// Table (one CTA per proposal): Q_b = M_0^(2^b) for b = 0 .. nb-1 by
// repeated squaring, Q_{b+1} = Q_b Q_b. Every row is stored as floats whose
// largest entry lies in [1, 2) and an int32 power-of-two exponent of its own:
// when P is reducible, rows of M_0^n decay at rates that differ by far more
// than the float range, so one exponent per matrix would flush whole rows
// to zero.
//
// Chunk kernel (one CTA per chunk and proposal, one thread per row of the
// running product): walks the chunk's steps like the FP32 chunk kernel;
// at a step without a tremor it measures the run of no-tremor steps ahead
// (one warp-wide ballot per 32 steps) and, when the run has at least
// `min_run` steps, multiplies the running product by the table entries of
// the run length's set bits and jumps past the run. Shorter runs take the
// ordinary step and are not measured again.
#include "hmm_internal.cuh"

namespace hmm {
namespace {

// threads per CTA: one per row, rounded up to whole warps (every warp joins
// the ballots that measure a run)
template <int KP>
constexpr int rle_threads() {
    return (KP + 31) / 32 * 32;
}

// Divide a row by the power of two of its largest entry and add that power
// to its exponent. Returns false (and leaves the row alone) when the row has
// no positive entry.
template <int KP>
__device__ __forceinline__ bool renorm_row(float (&row)[KP], int &expo, bool &bad) {
    float mx = 0.0f;
#pragma unroll
    for (int j = 0; j < KP; ++j) mx = fmaxf(mx, row[j]);
    if (!(mx > 0.0f)) return false;
    if (!isfinite(mx)) bad = true;
    int r = float_exponent(mx);
    r = r < -126 ? -126 : (r > 126 ? 126 : r);
    const float s = pow2f(-r);
#pragma unroll
    for (int j = 0; j < KP; ++j) row[j] *= s;
    expo += r;
    return true;
}

// row <- row * (2^R Q), Q a KP x KP row-major float matrix (shared or
// global memory) whose row k carries the exponent R[k] (ZERO_ROW_EXP32: the
// row is zero). The terms
// row[k] 2^R[k] are aligned to the largest one before the product, so a
// term far below it (where it cannot change the float sum) flushes to zero
// instead of every term overflowing or underflowing together.
template <int KP>
__device__ __forceinline__ void mul_scaled(float (&row)[KP], int &expo, const float *__restrict__ Q,
                                           const int32_t *__restrict__ R) {
    int top = INT32_MIN;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int rk = R[k];
        if (row[k] > 0.0f && rk != ZERO_ROW_EXP32) top = max(top, rk + float_exponent(row[k]));
    }
    if (top == INT32_MIN) {  // nothing reaches a non-zero row: the product row is zero
#pragma unroll
        for (int j = 0; j < KP; ++j) row[j] = 0.0f;
        return;
    }
    float nw[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) nw[j] = 0.0f;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int rk = R[k];
        const float w = (row[k] > 0.0f && rk != ZERO_ROW_EXP32) ? ldexpf(row[k], rk - top) : 0.0f;
        const float4 *qk = reinterpret_cast<const float4 *>(Q + k * KP);
#pragma unroll
        for (int j4 = 0; j4 < KP / 4; ++j4) {
            const float4 v = qk[j4];
            nw[4 * j4 + 0] = fmaf(w, v.x, nw[4 * j4 + 0]);
            nw[4 * j4 + 1] = fmaf(w, v.y, nw[4 * j4 + 1]);
            nw[4 * j4 + 2] = fmaf(w, v.z, nw[4 * j4 + 2]);
            nw[4 * j4 + 3] = fmaf(w, v.w, nw[4 * j4 + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < KP; ++j) row[j] = nw[j];
    expo += top;
}

// Number of consecutive no-tremor steps at obs[0 ..], at most cap (cap >= 1).
// Every lane of the calling warp must take part; all lanes return the same
// value. At most cap / 32 + 1 iterations.
__device__ __forceinline__ int quiet_run(const float2 *__restrict__ obs, int cap) {
    const int lane = threadIdx.x & 31;
    int n = 0;
    for (;;) {
        const int u = n + lane;
        const bool stop = u >= cap || !isnan(obs[u].x);
        const unsigned m = __ballot_sync(0xffffffffu, stop);
        if (m) return n + __ffs(m) - 1;
        n += 32;
    }
}

template <int KP>
__global__ void __launch_bounds__(rle_threads<KP>())
rle_table_kernel(int nb, ConstLayout lay, const float *__restrict__ cblock, float *__restrict__ qtab,
                 int32_t *__restrict__ qexp, unsigned *__restrict__ status) {
    __shared__ __align__(16) float sQ[KP * KP];
    __shared__ int32_t sR[KP];
    const int q = blockIdx.x;
    const int i = threadIdx.x;
    const float *cb = cblock + (size_t)q * lay.stride;
    const float *cno = cb + lay.off_emis + EM_CNO * KP;
    float *Qt = qtab + (size_t)q * nb * KP * KP;
    int32_t *Qr = qexp + (size_t)q * nb * KP;

    // Q_0 = P D_0, with the step's prescale 2^-E as in an ordinary step
    float m = -INFINITY;
    for (int k = 0; k < KP; ++k) m = fmaxf(m, cno[k]);
    const bool repr = m >= -(float)EXP_LIMIT;
    const int E = repr ? (int)floorf(m) : 0;
    float row[KP];
    int expo = E;
    bool bad = false;
    bool live = false;  // the row has a positive entry
    if (i < KP) {
#pragma unroll
        for (int j = 0; j < KP; ++j)
            row[j] = repr ? cb[lay.off_p32 + i * KP + j] * exp2f(cno[j] - (float)E) : 0.0f;
        live = renorm_row<KP>(row, expo, bad);
    }
    for (int b = 0; b < nb; ++b) {
        if (b > 0) {
            // Q_b = Q_{b-1} Q_{b-1}: this thread's row times the matrix in shared memory
            if (i < KP && live) {
                mul_scaled<KP>(row, expo, sQ, sR);
                live = renorm_row<KP>(row, expo, bad);
            }
            __syncthreads();  // everyone has read Q_{b-1}
        }
        if (i < KP) {
            if (!live) {
#pragma unroll
                for (int j = 0; j < KP; ++j) row[j] = 0.0f;
                expo = ZERO_ROW_EXP32;
            }
#pragma unroll
            for (int j4 = 0; j4 < KP / 4; ++j4) {
                const float4 v = make_float4(row[4 * j4], row[4 * j4 + 1], row[4 * j4 + 2], row[4 * j4 + 3]);
                reinterpret_cast<float4 *>(sQ + i * KP)[j4] = v;
                reinterpret_cast<float4 *>(Qt + (size_t)b * KP * KP + i * KP)[j4] = v;
            }
            sR[i] = expo;
            Qr[(size_t)b * KP + i] = expo;
        }
        __syncthreads();  // Q_b is complete in shared memory
    }
    if (bad) atomicOr(status, ST_ENUMERIC);
}

template <int KP>
__global__ void __launch_bounds__(rle_threads<KP>())
chunk_rle_kernel(int n_chunks, int renorm, int min_run, int nb, ConstLayout lay,
                 const float *__restrict__ cblock, const float *__restrict__ qtab,
                 const int32_t *__restrict__ qexp, const ChunkDesc *__restrict__ chunks,
                 const float2 *__restrict__ packed, float *__restrict__ A0, int32_t *__restrict__ e0,
                 unsigned *__restrict__ status) {
    __shared__ __align__(16) float sP[KP * KP];
    __shared__ float sEm[EM_ROWS * KP];
    __shared__ float sL[KP];
    __shared__ __align__(16) float sD[KP];

    const int q = blockIdx.y;
    const int ch = blockIdx.x;
    const int i = threadIdx.x;
    const bool owner = i < KP;
    const float *cb = cblock + (size_t)q * lay.stride;
    for (int idx = i; idx < KP * KP; idx += blockDim.x) sP[idx] = cb[lay.off_p32 + idx];
    for (int idx = i; idx < EM_ROWS * KP; idx += blockDim.x) sEm[idx] = cb[lay.off_emis + idx];
    const ChunkDesc d = chunks[ch];
    const float2 *obs = packed + d.pstart;
    const int len = d.len;
    const float *Qt = qtab + (size_t)q * nb * KP * KP;
    const int32_t *Qr = qexp + (size_t)q * nb * KP;
    __syncthreads();

    float row[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) row[j] = (j == i) ? 1.0f : 0.0f;
    int expo = 0;
    bool bad = false;
    int since = 0;     // ordinary steps since the last renormalisation
    int measured = 0;  // steps before this index are known not to start a long run

    // every branch below depends only on values shared by the whole CTA
    for (int t = 0; t < len;) {
        const float2 o = obs[t];
        const bool tremor = !isnan(o.x);
        if (!tremor && min_run > 0 && t >= measured) {
            const int n = quiet_run(obs + t, len - t);
            if (n >= min_run) {
                if (owner) {
                    for (int b = 0; b < nb; ++b) {
                        if (!((n >> b) & 1)) continue;
                        mul_scaled<KP>(row, expo, Qt + (size_t)b * KP * KP, Qr + (size_t)b * KP);
                        if (!renorm_row<KP>(row, expo, bad)) break;  // the row is zero from here on
                    }
                }
                since = 0;
                t += n;
                measured = t;
                continue;
            }
            measured = t + n;
        }
        // an ordinary step: emissions, row * P, column scale by D_t
        if (owner) sL[i] = log2_emission(sEm, KP, i, o.x, o.y, tremor);
        float nw[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) nw[j] = 0.0f;
        if (owner) {
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const float rk = row[k];
                const float4 *pk = reinterpret_cast<const float4 *>(&sP[k * KP]);
#pragma unroll
                for (int j4 = 0; j4 < KP / 4; ++j4) {
                    const float4 pv = pk[j4];
                    nw[4 * j4 + 0] = fmaf(rk, pv.x, nw[4 * j4 + 0]);
                    nw[4 * j4 + 1] = fmaf(rk, pv.y, nw[4 * j4 + 1]);
                    nw[4 * j4 + 2] = fmaf(rk, pv.z, nw[4 * j4 + 2]);
                    nw[4 * j4 + 3] = fmaf(rk, pv.w, nw[4 * j4 + 3]);
                }
            }
        }
        __syncthreads();  // sL complete
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < KP; ++k) m = fmaxf(m, sL[k]);
        int E = 0;
        if (owner) {
            float d_i;
            if (m >= -(float)EXP_LIMIT) {
                E = (int)floorf(m);
                d_i = exp2f(sL[i] - (float)E);
            } else {
                if (m != -INFINITY) bad = true;  // finite but not representable
                d_i = 0.0f;                       // zero likelihood
            }
            sD[i] = d_i;
        }
        __syncthreads();  // sD complete
        if (owner) {
            const float4 *dv = reinterpret_cast<const float4 *>(sD);
#pragma unroll
            for (int j4 = 0; j4 < KP / 4; ++j4) {
                const float4 dd = dv[j4];
                row[4 * j4 + 0] = nw[4 * j4 + 0] * dd.x;
                row[4 * j4 + 1] = nw[4 * j4 + 1] * dd.y;
                row[4 * j4 + 2] = nw[4 * j4 + 2] * dd.z;
                row[4 * j4 + 3] = nw[4 * j4 + 3] * dd.w;
            }
            expo += E;
            if (++since == renorm) {
                renorm_row<KP>(row, expo, bad);
                since = 0;
            }
        }
        ++t;
    }
    if (owner) {
        if (since > 0) renorm_row<KP>(row, expo, bad);
        float mx = 0.0f;
#pragma unroll
        for (int j = 0; j < KP; ++j) mx = fmaxf(mx, row[j]);
        if (!(mx > 0.0f)) expo = ZERO_ROW_EXP32;
        float *dst = A0 + ((size_t)q * n_chunks + ch) * KP * KP + (size_t)i * KP;
#pragma unroll
        for (int j4 = 0; j4 < KP / 4; ++j4)
            reinterpret_cast<float4 *>(dst)[j4] =
                make_float4(row[4 * j4], row[4 * j4 + 1], row[4 * j4 + 2], row[4 * j4 + 3]);
        e0[((size_t)q * n_chunks + ch) * KP + i] = expo;
    }
    if (bad) atomicOr(status, ST_ENUMERIC);
}

}  // namespace

int rle_levels(int L) {
    int nb = 1;
    while ((1 << nb) <= L) ++nb;
    return nb;
}

#define HMM_RLE_CASES(X) X(4) X(8) X(16) X(32) X(48) X(64) X(80)

cudaError_t launch_rle_table(int n_prop, int nb, const ConstLayout &lay, const float *cblock, float *qtab,
                             int32_t *qexp, unsigned *status, cudaStream_t st) {
    if (n_prop == 0) return cudaSuccess;
    switch (lay.KP) {
#define HMM_RLE_T(KPV)                                                                                 \
    case KPV:                                                                                          \
        rle_table_kernel<KPV><<<n_prop, rle_threads<KPV>(), 0, st>>>(nb, lay, cblock, qtab, qexp, status); \
        return cudaGetLastError();
        HMM_RLE_CASES(HMM_RLE_T)
#undef HMM_RLE_T
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_chunk_rle(int n_prop, int n_chunks, int renorm, int min_run, int nb, const ConstLayout &lay,
                             const float *cblock, const float *qtab, const int32_t *qexp, const ChunkDesc *chunks,
                             const float2 *packed, float *A0, int32_t *e0, unsigned *status, cudaStream_t st) {
    if (n_chunks == 0 || n_prop == 0) return cudaSuccess;
    const dim3 grid(n_chunks, n_prop);
    switch (lay.KP) {
#define HMM_RLE_C(KPV)                                                                                \
    case KPV:                                                                                         \
        chunk_rle_kernel<KPV><<<grid, rle_threads<KPV>(), 0, st>>>(n_chunks, renorm, min_run, nb, lay, \
                                                                   cblock, qtab, qexp, chunks, packed, \
                                                                   A0, e0, status);                    \
        return cudaGetLastError();
        HMM_RLE_CASES(HMM_RLE_C)
#undef HMM_RLE_C
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hmm
