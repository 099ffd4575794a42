// Parameter preparation and observation packing.
//
// prep (one CTA per proposal): checks a parameter set and turns it into the
// constants the chunk kernels read -- the emission coefficients of Eq.
// "emission-matrix" in the log2 domain, P padded to KP x KP, and the
// tensor-core operand images of P.
//
// pack: copies the observations of every segment into an aligned buffer the
// chunk kernels read in 64-step windows (x = NaN marks "no tremor"), and
// checks that every flagged tremor has a finite location.
#include <cuda_bf16.h>
#include <math.h>

#include "hmm_internal.cuh"

namespace hmm {

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

ConstLayout make_layout(int K, int precision) {
    ConstLayout L{};
    int KP;
    if (precision == HMM_PREC_FP32_SIMT) {
        KP = K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : K <= 32 ? 32 : round_up(K, 16);
    } else {
        KP = round_up(K < 16 ? 16 : K, 16);
    }
    L.KP = KP;
    L.off_emis = 0;
    L.off_p32 = round_up(EM_ROWS * KP, 32);
    L.off_tc = round_up(L.off_p32 + KP * KP, 32);
    switch (precision) {
        case HMM_PREC_TF32: L.tc_floats = KP * KP; break;            // P_hi (tf32)
        case HMM_PREC_TF32_SPLIT: L.tc_floats = 2 * KP * KP; break;  // P_hi, P_lo (tf32)
        case HMM_PREC_BF16: L.tc_floats = KP * KP; break;            // P_hi, P_lo (bf16)
        default: L.tc_floats = 0;
    }
    L.stride = round_up(L.off_tc + L.tc_floats, 32);
    return L;
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Offset (in elements) of B-operand element (n, k) in the canonical K-major,
// no-swizzle layout: 8-row x 16-byte core matrices, adjacent along K at
// 128 bytes, 8-row groups at (KP * esize / 16) * 128 bytes.
__device__ __forceinline__ int kmajor_offset(int n, int k, int KP, int elems16) {
    int sbo_elems = (KP / elems16) * 8 * elems16;  // one 8-row group spans all of K
    return (n >> 3) * sbo_elems + (k / elems16) * (8 * elems16) + (n & 7) * elems16 + (k % elems16);
}

__global__ void prep_kernel(int K, ConstLayout lay, int precision, const float *__restrict__ pi,
                            const float *__restrict__ P, const float *__restrict__ p,
                            const float *__restrict__ mu, const float *__restrict__ cov,
                            float *__restrict__ cblock, int *__restrict__ prop_bad,
                            unsigned *__restrict__ status) {
    const int q = blockIdx.x;
    const int KP = lay.KP;
    pi += (size_t)q * K;
    P += (size_t)q * K * K;
    p += (size_t)q * K;
    mu += (size_t)q * 2 * K;
    cov += (size_t)q * 3 * K;
    float *cb = cblock + (size_t)q * lay.stride;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();

    // rows of P: non-negative, finite, summing to 1 within 1e-5
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        double s = 0.0;
        bool ok = true;
        for (int j = 0; j < K; ++j) {
            float v = P[i * K + j];
            ok = ok && isfinite(v) && v >= 0.0f;
            s += v;
        }
        if (!ok || fabs(s - 1.0) > 1e-5) bad = 1;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        bool ok = true;
        for (int k = 0; k < K; ++k) {
            ok = ok && isfinite(pi[k]) && pi[k] >= 0.0f;
            s += pi[k];
        }
        if (!ok || fabs(s - 1.0) > 1e-5) bad = 1;
    }
    // per-state emission constants (log2 domain), padded states emit nothing
    const double LOG2E = 1.4426950408889634074;
    const double LOG2_2PI = 2.6514961294723187980;
    for (int k = threadIdx.x; k < KP; k += blockDim.x) {
        float mx = 0.f, my = 0.f, qa = 0.f, qb = 0.f, qc = 0.f;
        float ctr = -INFINITY, cno = -INFINITY;
        if (k < K) {
            double pk = p[k];
            double sxx = cov[3 * k], sxy = cov[3 * k + 1], syy = cov[3 * k + 2];
            double det = sxx * syy - sxy * sxy;
            bool ok = isfinite(pk) && pk >= 0.0 && pk <= 1.0 && isfinite(sxx) && isfinite(sxy) &&
                      isfinite(syy) && sxx > 0.0 && syy > 0.0 && det > 0.0 &&
                      isfinite(mu[2 * k]) && isfinite(mu[2 * k + 1]);
            if (!ok) {
                bad = 1;
            } else {
                mx = mu[2 * k];
                my = mu[2 * k + 1];
                qa = (float)(-0.5 * LOG2E * syy / det);
                qb = (float)(LOG2E * sxy / det);
                qc = (float)(-0.5 * LOG2E * sxx / det);
                ctr = (float)(log2(pk) - LOG2_2PI - 0.5 * log2(det));
                cno = (float)log2(1.0 - pk);
            }
        }
        float *em = cb + lay.off_emis;
        em[EM_MUX * KP + k] = mx;
        em[EM_MUY * KP + k] = my;
        em[EM_QA * KP + k] = qa;
        em[EM_QB * KP + k] = qb;
        em[EM_QC * KP + k] = qc;
        em[EM_CTR * KP + k] = ctr;
        em[EM_CNO * KP + k] = cno;
        em[7 * KP + k] = 0.f;
    }
    // P padded to KP x KP (FP32, row-major) and the tensor-core images
    for (int idx = threadIdx.x; idx < KP * KP; idx += blockDim.x) {
        int i = idx / KP, j = idx % KP;
        float v = (i < K && j < K) ? P[i * K + j] : 0.0f;
        cb[lay.off_p32 + idx] = v;
        // B operand is P itself: B[k = i][n = j]
        if (precision == HMM_PREC_TF32 || precision == HMM_PREC_TF32_SPLIT) {
            float hi = to_tf32(v);
            cb[lay.off_tc + kmajor_offset(j, i, KP, 4)] = hi;
            if (precision == HMM_PREC_TF32_SPLIT)
                cb[lay.off_tc + KP * KP + kmajor_offset(j, i, KP, 4)] = to_tf32(v - hi);
        } else if (precision == HMM_PREC_BF16) {
            __nv_bfloat16 *img = reinterpret_cast<__nv_bfloat16 *>(cb + lay.off_tc);
            __nv_bfloat16 hi = __float2bfloat16_rn(v);
            __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            img[kmajor_offset(j, i, KP, 8)] = hi;
            img[KP * KP + kmajor_offset(j, i, KP, 8)] = lo;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        prop_bad[q] = bad;
        if (bad) atomicOr(status, ST_EINVAL);
    }
}

cudaError_t launch_prep(int n_prop, int K, const ConstLayout &lay, int precision, int init_mode,
                        const float *pi, const float *P, const float *p, const float *mu,
                        const float *cov, float *cblock, int *prop_bad, unsigned *status,
                        cudaStream_t st) {
    (void)init_mode;
    prep_kernel<<<n_prop, 128, 0, st>>>(K, lay, precision, pi, P, p, mu, cov, cblock, prop_bad,
                                        status);
    return cudaGetLastError();
}

// One thread per observation; the segment is found by binary search.
__global__ void pack_kernel(int n_seg, const int64_t *__restrict__ offs,
                            const int64_t *__restrict__ pbase, int64_t T_total,
                            const float2 *__restrict__ xy, const uint8_t *__restrict__ tremor,
                            float2 *__restrict__ packed, float2 *__restrict__ head,
                            int *__restrict__ obs_bad, unsigned *__restrict__ status) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T_total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_seg - 1;  // last s with offs[s] <= t
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= t) lo = mid; else hi = mid - 1;
        }
        // skip empty segments that share the offset
        int s = lo;
        float2 v = xy[t];
        bool tr = tremor[t] != 0;
        if (tr && !(isfinite(v.x) && isfinite(v.y))) {
            *obs_bad = 1;
            atomicOr(status, ST_EINVAL);
        }
        float2 o = tr ? v : make_float2(__int_as_float(0x7fc00000), 0.0f);
        int64_t u = t - offs[s];
        if (u == 0) head[s] = o;
        else packed[pbase[s] + u - 1] = o;
    }
}

cudaError_t launch_pack(int n_seg, const int64_t *d_offsets, const int64_t *d_pbase,
                        int64_t T_total, const float *xy, const uint8_t *tremor, float2 *packed,
                        float2 *head, int *obs_bad, unsigned *status, cudaStream_t st) {
    if (T_total == 0) return cudaSuccess;
    int64_t blocks = (T_total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    pack_kernel<<<(int)blocks, 256, 0, st>>>(n_seg, d_offsets, d_pbase, T_total,
                                             reinterpret_cast<const float2 *>(xy), tremor, packed,
                                             head, obs_bad, status);
    return cudaGetLastError();
}

}  // namespace hmm
