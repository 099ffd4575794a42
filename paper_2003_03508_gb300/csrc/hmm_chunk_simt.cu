// Chunk products on the CUDA cores in FP32 (the "plain GPU" path).
//
// Section "The likelihood algorithm", steps 1-3: the chain of matrices
// M_t = P D_t is cut into chunks and every chunk's product
//     A_c = prod_{t in c} P D_t
// is formed independently. Step 1 (the emissions) and step 2 (P D_t) are
// fused into the product loop: each step multiplies the running product by P
// and then scales column j by D_t[j], so neither D_t nor P D_t is ever
// written to memory.
//
// Scale coefficients (Section "Step 3", last paragraph): the emissions of a
// step are pre-scaled by 2^-E_t so that the best state's factor lies in
// [1, 2), and every `renorm` steps each row of the running product is
// divided by the power of two of its largest entry. Both are exact in binary
// floating point; the exponents are returned per row as int32.
//
// Thread mapping: one thread owns one row of one chunk's running product
// (KP registers) and reads P from shared memory by broadcast. A CTA holds CPC
// chunks of one proposal.
#include "hmm_internal.cuh"

namespace hmm {

template <int KP>
__device__ __forceinline__ void chunk_sync() {
    if constexpr (KP <= 32) __syncwarp(); else __syncthreads();
}

template <int KP, int CPC>
__global__ void __launch_bounds__(KP *CPC)
chunk_simt_kernel(int n_chunks, int L, int renorm, ConstLayout lay, const float *__restrict__ cblock,
                  const ChunkDesc *__restrict__ chunks, const float2 *__restrict__ packed,
                  float *__restrict__ A0, int32_t *__restrict__ e0, unsigned *__restrict__ status) {
    __shared__ __align__(16) float sP[KP * KP];
    __shared__ float sEm[EM_ROWS * KP];
    __shared__ float sL[CPC][KP];
    __shared__ __align__(16) float sD[CPC][KP];
    __shared__ float2 sObs[CPC][OBS_WIN];

    const int q = blockIdx.y;
    const int c = threadIdx.x / KP;  // chunk slot in this CTA
    const int i = threadIdx.x % KP;  // row of the chunk product (= start state)
    const int j_chunk = blockIdx.x * CPC + c;
    const bool live = j_chunk < n_chunks;
    const float *cb = cblock + (size_t)q * lay.stride;

    for (int idx = threadIdx.x; idx < KP * KP; idx += blockDim.x) sP[idx] = cb[lay.off_p32 + idx];
    for (int idx = threadIdx.x; idx < EM_ROWS * KP; idx += blockDim.x) sEm[idx] = cb[lay.off_emis + idx];

    int64_t pstart = 0;
    int len = 0;
    if (live) {
        ChunkDesc d = chunks[j_chunk];
        pstart = d.pstart;
        len = d.len;
    }
    // the CTA loops over the longest chunk it holds
    __shared__ int sMax;
    if (threadIdx.x == 0) sMax = 0;
    __syncthreads();
    if (i == 0 && live) atomicMax(&sMax, len);
    __syncthreads();
    const int steps = sMax;

    float row[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) row[j] = (j == i) ? 1.0f : 0.0f;
    int expo = 0;       // power-of-two exponent of this row
    bool bad = false;

    for (int t = 0; t < steps; ++t) {
        const int w = t % OBS_WIN;
        if (w == 0) {
            __syncthreads();
            for (int u = i; u < OBS_WIN; u += KP) {
                int64_t g = pstart + t + u;
                sObs[c][u] = (t + u < len) ? packed[g] : make_float2(__int_as_float(0x7fc00000), 0.f);
            }
            __syncthreads();
        }
        const float2 o = sObs[c][w];
        const bool tremor = !isnan(o.x);
        // Step 1: this thread's state emission (log2 domain)
        sL[c][i] = log2_emission(sEm, KP, i, o.x, o.y, tremor);

        // Step 3 (first half): new = row * P
        float nw[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) nw[j] = 0.0f;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const float rk = row[k];
            const float4 *pk = reinterpret_cast<const float4 *>(&sP[k * KP]);
#pragma unroll
            for (int j4 = 0; j4 < KP / 4; ++j4) {
                float4 pv = pk[j4];
                nw[4 * j4 + 0] = fmaf(rk, pv.x, nw[4 * j4 + 0]);
                nw[4 * j4 + 1] = fmaf(rk, pv.y, nw[4 * j4 + 1]);
                nw[4 * j4 + 2] = fmaf(rk, pv.z, nw[4 * j4 + 2]);
                nw[4 * j4 + 3] = fmaf(rk, pv.w, nw[4 * j4 + 3]);
            }
        }
        chunk_sync<KP>();
        // best state of the step; prescale exponent E_t; D_t[i] = 2^(l_i - E_t)
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < KP; ++k) m = fmaxf(m, sL[c][k]);
        int E = 0;
        float d_i;
        if (m >= -(float)EXP_LIMIT) {
            E = (int)floorf(m);
            d_i = exp2f(sL[c][i] - (float)E);
        } else {
            if (m != -INFINITY && t < len) bad = true;  // finite but not representable
            d_i = 0.0f;                                  // zero likelihood
        }
        sD[c][i] = d_i;
        chunk_sync<KP>();
        if (t < len) {
            // Step 2 fused: column scale by D_t
            const float4 *dv = reinterpret_cast<const float4 *>(&sD[c][0]);
#pragma unroll
            for (int j4 = 0; j4 < KP / 4; ++j4) {
                float4 d = dv[j4];
                row[4 * j4 + 0] = nw[4 * j4 + 0] * d.x;
                row[4 * j4 + 1] = nw[4 * j4 + 1] * d.y;
                row[4 * j4 + 2] = nw[4 * j4 + 2] * d.z;
                row[4 * j4 + 3] = nw[4 * j4 + 3] * d.w;
            }
            expo += E;
            if ((t + 1) % renorm == 0 || t + 1 == len) {
                float mx = 0.0f;
#pragma unroll
                for (int j = 0; j < KP; ++j) mx = fmaxf(mx, row[j]);
                if (mx > 0.0f) {
                    if (!isfinite(mx)) bad = true;
                    int r = float_exponent(mx);
                    r = r < -126 ? -126 : (r > 126 ? 126 : r);
                    float s = pow2f(-r);
#pragma unroll
                    for (int j = 0; j < KP; ++j) row[j] *= s;
                    expo += r;
                }
            }
        }
    }
    if (bad) atomicOr(status, ST_ENUMERIC);
    if (live) {
        float mx = 0.0f;
#pragma unroll
        for (int j = 0; j < KP; ++j) mx = fmaxf(mx, row[j]);
        if (!(mx > 0.0f)) expo = ZERO_ROW_EXP32;
        float *dst = A0 + ((size_t)q * n_chunks + j_chunk) * KP * KP + (size_t)i * KP;
#pragma unroll
        for (int j4 = 0; j4 < KP / 4; ++j4)
            reinterpret_cast<float4 *>(dst)[j4] =
                make_float4(row[4 * j4], row[4 * j4 + 1], row[4 * j4 + 2], row[4 * j4 + 3]);
        e0[((size_t)q * n_chunks + j_chunk) * KP + i] = expo;
    }
}

template <int KP, int CPC>
static cudaError_t launch_simt_t(int n_prop, int n_chunks, int L, int renorm, const ConstLayout &lay,
                                 const float *cblock, const ChunkDesc *chunks, const float2 *packed,
                                 float *A0, int32_t *e0, unsigned *status, cudaStream_t st) {
    dim3 grid((n_chunks + CPC - 1) / CPC, n_prop);
    chunk_simt_kernel<KP, CPC><<<grid, KP * CPC, 0, st>>>(n_chunks, L, renorm, lay, cblock, chunks,
                                                          packed, A0, e0, status);
    return cudaGetLastError();
}

cudaError_t launch_chunk_simt(int n_prop, int n_chunks, int L, int renorm, const ConstLayout &lay,
                              const float *cblock, const ChunkDesc *chunks, const float2 *packed,
                              float *A0, int32_t *e0, unsigned *status, cudaStream_t st) {
    if (n_chunks == 0 || n_prop == 0) return cudaSuccess;
#define HMM_SIMT_CASE(KPV, CPCV)                                                                 \
    case KPV:                                                                                    \
        return launch_simt_t<KPV, CPCV>(n_prop, n_chunks, L, renorm, lay, cblock, chunks, packed, \
                                        A0, e0, status, st);
    switch (lay.KP) {
        HMM_SIMT_CASE(4, 32)
        HMM_SIMT_CASE(8, 16)
        HMM_SIMT_CASE(16, 8)
        HMM_SIMT_CASE(32, 4)
        HMM_SIMT_CASE(48, 2)
        HMM_SIMT_CASE(64, 2)
        HMM_SIMT_CASE(80, 2)
        default: return cudaErrorInvalidValue;
    }
#undef HMM_SIMT_CASE
}

}  // namespace hmm
