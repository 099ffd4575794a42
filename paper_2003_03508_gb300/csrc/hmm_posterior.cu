// Posterior state probabilities on the chunk structure (the forward-backward
// smoothing step that follows the likelihood).
//
// gamma_t(k) = P(s_t = k | all observations) = alpha_t(k) b_t(k) / L, with
// alpha_t the forward vector and b_t the backward vector. The likelihood
// path already holds every chunk's product A_c = prod_{t in c} P D_t (with
// per-row power-of-two exponents), so:
//   1. two scans over the chunk products give the forward vector entering
//      every chunk (f_c = h A_0 ... A_{c-1}, h = pi o e(o_0)) and the backward
//      vector leaving it (b_c = A_{c+1} ... A_{C-1} 1) -- K^2 work per chunk;
//   2. every chunk then, in parallel, recomputes its forward vectors from f_c
//      (storing them in the output), and runs the backward recursion from b_c,
//      turning each stored alpha_t into gamma_t = alpha_t o b_t / sum.
// Each vector is normalised every step; gamma needs no absolute scale.
#include "hmm_internal.cuh"

namespace hmm {

namespace {

constexpr int FB_THREADS = 128;

__device__ float block_reduce(float v, float *red, bool is_max) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmaxf(v, w) : v + w;
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float r = red[0];
    for (int w = 1; w < FB_THREADS / 32; ++w) r = is_max ? fmaxf(r, red[w]) : r + red[w];
    __syncthreads();
    return r;
}

__device__ int block_max_int(int v, int *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int r = red[0];
    for (int w = 1; w < FB_THREADS / 32; ++w) r = max(r, red[w]);
    __syncthreads();
    return r;
}

// the head vector h_j = v0_j e_j(o_0) for thread j < K, scaled by a power of
// two so that its largest entry lies in [1, 2) (zero if all are zero)
__device__ float head_vector(int K, int KP, int init_mode, const float *__restrict__ pi,
                             const float *__restrict__ P, const float *__restrict__ em, float2 o0, float *red) {
    const int j = threadIdx.x;
    float l = -INFINITY;
    if (j < K) {
        double v = 0.0;
        if (init_mode == HMM_INIT_TRANSITION_FIRST) {
            for (int i = 0; i < K; ++i) v += (double)pi[i] * (double)P[i * K + j];
        } else {
            v = pi[j];
        }
        l = v > 0.0 ? (float)log2(v) + log2_emission(em, KP, j, o0.x, o0.y, !isnan(o0.x)) : -INFINITY;
    }
    const float m = block_reduce(l, red, true);
    if (!(m > -INFINITY)) return 0.0f;
    return (j < K) ? exp2f(l - floorf(m)) : 0.0f;
}

// Block 0: forward boundary vectors fvec[c] (entering chunk c). Block 1:
// backward boundary vectors bvec[c] (leaving chunk c). The chunk products
// are staged in shared memory; their row exponents enter through ldexp so
// the sums stay in range.
__global__ void __launch_bounds__(FB_THREADS) fb_scan_kernel(int K, int KP, int init_mode, int n_chunks,
                                                             const float *__restrict__ pi, const float *__restrict__ P,
                                                             const float *__restrict__ em, const float2 *__restrict__ head,
                                                             const float *__restrict__ A0, const int32_t *__restrict__ e0,
                                                             float *fvec, float *bvec, float *gamma) {
    extern __shared__ float sA[];           // KP x KP
    float *vec = sA + KP * KP;              // KP
    float *red = vec + KP;                  // FB_THREADS / 32
    int *ired = reinterpret_cast<int *>(red + FB_THREADS / 32);
    const int j = threadIdx.x;
    if (blockIdx.x == 0) {
        float f = head_vector(K, KP, init_mode, pi, P, em, head[0], red);
        if (n_chunks == 0) {  // one observation: gamma_0 is the normalised head
            const float s = block_reduce(f, red, false);
            if (j < K) gamma[j] = f / s;
            return;
        }
        if (j < KP) fvec[j] = f;
        for (int c = 0; c + 1 < n_chunks; ++c) {
            const float *A = A0 + (size_t)c * KP * KP;
            for (int idx = j; idx < KP * KP; idx += FB_THREADS) sA[idx] = A[idx];
            const int ex = (j < K) ? e0[(size_t)c * KP + j] : ZERO_ROW_EXP32;
            const bool live = j < K && f > 0.0f && ex != ZERO_ROW_EXP32;
            const int em_ = block_max_int(live ? ex + ilogbf(f) : INT32_MIN, ired);
            if (j < KP) vec[j] = live ? ldexpf(f, ex - em_) : 0.0f;
            __syncthreads();
            float s = 0.0f;
            if (j < K)
                for (int i = 0; i < K; ++i) s = fmaf(vec[i], sA[i * KP + j], s);
            const float mx = block_reduce(s, red, true);
            f = mx > 0.0f ? s / mx : 0.0f;
            if (j < KP) fvec[(size_t)(c + 1) * KP + j] = f;
        }
    } else {
        if (n_chunks == 0) return;
        float b = j < K ? 1.0f : 0.0f;
        if (j < KP) bvec[(size_t)(n_chunks - 1) * KP + j] = b;
        for (int c = n_chunks - 1; c >= 1; --c) {
            const float *A = A0 + (size_t)c * KP * KP;
            for (int idx = j; idx < KP * KP; idx += FB_THREADS) sA[idx] = A[idx];
            if (j < KP) vec[j] = b;
            __syncthreads();
            float w = 0.0f;
            if (j < K)
                for (int k = 0; k < K; ++k) w = fmaf(sA[j * KP + k], vec[k], w);
            const int ex = (j < K) ? e0[(size_t)c * KP + j] : ZERO_ROW_EXP32;
            const bool live = j < K && w > 0.0f && ex != ZERO_ROW_EXP32;
            const int em_ = block_max_int(live ? ex + ilogbf(w) : INT32_MIN, ired);
            float v = live ? ldexpf(w, ex - em_) : 0.0f;
            const float mx = block_reduce(v, red, true);
            b = mx > 0.0f ? v / mx : 0.0f;
            if (j < KP) bvec[(size_t)(c - 1) * KP + j] = b;
        }
    }
}

// One CTA per chunk: forward vectors from fvec[c] (stored in gamma), then the
// backward recursion from bvec[c] turning them into posterior probabilities;
// chunk 0 also writes gamma_0 from the head vector.
__global__ void __launch_bounds__(FB_THREADS) fb_chunk_kernel(int K, int KP, int init_mode, int L,
                                                              const ChunkDesc *__restrict__ chunks,
                                                              const float *__restrict__ pi, const float *__restrict__ P,
                                                              const float *__restrict__ em,
                                                              const float2 *__restrict__ head,
                                                              const float2 *__restrict__ packed,
                                                              const float *__restrict__ fvec,
                                                              const float *__restrict__ bvec, float *gamma) {
    extern __shared__ float sP[];            // K x K (row-major), then its transpose
    float *sPT = sP + K * K;
    float *vec = sPT + K * K;                // K
    float *red = vec + KP;                   // FB_THREADS / 32
    const int c = blockIdx.x;
    const int j = threadIdx.x;
    for (int idx = j; idx < K * K; idx += FB_THREADS) {
        const float v = P[idx];
        sP[idx] = v;
        sPT[(idx % K) * K + idx / K] = v;
    }
    const ChunkDesc cd = chunks[c];
    const int64_t t0 = (int64_t)c * L + 1;  // observation index of the chunk's first step (one segment)
    float a = j < K ? fvec[(size_t)c * KP + j] : 0.0f;
    // forward: alpha_t = normalise((alpha_{t-1} P) o d_t)
    for (int s = 0; s < cd.len; ++s) {
        const float2 o = packed[cd.pstart + s];
        const float l = j < K ? log2_emission(em, KP, j, o.x, o.y, !isnan(o.x)) : -INFINITY;
        const float m = block_reduce(l, red, true);
        if (j < KP) vec[j] = a;
        __syncthreads();
        float v = 0.0f;
        if (j < K && m > -INFINITY) {
            for (int i = 0; i < K; ++i) v = fmaf(vec[i], sP[i * K + j], v);
            v *= exp2f(l - m);
        }
        const float mx = block_reduce(v, red, true);
        a = mx > 0.0f ? v / mx : 0.0f;
        if (j < K) gamma[(size_t)(t0 + s) * K + j] = a;
    }
    // backward: gamma_t = normalise(alpha_t o b_t); b_{t-1} = P (d_t o b_t)
    float b = j < K ? bvec[(size_t)c * KP + j] : 0.0f;
    for (int s = cd.len - 1; s >= 0; --s) {
        const int64_t t = t0 + s;
        const float g = j < K ? gamma[(size_t)t * K + j] * b : 0.0f;
        const float sum = block_reduce(g, red, false);
        if (j < K) gamma[(size_t)t * K + j] = sum > 0.0f ? g / sum : __int_as_float(0x7fc00000);
        const float2 o = packed[cd.pstart + s];
        const float l = j < K ? log2_emission(em, KP, j, o.x, o.y, !isnan(o.x)) : -INFINITY;
        const float m = block_reduce(l, red, true);
        if (j < KP) vec[j] = (j < K && m > -INFINITY) ? exp2f(l - m) * b : 0.0f;
        __syncthreads();
        float w = 0.0f;
        if (j < K)
            for (int k = 0; k < K; ++k) w = fmaf(sPT[k * K + j], vec[k], w);
        const float mx = block_reduce(w, red, true);
        b = mx > 0.0f ? w / mx : 0.0f;
    }
    if (c == 0) {
        const float h = head_vector(K, KP, init_mode, pi, P, em, head[0], red);
        const float g = j < K ? h * b : 0.0f;
        const float sum = block_reduce(g, red, false);
        if (j < K) gamma[j] = sum > 0.0f ? g / sum : __int_as_float(0x7fc00000);
    }
}

}  // namespace

cudaError_t launch_posterior(int K, int KP, int init_mode, int n_chunks, int L, const ChunkDesc *chunks,
                             const float *pi, const float *P, const float *em, const float2 *head,
                             const float2 *packed, const float *A0, const int32_t *e0, float *fvec, float *bvec,
                             float *gamma, cudaStream_t st) {
    const size_t scan_smem = sizeof(float) * ((size_t)KP * KP + KP + FB_THREADS / 32) + sizeof(int) * FB_THREADS / 32;
    const size_t chunk_smem = sizeof(float) * (2 * (size_t)K * K + KP + FB_THREADS / 32);
    cudaError_t e = cudaFuncSetAttribute(fb_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scan_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fb_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chunk_smem);
    if (e != cudaSuccess) return e;
    fb_scan_kernel<<<2, FB_THREADS, scan_smem, st>>>(K, KP, init_mode, n_chunks, pi, P, em, head, A0, e0, fvec,
                                                      bvec, gamma);
    if (n_chunks > 0)
        fb_chunk_kernel<<<n_chunks, FB_THREADS, chunk_smem, st>>>(K, KP, init_mode, L, chunks, pi, P, em, head,
                                                                   packed, fvec, bvec, gamma);
    return cudaGetLastError();
}

}  // namespace hmm
