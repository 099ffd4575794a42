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
//
// With a statistics buffer, the backward pass also accumulates the E-step
// statistics of the chunk (Baum-Welch): the pairwise posteriors
// xi_t(i, j) ∝ alpha_{t-1}(i) P_ij e_j(o_t) b_t(j) summed into expected
// transition counts, and the gamma-weighted tremor counts and location
// moments; a second kernel adds the chunks' partial sums in chunk order in
// FP64, so the result does not depend on scheduling.
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

// per-chunk partial statistics: N (K x K), then Gs, Gr, Sx, Sy, Sxx, Sxy, Syy (K each)
constexpr int N_MOM = 7;

__device__ void add_gamma_moments(double *acc, float g, float2 o) {
    acc[0] += g;
    if (!isnan(o.x)) {
        const double x = o.x, y = o.y;
        acc[1] += g;
        acc[2] += g * x;
        acc[3] += g * y;
        acc[4] += g * x * x;
        acc[5] += g * x * y;
        acc[6] += g * y * y;
    }
}

// One CTA per chunk: forward vectors from fvec[c] (stored in gamma), then the
// backward recursion from bvec[c] turning them into posterior probabilities
// (and, with stats_part, the chunk's E-step statistics); chunk 0 also writes
// gamma_0 from the head vector.
__global__ void __launch_bounds__(FB_THREADS) fb_chunk_kernel(int K, int KP, int init_mode, int L,
                                                              const ChunkDesc *__restrict__ chunks,
                                                              const float *__restrict__ pi, const float *__restrict__ P,
                                                              const float *__restrict__ em,
                                                              const float2 *__restrict__ head,
                                                              const float2 *__restrict__ packed,
                                                              const float *__restrict__ fvec,
                                                              const float *__restrict__ bvec, float *gamma,
                                                              double *stats_part, double *g0) {
    extern __shared__ double sN[];           // K x K expected transitions (with statistics, FP64)
    float *sP = reinterpret_cast<float *>(sN + (stats_part ? K * K : 0));  // K x K (row-major)
    float *sPT = sP + K * K;                 // its transpose
    float *vec = sPT + K * K;                // KP
    float *aprev = vec + KP;                 // KP
    float *red = aprev + KP;                 // FB_THREADS / 32
    const int c = blockIdx.x;
    const int j = threadIdx.x;
    for (int idx = j; idx < K * K; idx += FB_THREADS) {
        const float v = P[idx];
        sP[idx] = v;
        sPT[(idx % K) * K + idx / K] = v;
        if (stats_part) sN[idx] = 0.0;
    }
    double mom[N_MOM] = {0, 0, 0, 0, 0, 0, 0};
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
        const float gn = sum > 0.0f ? g / sum : __int_as_float(0x7fc00000);
        if (j < K) gamma[(size_t)t * K + j] = gn;
        const float2 o = packed[cd.pstart + s];
        if (stats_part && j < K) add_gamma_moments(mom, gn, o);
        const float l = j < K ? log2_emission(em, KP, j, o.x, o.y, !isnan(o.x)) : -INFINITY;
        const float m = block_reduce(l, red, true);
        if (j < KP) vec[j] = (j < K && m > -INFINITY) ? exp2f(l - m) * b : 0.0f;
        if (stats_part && j < KP)
            aprev[j] = j < K ? (s > 0 ? gamma[(size_t)(t - 1) * K + j] : fvec[(size_t)c * KP + j]) : 0.0f;
        __syncthreads();
        if (stats_part) {
            // xi_t(i, j) = aprev_i P_ij vec_j / Z, Z = sum_j (aprev P)_j vec_j
            float colj = 0.0f;
            if (j < K)
                for (int i = 0; i < K; ++i) colj = fmaf(aprev[i], sP[i * K + j], colj);
            const float Z = block_reduce(j < K ? colj * vec[j] : 0.0f, red, false);
            if (j < K && Z > 0.0f) {
                const float u = vec[j] / Z;
                for (int i = 0; i < K; ++i) sN[i * K + j] += (double)(aprev[i] * sP[i * K + j] * u);
            }
        }
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
        const float gn = sum > 0.0f ? g / sum : __int_as_float(0x7fc00000);
        if (j < K) gamma[j] = gn;
        if (stats_part && j < K) {
            add_gamma_moments(mom, gn, head[0]);
            g0[j] = gn;
        }
    }
    if (stats_part) {
        __syncthreads();
        double *dst = stats_part + (size_t)c * (K * K + N_MOM * K);
        for (int idx = j; idx < K * K; idx += FB_THREADS) dst[idx] = sN[idx];
        if (j < K)
            for (int r = 0; r < N_MOM; ++r) dst[K * K + r * K + j] = mom[r];
    }
}

// stats = [N (K x K), G0, Gs, Gr, Sx, Sy, Sxx, Sxy, Syy]: the chunks'
// partial sums added in chunk order (one thread per entry)
__global__ void fb_stats_reduce_kernel(int K, int n_chunks, const double *__restrict__ part,
                                       const double *__restrict__ g0, double *stats) {
    const int n = K * K + N_MOM * K;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < n_chunks; ++c) acc += part[(size_t)c * n + e];
        // G0 sits between N and the moments
        stats[e < K * K ? e : e + K] = acc;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) stats[K * K + k] = g0[k];
}

}  // namespace

cudaError_t launch_posterior(int K, int KP, int init_mode, int n_chunks, int L, const ChunkDesc *chunks,
                             const float *pi, const float *P, const float *em, const float2 *head,
                             const float2 *packed, const float *A0, const int32_t *e0, float *fvec, float *bvec,
                             float *gamma, double *stats_part, double *g0, double *stats, cudaStream_t st) {
    const size_t scan_smem = sizeof(float) * ((size_t)KP * KP + KP + FB_THREADS / 32) + sizeof(int) * FB_THREADS / 32;
    const size_t chunk_smem = (stats_part ? sizeof(double) * (size_t)K * K : 0) +
                              sizeof(float) * (2 * (size_t)K * K + 2 * KP + FB_THREADS / 32);
    cudaError_t e = cudaFuncSetAttribute(fb_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scan_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fb_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chunk_smem);
    if (e != cudaSuccess) return e;
    fb_scan_kernel<<<2, FB_THREADS, scan_smem, st>>>(K, KP, init_mode, n_chunks, pi, P, em, head, A0, e0, fvec,
                                                      bvec, gamma);
    if (n_chunks > 0)
        fb_chunk_kernel<<<n_chunks, FB_THREADS, chunk_smem, st>>>(K, KP, init_mode, L, chunks, pi, P, em, head,
                                                                   packed, fvec, bvec, gamma, stats_part, g0);
    if (stats && n_chunks > 0)
        fb_stats_reduce_kernel<<<(K * K + N_MOM * K + 255) / 256, 256, 0, st>>>(K, n_chunks, stats_part, g0, stats);
    return cudaGetLastError();
}

}  // namespace hmm
