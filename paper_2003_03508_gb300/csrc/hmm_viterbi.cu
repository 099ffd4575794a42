// The most probable hidden path (Viterbi) on the chunk structure.
//
// Viterbi is the likelihood's recursion with (max, +) in place of (+, x) on
// log probabilities, so the paper's restructuring carries over: every chunk
// forms its max-plus "product" V_c[i][j] -- the best log2 score of a path
// through the chunk entering in state i and leaving in state j -- all chunks
// in parallel; a scan over the chunks (FP64) finds the best entering score
// of every chunk and, by back-pointers over chunk boundaries, the states the
// best path takes at every boundary; then every chunk, in parallel, re-runs
// its recursion from its known entering state with per-step back-pointers
// and traces the path back from its known leaving state.
//
// Scores are kept relative: each step subtracts the step's best emission
// (common to all paths) and each row its maximum, with the offsets summed in
// FP64, so FP32 values stay near zero. Ties go to the smallest state index,
// as in the FP64 oracle; paths whose scores differ by rounding may differ.
#include "hmm_internal.cuh"

namespace hmm {

namespace {

constexpr int VT = 128;  // threads of the scan and path kernels

// ---- max-plus chunk products: one thread per row (entering state) ----
template <int KP, int CPC>
__global__ void __launch_bounds__(KP *CPC)
vit_chunk_kernel(int n_chunks, ConstLayout lay, const float *__restrict__ cblock,
                 const ChunkDesc *__restrict__ chunks, const float2 *__restrict__ packed, float *__restrict__ V,
                 double *__restrict__ voff) {
    __shared__ float sLP[KP * KP];
    __shared__ float sEm[EM_ROWS * KP];
    __shared__ float sL[CPC][KP];
    __shared__ float2 sObs[CPC][OBS_WIN];
    __shared__ int sMax;
    const int c = threadIdx.x / KP;
    const int i = threadIdx.x % KP;
    const int j_chunk = blockIdx.x * CPC + c;
    const bool live = j_chunk < n_chunks;
    for (int idx = threadIdx.x; idx < KP * KP; idx += blockDim.x) {
        const float pv = cblock[lay.off_p32 + idx];
        sLP[idx] = pv > 0.0f ? log2f(pv) : -INFINITY;
    }
    for (int idx = threadIdx.x; idx < EM_ROWS * KP; idx += blockDim.x) sEm[idx] = cblock[lay.off_emis + idx];
    int64_t pstart = 0;
    int len = 0;
    if (live) {
        const ChunkDesc d = chunks[j_chunk];
        pstart = d.pstart;
        len = d.len;
    }
    if (threadIdx.x == 0) sMax = 0;
    __syncthreads();
    if (i == 0 && live) atomicMax(&sMax, len);
    __syncthreads();
    const int steps = sMax;
    float row[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) row[j] = (j == i) ? 0.0f : -INFINITY;
    double off = 0.0;  // row offset plus the steps' common offsets
    for (int t = 0; t < steps; ++t) {
        const int w = t % OBS_WIN;
        if (w == 0) {
            __syncthreads();
            for (int u = i; u < OBS_WIN; u += KP)
                sObs[c][u] = (t + u < len) ? packed[pstart + t + u] : make_float2(__int_as_float(0x7fc00000), 0.f);
            __syncthreads();
        }
        const float2 o = sObs[c][w];
        sL[c][i] = log2_emission(sEm, KP, i, o.x, o.y, !isnan(o.x));
        __syncthreads();
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < KP; ++k) m = fmaxf(m, sL[c][k]);
        if (!(m > -INFINITY)) m = 0.0f;  // no state can emit: every score becomes -inf below
        float nw[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            float best = -INFINITY;
#pragma unroll
            for (int k = 0; k < KP; ++k) best = fmaxf(best, row[k] + sLP[k * KP + j]);
            nw[j] = best + (sL[c][j] - m);
        }
        __syncthreads();
        if (t < len) {
            float r = -INFINITY;
#pragma unroll
            for (int j = 0; j < KP; ++j) r = fmaxf(r, nw[j]);
            if (r > -INFINITY) {
#pragma unroll
                for (int j = 0; j < KP; ++j) row[j] = nw[j] - r;
                off += (double)r + (double)m;
            } else {
#pragma unroll
                for (int j = 0; j < KP; ++j) row[j] = -INFINITY;
                off = -INFINITY;
            }
        }
    }
    if (live) {
        float *dst = V + ((size_t)j_chunk * KP + i) * KP;
#pragma unroll
        for (int j = 0; j < KP; ++j) dst[j] = row[j];
        voff[(size_t)j_chunk * KP + i] = off;
    }
}

// ---- scan over chunk boundaries (one CTA) ----
__global__ void __launch_bounds__(VT) vit_scan_kernel(int K, int KP, int init_mode, int n_chunks,
                                                      const float *__restrict__ pi, const float *__restrict__ P,
                                                      const float *__restrict__ em, const float2 *__restrict__ head,
                                                      const float *__restrict__ V, const double *__restrict__ voff,
                                                      int32_t *__restrict__ ptr, int32_t *__restrict__ bstate,
                                                      double *__restrict__ score) {
    __shared__ double d[128];
    __shared__ double red[VT];
    __shared__ int ired[VT];
    const int j = threadIdx.x;
    // entering scores of chunk 0: log2 v0 + log2 e(o_0)
    double dj = -INFINITY;
    if (j < K) {
        double v = 0.0;
        if (init_mode == HMM_INIT_TRANSITION_FIRST) {
            for (int i = 0; i < K; ++i) v += (double)pi[i] * (double)P[i * K + j];
        } else {
            v = pi[j];
        }
        const float2 o = head[0];
        dj = v > 0.0 ? log2(v) + (double)log2_emission(em, KP, j, o.x, o.y, !isnan(o.x)) : -INFINITY;
    }
    double total = 0.0;
    for (int c = 0; c <= n_chunks; ++c) {
        // normalise by the maximum (kept in `total`)
        red[j] = dj;
        __syncthreads();
        for (int s = VT / 2; s > 0; s >>= 1) {
            if (j < s) red[j] = fmax(red[j], red[j + s]);
            __syncthreads();
        }
        const double mx = red[0];
        __syncthreads();
        if (mx == -INFINITY) {  // every path has probability zero
            if (j == 0) *score = -INFINITY;
            for (int t = j; t <= n_chunks; t += VT) bstate[t] = 0;
            return;
        }
        dj = dj - mx;
        total += mx;
        if (c == n_chunks) break;
        if (j < KP) d[j] = j < K ? dj : -INFINITY;
        __syncthreads();
        if (j < K) {
            double best = -INFINITY;
            int arg = 0;
            for (int i = 0; i < K; ++i) {
                const double v = d[i] + voff[(size_t)c * KP + i] + (double)V[((size_t)c * KP + i) * KP + j];
                if (v > best) {
                    best = v;
                    arg = i;
                }
            }
            dj = best;
            ptr[(size_t)c * KP + j] = arg;
        }
        __syncthreads();
    }
    // the best leaving state (smallest index on ties) and the boundary states
    ired[j] = (j < K && dj == 0.0) ? j : 1 << 30;
    __syncthreads();
    for (int s = VT / 2; s > 0; s >>= 1) {
        if (j < s) ired[j] = min(ired[j], ired[j + s]);
        __syncthreads();
    }
    if (j == 0) {
        int s = ired[0];
        bstate[n_chunks] = s;
        for (int c = n_chunks - 1; c >= 0; --c) {
            s = ptr[(size_t)c * KP + s];
            bstate[c] = s;
        }
        *score = total * 0.69314718055994530942;  // log2 -> natural log
    }
}

// ---- per-chunk paths (one CTA per chunk) ----
__global__ void __launch_bounds__(VT) vit_path_kernel(int K, int KP, int L, const ChunkDesc *__restrict__ chunks,
                                                      const float *__restrict__ cblock, ConstLayout lay,
                                                      const float2 *__restrict__ packed,
                                                      const int32_t *__restrict__ bstate, uint8_t *__restrict__ bp,
                                                      int32_t *__restrict__ path) {
    extern __shared__ float sLP[];  // K x K log2 P
    float *sd = sLP + K * K;        // K
    float *red = sd + K;            // VT
    const int c = blockIdx.x;
    const int j = threadIdx.x;
    const float *em = cblock + lay.off_emis;
    for (int idx = j; idx < K * K; idx += VT) {
        const float pv = cblock[lay.off_p32 + (idx / K) * KP + idx % K];
        sLP[idx] = pv > 0.0f ? log2f(pv) : -INFINITY;
    }
    const ChunkDesc cd = chunks[c];
    const int64_t t0 = (int64_t)c * L + 1;
    const int entry = bstate[c], leave = bstate[c + 1];
    float dj = (j == entry) ? 0.0f : -INFINITY;
    uint8_t *bpc = bp + (size_t)c * L * KP;
    for (int s = 0; s < cd.len; ++s) {
        const float2 o = packed[cd.pstart + s];
        const float l = j < K ? log2_emission(em, KP, j, o.x, o.y, !isnan(o.x)) : -INFINITY;
        if (j < K) sd[j] = dj;
        __syncthreads();
        float best = -INFINITY;
        int arg = 0;
        if (j < K)
            for (int i = 0; i < K; ++i) {
                const float v = sd[i] + sLP[i * K + j];
                if (v > best) {
                    best = v;
                    arg = i;
                }
            }
        if (j < K) bpc[(size_t)s * KP + j] = (uint8_t)arg;
        const float nv = best + l;
        red[j] = j < K ? nv : -INFINITY;
        __syncthreads();
        for (int h = VT / 2; h > 0; h >>= 1) {
            if (j < h) red[j] = fmaxf(red[j], red[j + h]);
            __syncthreads();
        }
        const float mx = red[0];
        __syncthreads();
        dj = (j < K && mx > -INFINITY) ? nv - mx : -INFINITY;
    }
    __syncthreads();
    if (j == 0) {
        int s_ = leave;
        for (int s = cd.len - 1; s >= 0; --s) {
            path[t0 + s] = s_;
            s_ = bpc[(size_t)s * KP + s_];
        }
        if (c == 0) path[0] = entry;
    }
}

template <int KP, int CPC>
cudaError_t launch_vit_chunk_t(int n_chunks, const ConstLayout &lay, const float *cblock, const ChunkDesc *chunks,
                               const float2 *packed, float *V, double *voff, cudaStream_t st) {
    const int blocks = (n_chunks + CPC - 1) / CPC;
    vit_chunk_kernel<KP, CPC><<<blocks, KP * CPC, 0, st>>>(n_chunks, lay, cblock, chunks, packed, V, voff);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_viterbi(int K, int init_mode, int n_chunks, int L, const ConstLayout &lay, const ChunkDesc *chunks,
                           const float *pi, const float *P, const float *cblock, const float2 *head,
                           const float2 *packed, float *V, double *voff, int32_t *ptr, int32_t *bstate, uint8_t *bp,
                           int32_t *path, double *score, cudaStream_t st) {
    const int KP = lay.KP;
    cudaError_t e = cudaSuccess;
    if (n_chunks > 0) {
        switch (KP) {
            case 4: e = launch_vit_chunk_t<4, 32>(n_chunks, lay, cblock, chunks, packed, V, voff, st); break;
            case 8: e = launch_vit_chunk_t<8, 16>(n_chunks, lay, cblock, chunks, packed, V, voff, st); break;
            case 16: e = launch_vit_chunk_t<16, 8>(n_chunks, lay, cblock, chunks, packed, V, voff, st); break;
            case 32: e = launch_vit_chunk_t<32, 4>(n_chunks, lay, cblock, chunks, packed, V, voff, st); break;
            case 48: e = launch_vit_chunk_t<48, 2>(n_chunks, lay, cblock, chunks, packed, V, voff, st); break;
            case 64: e = launch_vit_chunk_t<64, 2>(n_chunks, lay, cblock, chunks, packed, V, voff, st); break;
            case 80: e = launch_vit_chunk_t<80, 2>(n_chunks, lay, cblock, chunks, packed, V, voff, st); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    vit_scan_kernel<<<1, VT, 0, st>>>(K, KP, init_mode, n_chunks, pi, P, cblock + lay.off_emis, head, V, voff, ptr,
                                      bstate, score);
    if (n_chunks == 0) {
        // one observation: the path is the best entering state
        return cudaMemcpyAsync(path, bstate, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    }
    const size_t smem = sizeof(float) * ((size_t)K * K + K + VT);
    e = cudaFuncSetAttribute(vit_path_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    vit_path_kernel<<<n_chunks, VT, smem, st>>>(K, KP, L, chunks, cblock, lay, packed, bstate, bp, path);
    return cudaGetLastError();
}

}  // namespace hmm
