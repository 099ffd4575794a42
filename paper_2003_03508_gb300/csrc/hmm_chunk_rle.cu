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
// Chunk kernels (one thread per row of a chunk's running product): walk the
// chunk's steps like the FP32 chunk kernel; at a step without a tremor they
// measure the run of no-tremor steps ahead and, when it has at least
// `min_run` steps, multiply the running product by the table entries of the
// run length's set bits and jump past the run. Shorter runs take the
// ordinary step and are not measured again.
//   KP <= 32: one warp per chunk, WPC chunks of one proposal per CTA sharing
//     P and the whole table in shared memory; the state's emission constants
//     live in its lane's registers, the step's best emission is a warp
//     reduction, and the observations come in 32-step windows held one per
//     lane, whose ballot mask gives run lengths without further loads.
//   KP > 32: one CTA per chunk (several warps per row set), table read
//     through L1/L2, one warp ballot per 32 steps of a run.
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
// global memory, 16-byte aligned, as is R) whose row k carries the exponent
// R[k] (ZERO_ROW_EXP32: the row is zero). The terms
// row[k] 2^R[k] are aligned to the largest one before the product, so a
// term far below it (where it cannot change the float sum) flushes to zero
// instead of every term overflowing or underflowing together.
template <int KP>
__device__ __forceinline__ void mul_scaled(float (&row)[KP], int &expo, const float *__restrict__ Q,
                                           const int32_t *__restrict__ R) {
    int top = INT32_MIN;
#pragma unroll
    for (int k4 = 0; k4 < KP / 4; ++k4) {
        const int4 v = reinterpret_cast<const int4 *>(R)[k4];
        const int rv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = 4 * k4 + u;
            if (row[k] > 0.0f && rv[u] != ZERO_ROW_EXP32) top = max(top, rv[u] + float_exponent(row[k]));
        }
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
        // w = row[k] 2^(R[k] - top) <= 2, as two exact power-of-two factors
        // (each within the normal exponent range); below 2^-252 it is zero
        float w = 0.0f;
        const int rk = R[k];  // reloaded (a broadcast load) rather than held in registers
        if (row[k] > 0.0f && rk != ZERO_ROW_EXP32) {
            const int d = rk - top;
            const int d1 = d < -126 ? -126 : d;
            const int d2 = d - d1 < -126 ? -126 : d - d1;
            w = row[k] * pow2f(d1) * pow2f(d2);
        }
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

// The first half of mul_scaled on its own: row[k] <- row[k] 2^(R[k] - top)
// in place; returns top, or INT32_MIN after zeroing a row that reaches no
// non-zero row of Q. R is 16-byte aligned.
template <int KP>
__device__ __forceinline__ int prescale_row(float (&row)[KP], const int32_t *__restrict__ R) {
    int top = INT32_MIN;
#pragma unroll
    for (int k4 = 0; k4 < KP / 4; ++k4) {
        const int4 v = reinterpret_cast<const int4 *>(R)[k4];
        const int rv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = 4 * k4 + u;
            if (row[k] > 0.0f && rv[u] != ZERO_ROW_EXP32) top = max(top, rv[u] + float_exponent(row[k]));
        }
    }
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        float w = 0.0f;
        const int rk = R[k];
        if (top != INT32_MIN && row[k] > 0.0f && rk != ZERO_ROW_EXP32) {
            const int d = rk - top;
            const int d1 = d < -126 ? -126 : d;
            const int d2 = d - d1 < -126 ? -126 : d - d1;
            w = row[k] * pow2f(d1) * pow2f(d2);
        }
        row[k] = w;
    }
    return top;
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
    __shared__ __align__(16) int32_t sR[KP];
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

constexpr int RLE_WPC = 8;  // chunks (warps) per CTA of the warp kernel

template <int KP>
__global__ void __launch_bounds__(32 * RLE_WPC, 2)
chunk_rle_warp_kernel(int n_chunks, int renorm, int min_run, int nb, ConstLayout lay,
                      const float *__restrict__ cblock, const float *__restrict__ qtab,
                      const int32_t *__restrict__ qexp, const ChunkDesc *__restrict__ chunks,
                      const float2 *__restrict__ packed, float *__restrict__ A0, int32_t *__restrict__ e0,
                      unsigned *__restrict__ status) {
    static_assert(KP <= 32, "one lane per row");
    extern __shared__ __align__(16) float smem[];
    float *sP = smem;                                   // KP x KP
    float *sQ = sP + KP * KP;                           // nb x KP x KP
    int32_t *sR = reinterpret_cast<int32_t *>(sQ + (size_t)nb * KP * KP);  // nb x KP
    float *sD = reinterpret_cast<float *>(sR + (size_t)nb * KP);           // RLE_WPC x KP

    const int q = blockIdx.y;
    const int warp = threadIdx.x >> 5;
    const int i = threadIdx.x & 31;  // row of the running product = lane
    const int ch = blockIdx.x * RLE_WPC + warp;
    const float *cb = cblock + (size_t)q * lay.stride;
    {
        const float4 *src = reinterpret_cast<const float4 *>(cb + lay.off_p32);
        for (int idx = threadIdx.x; idx < KP * KP / 4; idx += blockDim.x)
            reinterpret_cast<float4 *>(sP)[idx] = src[idx];
        const float4 *qsrc = reinterpret_cast<const float4 *>(qtab + (size_t)q * nb * KP * KP);
        for (int idx = threadIdx.x; idx < nb * KP * KP / 4; idx += blockDim.x)
            reinterpret_cast<float4 *>(sQ)[idx] = qsrc[idx];
        const int32_t *rsrc = qexp + (size_t)q * nb * KP;
        for (int idx = threadIdx.x; idx < nb * KP; idx += blockDim.x) sR[idx] = rsrc[idx];
    }
    __syncthreads();  // the only CTA-wide barrier
    if (ch >= n_chunks) return;

    // this lane's state's emission constants (lanes past KP never win the max)
    const float *em = cb + lay.off_emis;
    const bool owner = i < KP;
    const float mux = owner ? em[EM_MUX * KP + i] : 0.f, muy = owner ? em[EM_MUY * KP + i] : 0.f;
    const float qa = owner ? em[EM_QA * KP + i] : 0.f, qb = owner ? em[EM_QB * KP + i] : 0.f;
    const float qc = owner ? em[EM_QC * KP + i] : 0.f;
    const float ctr = owner ? em[EM_CTR * KP + i] : -INFINITY, cno = owner ? em[EM_CNO * KP + i] : -INFINITY;
    float *wD = sD + warp * KP;

    const ChunkDesc d = chunks[ch];
    const float2 *obs = packed + d.pstart;
    const int len = d.len;

    float row[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) row[j] = (j == i) ? 1.0f : 0.0f;
    int expo = 0;
    bool bad = false;
    int since = 0;
    int measured = 0;
    int w0 = -32;        // first step of the window held in the lanes
    float2 ob = make_float2(0.f, 0.f);
    unsigned quiet = 0;  // bit u: step w0 + u has no tremor

    // One token per iteration: an ordinary step, or one table power of the run
    // in progress (`pending` holds the powers still to apply). Both share the
    // one copy of the K^3 product below, which keeps the loop small enough
    // for the instruction cache. Control flow is warp-uniform throughout.
    int pending = 0;
    for (int t = 0; t < len || pending;) {
        int boff;      // offset of the right operand in shared memory
        int add;       // exponent this token adds to the row
        bool ordinary;
        if (pending) {
            const int b = __ffs(pending) - 1;
            pending &= pending - 1;
            boff = (1 + b) * KP * KP;
            add = prescale_row<KP>(row, sR + b * KP);
            if (add == INT32_MIN) add = 0;  // the row is zero (and stays zero)
            ordinary = false;
        } else {
            if (t >= w0 + 32) {
                w0 = t;
                const int u = w0 + i;
                ob = u < len ? obs[u] : make_float2(0.f, 0.f);
                quiet = __ballot_sync(0xffffffffu, u < len && isnan(ob.x));
            }
            const int sft = t - w0;
            const float ox = __shfl_sync(0xffffffffu, ob.x, sft);
            const float oy = __shfl_sync(0xffffffffu, ob.y, sft);
            const bool tremor = !isnan(ox);
            if (!tremor && min_run > 0 && t >= measured) {
                const unsigned rest = ~quiet >> sft;  // bit 0 is this (quiet) step
                int n = rest ? __ffs(rest) - 1 : 32 - sft;
                if (!rest && w0 + 32 < len) n += quiet_run(obs + w0 + 32, len - (w0 + 32));
                if (n >= min_run) {
                    pending = n;
                    t += n;
                    measured = t;
                    continue;
                }
                measured = t + n;
            }
            float l;
            if (!tremor) {
                l = cno;
            } else {
                const float dx = ox - mux, dy = oy - muy;
                l = fmaf(qa * dx, dx, fmaf(qb * dx, dy, fmaf(qc * dy, dy, ctr)));
            }
            float m = l;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            int E = 0;
            float di = 0.0f;
            if (m >= -(float)EXP_LIMIT) {
                E = (int)floorf(m);
                di = exp2f(l - (float)E);
            } else if (m != -INFINITY) {
                bad = true;
            }
            if (owner) wD[i] = di;
            boff = 0;
            add = E;
            ordinary = true;
        }
        float nw[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) nw[j] = 0.0f;
        const float *B = smem + boff;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const float rk = row[k];
            const float4 *pk = reinterpret_cast<const float4 *>(B + k * KP);
#pragma unroll
            for (int j4 = 0; j4 < KP / 4; ++j4) {
                const float4 pv = pk[j4];
                nw[4 * j4 + 0] = fmaf(rk, pv.x, nw[4 * j4 + 0]);
                nw[4 * j4 + 1] = fmaf(rk, pv.y, nw[4 * j4 + 1]);
                nw[4 * j4 + 2] = fmaf(rk, pv.z, nw[4 * j4 + 2]);
                nw[4 * j4 + 3] = fmaf(rk, pv.w, nw[4 * j4 + 3]);
            }
        }
        if (ordinary) {
            __syncwarp();  // wD complete
            const float4 *dv = reinterpret_cast<const float4 *>(wD);
#pragma unroll
            for (int j4 = 0; j4 < KP / 4; ++j4) {
                const float4 dd = dv[j4];
                row[4 * j4 + 0] = nw[4 * j4 + 0] * dd.x;
                row[4 * j4 + 1] = nw[4 * j4 + 1] * dd.y;
                row[4 * j4 + 2] = nw[4 * j4 + 2] * dd.z;
                row[4 * j4 + 3] = nw[4 * j4 + 3] * dd.w;
            }
            __syncwarp();  // wD read by every lane before the next step writes it
            ++t;
        } else {
#pragma unroll
            for (int j = 0; j < KP; ++j) row[j] = nw[j];
        }
        expo += add;
        if (!ordinary || ++since == renorm) {
            renorm_row<KP>(row, expo, bad);
            since = 0;
        }
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
        if (bad) atomicOr(status, ST_ENUMERIC);
    }
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
    if (lay.KP <= 32) {
        const dim3 wgrid((n_chunks + RLE_WPC - 1) / RLE_WPC, n_prop);
        const size_t smem = sizeof(float) * ((size_t)lay.KP * lay.KP * (1 + nb) + (size_t)nb * lay.KP +
                                             (size_t)RLE_WPC * lay.KP);
        switch (lay.KP) {
#define HMM_RLE_W(KPV)                                                                                    \
    case KPV: {                                                                                           \
        cudaError_t e = cudaFuncSetAttribute(chunk_rle_warp_kernel<KPV>,                                  \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
        if (e != cudaSuccess) return e;                                                                   \
        chunk_rle_warp_kernel<KPV><<<wgrid, 32 * RLE_WPC, smem, st>>>(n_chunks, renorm, min_run, nb, lay,  \
                                                                      cblock, qtab, qexp, chunks, packed,  \
                                                                      A0, e0, status);                    \
        return cudaGetLastError();                                                                        \
    }
            HMM_RLE_W(4) HMM_RLE_W(8) HMM_RLE_W(16) HMM_RLE_W(32)
#undef HMM_RLE_W
            default: return cudaErrorInvalidValue;
        }
    }
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
