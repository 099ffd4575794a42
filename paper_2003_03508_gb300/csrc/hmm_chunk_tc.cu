// Chunk products on the 5th-generation tensor cores (tcgen05, TMEM, TMA).
//
// Same computation as the FP32-SIMT path (Section "The likelihood algorithm",
// steps 1-3, fused): every chunk's product A_c = prod_{t in c} P D_t, each
// step being "multiply the running product by P, then scale column j by the
// emission D_t[j]", with exact power-of-two scaling (Section "Step 3", last
// paragraph).
//
// Mapping onto the tensor cores. The running products of 128/KP chunks of one
// proposal are stacked into a 128-row operand A (row = chunk x start state),
// so one M=128, N=KP MMA advances all of them by one step against the shared
// B operand P:
//     D[r][n] = sum_k A[r][k] P[k][n]            (tcgen05.mma, FP32 in TMEM)
//     A'[r][n] = D[r][n] * D_t(chunk(r))[n]      (epilogue, registers)
// A lives in shared memory (K-major, canonical no-swizzle layout), P arrives
// by a TMA bulk copy, D is an FP32 accumulator in tensor memory. A CTA keeps
// G such 128-row groups in flight so the tensor core works on one group while
// the epilogue warps scale and write back the others.
//
// Warp roles: warp 0 allocates TMEM and one lane issues every MMA; warps
// 4..4+4E-1 are the epilogue (warp w reads TMEM lanes 32*(w%4)..+31 and owns
// those rows of groups g = team, team+E, ...). Warps 1-3 only join the final
// barrier.
//
// Every wait is bounded: a wait that runs out sets the context's ETIMEOUT
// status bit and an abort flag; all warps then drain (in-flight copies and
// MMAs) and return, and the TMEM is freed.
#include <cuda_bf16.h>

#include "hmm_internal.cuh"

namespace hmm {

namespace {

constexpr int TC_M = 128;
constexpr long long SPIN_LIMIT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on one phase of an mbarrier. Returns false (and raises the
// CTA's abort flag and the ETIMEOUT status bit) if it runs out, or at once
// if another warp already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > SPIN_LIMIT_CYCLES) {
            *abort_flag = 1;
            atomicOr(status, ST_ETIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, `lbo` bytes between core matrices along K,
// `sbo` bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, no swizzle
}

// Instruction descriptor: FP32 accumulate, A and B K-major, M = 128, N = n.
template <int PREC>
__host__ __device__ constexpr uint32_t instr_desc(int n) {
    // A/B format: TF32 = 2 (kind::tf32), BF16 = 1 (kind::f16)
    return (1u << 4) | ((PREC == HMM_PREC_BF16 ? 1u : 2u) << 7) |
           ((PREC == HMM_PREC_BF16 ? 1u : 2u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(TC_M >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate) {
    if constexpr (PREC == HMM_PREC_BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 columns of 32-bit TMEM data into 16 registers per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// barrier over the epilogue warps that also ORs a predicate across them
__device__ __forceinline__ bool named_barrier_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

template <int KP, int PREC, int G, int E>
struct TcCfg {
    static constexpr int ESZ = PREC == HMM_PREC_BF16 ? 2 : 4;  // bytes per operand element
    static constexpr int KSTEP = 32 / ESZ;                      // K per MMA instruction
    static constexpr int NKS = KP / KSTEP;                      // MMAs per pass over K
    static constexpr int NIMG = PREC == HMM_PREC_TF32 ? 1 : 2;  // P (hi) or P hi + lo
    static constexpr int CPW = 32 / KP;                         // chunks per warp
    static constexpr int CPG = TC_M / KP;                       // chunks per group
    static constexpr int GPW = G / E;                           // groups per epilogue warp
    static constexpr int SBO = KP * ESZ * 8;                    // bytes between 8-row groups
    static constexpr int A_BYTES = TC_M * KP * ESZ;             // one group's A operand
    static constexpr int P_BYTES = KP * KP * ESZ * NIMG;
    static constexpr int NWIN = OBS_WIN / KP;                   // window entries per lane
    static constexpr int EPI_WARPS = 4 * E;
    static constexpr int THREADS = 32 * (4 + EPI_WARPS);
    static constexpr int TMEM_COLS = (G * KP <= 32) ? 32 : (G * KP <= 64) ? 64 : (G * KP <= 128) ? 128
                                     : (G * KP <= 256) ? 256 : 512;
    // shared memory carve (bytes)
    static constexpr int OFF_A = 0;
    static constexpr int OFF_P = OFF_A + G * A_BYTES;
    static constexpr int OFF_OBS = OFF_P + ((P_BYTES + 127) / 128) * 128;
    static constexpr int OBS_BYTES = EPI_WARPS * GPW * CPW * OBS_WIN * 8;
    static constexpr int OFF_D = OFF_OBS + OBS_BYTES;
    static constexpr int OFF_BAR = OFF_D + EPI_WARPS * 32 * 4;
    static constexpr int NBAR = 2 * G + 2;  // full[G], empty[G], pload, drain
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
    static constexpr int SMEM = OFF_MISC + 16 + 1024;  // + slack for 1 KB alignment
    static_assert(G % E == 0, "groups must split evenly over epilogue teams");
    static_assert(KP == 16 || KP == 32, "this tile shape covers KP = 16 and 32");
    static_assert(G * KP <= 512, "TMEM holds 512 FP32 columns");
};

template <int KP, int PREC, int G, int E>
__global__ void __launch_bounds__(TcCfg<KP, PREC, G, E>::THREADS, 1)
chunk_tc_kernel(int n_prop, int n_chunks, int renorm, int K, ConstLayout lay,
                const float *__restrict__ cblock, const ChunkDesc *__restrict__ chunks,
                const float2 *__restrict__ packed, float *__restrict__ A0, int32_t *__restrict__ e0,
                unsigned *__restrict__ status) {
    using C = TcCfg<KP, PREC, G, E>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *full = bars;
    uint64_t *empty = bars + G;
    uint64_t *pload = bars + 2 * G;
    uint64_t *drain = bars + 2 * G + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + C::OFF_MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + C::OFF_MISC + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int per_item = G * C::CPG;  // chunks per work item
    const int items_per_prop = (n_chunks + per_item - 1) / per_item;
    const int n_items = n_prop * items_per_prop;

    if (threadIdx.x == 0) {
        for (int g = 0; g < G; ++g) {
            mbar_init(&full[g], 1);
            mbar_init(&empty[g], 4);  // one arrival per lane-quadrant warp of the team
        }
        mbar_init(pload, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    auto item_steps = [&](int b) {
        int j0 = b * per_item, j1 = min(j0 + per_item, n_chunks), s = 0;
        for (int j = j0; j < j1; ++j) s = max(s, chunks[j].len);
        return s;
    };

    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc<PREC>(KP);
            const uint32_t a_base = smem_u32(smem + C::OFF_A);
            const uint32_t p_base = smem_u32(smem + C::OFF_P);
            uint32_t empty_par = 0, pload_par = 0;
            bool ok = true;
            bool issued = false;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const int b = item % items_per_prop;
                const int steps = item_steps(b);
                const int live_groups = min(G, (n_chunks - b * per_item + C::CPG - 1) / C::CPG);
                ok = mbar_wait(pload, pload_par, abort_flag, status);
                pload_par ^= 1;
                for (int t = 0; t < steps && ok; ++t) {
                    for (int g = 0; g < live_groups && ok; ++g) {
                        ok = mbar_wait(&empty[g], (empty_par >> g) & 1u, abort_flag, status);
                        if (!ok) break;
                        empty_par ^= 1u << g;
                        tc_fence_after();
                        const uint32_t d_tmem = tmem_base + (uint32_t)(g * KP);
                        const uint32_t a_g = a_base + (uint32_t)(g * C::A_BYTES);
#pragma unroll
                        for (int img = 0; img < C::NIMG; ++img) {
#pragma unroll
                            for (int ks = 0; ks < C::NKS; ++ks) {
                                const uint64_t ad = smem_desc(a_g + ks * 256, 128, C::SBO);
                                const uint64_t bd = smem_desc(p_base + img * (KP * KP * C::ESZ) + ks * 256, 128, C::SBO);
                                mma<PREC>(d_tmem, ad, bd, idesc, (img | ks) != 0);
                            }
                        }
                        mma_commit(&full[g]);
                        issued = true;
                    }
                }
            }
            if (issued) {
                // every MMA issued so far completes before the TMEM is freed
                mma_commit(drain);
                const long long t0 = clock64();
                while (!mbar_try_wait(drain, 0) && clock64() - t0 < SPIN_LIMIT_CYCLES) {
                }
            }
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---------------- epilogue ----------------
        const int ew = warp - 4;          // epilogue warp index
        const int quad = warp & 3;        // TMEM lane quadrant
        const int team = ew >> 2;
        const int r = quad * 32 + lane;   // row of the 128-row group
        const int cs = r / KP;            // chunk slot within the group
        const int i = r % KP;             // start state / state index of this lane
        const int half = lane / KP;       // chunk within the warp
        const int jl = lane % KP;         // lane within its chunk
        float2 *sObs = reinterpret_cast<float2 *>(smem + C::OFF_OBS) + (size_t)ew * C::GPW * C::CPW * OBS_WIN;
        float *sD = reinterpret_cast<float *>(smem + C::OFF_D) + ew * 32;
        const uint32_t a_base = smem_u32(smem + C::OFF_A);
        const int nthr_epi = 32 * C::EPI_WARPS;
        uint32_t full_par = 0, pload_issued = 0;
        int cur_q = -1;
        float mux = 0.f, muy = 0.f, qa = 0.f, qb = 0.f, qc = 0.f, ctr = -INFINITY, cno = -INFINITY;

        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            // previous item fully consumed by every epilogue warp (so every MMA
            // that read P has completed); agree on abort
            if (named_barrier_or(1, nthr_epi, *abort_flag != 0)) break;
            const int q = item / items_per_prop;
            const int b = item % items_per_prop;
            const int steps = item_steps(b);
            if (ew == 0 && lane == 0) {
                mbar_arrive_expect_tx(pload, C::P_BYTES);
                const float *src = cblock + (size_t)q * lay.stride + lay.off_tc;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(smem + C::OFF_P)),
                    "l"(src), "r"((uint32_t)C::P_BYTES), "r"(smem_u32(pload))
                    : "memory");
                ++pload_issued;
            }
            if (q != cur_q) {
                const float *em = cblock + (size_t)q * lay.stride + lay.off_emis;
                mux = em[EM_MUX * KP + i];
                muy = em[EM_MUY * KP + i];
                qa = em[EM_QA * KP + i];
                qb = em[EM_QB * KP + i];
                qc = em[EM_QC * KP + i];
                ctr = em[EM_CTR * KP + i];
                cno = em[EM_CNO * KP + i];
                cur_q = q;
            }
            // per group state of this lane's chunk
            int64_t pstart[C::GPW];
            int len[C::GPW];
            int jchunk[C::GPW];
            int expo[C::GPW];
            bool glive[C::GPW];
            float2 pf[C::GPW][C::NWIN];
#pragma unroll
            for (int u = 0; u < C::GPW; ++u) {
                const int g = team + E * u;
                const int jg = b * per_item + g * C::CPG;
                glive[u] = jg < n_chunks;
                const int j = jg + cs;
                jchunk[u] = j;
                expo[u] = 0;
                if (j < n_chunks) {
                    pstart[u] = chunks[j].pstart;
                    len[u] = chunks[j].len;
                } else {
                    pstart[u] = 0;
                    len[u] = 0;
                }
                if (!glive[u]) continue;
                // running product starts as the identity row e_i
                const uint32_t arow = a_base + g * C::A_BYTES + (r >> 3) * C::SBO + (r & 7) * 16;
#pragma unroll
                for (int kc = 0; kc < KP * C::ESZ / 16; ++kc) {
                    uint32_t w[4] = {0u, 0u, 0u, 0u};
                    if constexpr (C::ESZ == 4) {
                        if (i / 4 == kc) w[i % 4] = 0x3f800000u;  // 1.0f
                    } else {
                        if (i / 8 == kc) w[(i % 8) / 2] = (i % 2) ? 0x3f800000u : 0x00003f80u;  // bf16 1.0
                    }
                    st_shared_v4(arow + kc * 128, w[0], w[1], w[2], w[3]);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[g]);
                // prefetch the first observation window of this lane's chunk
#pragma unroll
                for (int v = 0; v < C::NWIN; ++v) {
                    const int s = jl + KP * v;
                    pf[u][v] = (s < len[u]) ? packed[pstart[u] + s]
                                            : make_float2(__int_as_float(0x7fc00000), 0.f);
                }
            }

            for (int t = 0; t < steps; ++t) {
                const int w = t % OBS_WIN;
#pragma unroll
                for (int u = 0; u < C::GPW; ++u) {
                    if (!glive[u]) continue;
                    const int g = team + E * u;
                    float2 *win = sObs + ((size_t)u * C::CPW + half) * OBS_WIN;
                    if (w == 0) {
                        __syncwarp();
#pragma unroll
                        for (int v = 0; v < C::NWIN; ++v) win[jl + KP * v] = pf[u][v];
                        __syncwarp();
#pragma unroll
                        for (int v = 0; v < C::NWIN; ++v) {
                            const int s = t + OBS_WIN + jl + KP * v;
                            pf[u][v] = (s < len[u]) ? packed[pstart[u] + s]
                                                    : make_float2(__int_as_float(0x7fc00000), 0.f);
                        }
                    }
                    const bool act = t < len[u];
                    // Step 1 fused: emission of state i for this chunk's step t (log2)
                    const float2 o = win[w];
                    float l;
                    if (isnan(o.x)) {
                        l = cno;
                    } else {
                        const float dx = o.x - mux, dy = o.y - muy;
                        l = fmaf(qa * dx, dx, fmaf(qb * dx, dy, fmaf(qc * dy, dy, ctr)));
                    }
                    float m = l;
#pragma unroll
                    for (int off = KP / 2; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                    int Et = 0;
                    float d;
                    if (m >= -(float)EXP_LIMIT) {
                        Et = (int)floorf(m);
                        d = exp2f(l - (float)Et);
                    } else {
                        if (m != -INFINITY && act) atomicOr(status, ST_ENUMERIC);
                        d = 0.0f;
                    }
                    sD[lane] = d;
                    __syncwarp();
                    // the MMA for this step has finished (warp-uniform decision)
                    const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[g], (full_par >> g) & 1u, abort_flag, status));
                    full_par ^= 1u << g;
                    if (ok) {
                        tc_fence_after();
                        float acc[KP];
                        const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(g * KP);
#pragma unroll
                        for (int c16 = 0; c16 < KP / 16; ++c16) tmem_ld16(taddr + c16 * 16, acc + c16 * 16);
                        tmem_wait_ld();
                        if (act) {
                            // Step 2 fused: column scale by D_t
                            const float4 *dv = reinterpret_cast<const float4 *>(sD + half * KP);
#pragma unroll
                            for (int j4 = 0; j4 < KP / 4; ++j4) {
                                const float4 dd = dv[j4];
                                acc[4 * j4 + 0] *= dd.x;
                                acc[4 * j4 + 1] *= dd.y;
                                acc[4 * j4 + 2] *= dd.z;
                                acc[4 * j4 + 3] *= dd.w;
                            }
                            expo[u] += Et;
                            const bool last = (t + 1 == len[u]);
                            if ((t + 1) % renorm == 0 || last) {
                                float mx = 0.0f;
#pragma unroll
                                for (int j = 0; j < KP; ++j) mx = fmaxf(mx, acc[j]);
                                if (mx > 0.0f) {
                                    if (!isfinite(mx)) atomicOr(status, ST_ENUMERIC);
                                    int rr = float_exponent(mx);
                                    rr = rr < -126 ? -126 : (rr > 126 ? 126 : rr);
                                    const float s = pow2f(-rr);
#pragma unroll
                                    for (int j = 0; j < KP; ++j) acc[j] *= s;
                                    expo[u] += rr;
                                }
                            }
                            if (!last) {
                                // next A operand row (rounded to the operand type)
                                const uint32_t arow = a_base + g * C::A_BYTES + (r >> 3) * C::SBO + (r & 7) * 16;
                                if constexpr (C::ESZ == 4) {
#pragma unroll
                                    for (int kc = 0; kc < KP / 4; ++kc)
                                        st_shared_v4(arow + kc * 128, to_tf32_bits(acc[4 * kc]),
                                                     to_tf32_bits(acc[4 * kc + 1]), to_tf32_bits(acc[4 * kc + 2]),
                                                     to_tf32_bits(acc[4 * kc + 3]));
                                } else {
#pragma unroll
                                    for (int kc = 0; kc < KP / 8; ++kc) {
                                        uint32_t w4[4];
#pragma unroll
                                        for (int h = 0; h < 4; ++h) {
                                            __nv_bfloat162 bb = __floats2bfloat162_rn(acc[8 * kc + 2 * h], acc[8 * kc + 2 * h + 1]);
                                            w4[h] = *reinterpret_cast<uint32_t *>(&bb);
                                        }
                                        st_shared_v4(arow + kc * 128, w4[0], w4[1], w4[2], w4[3]);
                                    }
                                }
                                fence_proxy_async_smem();
                            } else {
                                float mx = 0.0f;
#pragma unroll
                                for (int j = 0; j < KP; ++j) mx = fmaxf(mx, acc[j]);
                                const size_t j = (size_t)q * n_chunks + jchunk[u];
                                float4 *dst = reinterpret_cast<float4 *>(A0 + j * KP * KP + (size_t)i * KP);
#pragma unroll
                                for (int j4 = 0; j4 < KP / 4; ++j4)
                                    dst[j4] = make_float4(acc[4 * j4], acc[4 * j4 + 1], acc[4 * j4 + 2], acc[4 * j4 + 3]);
                                e0[j * KP + i] = (mx > 0.0f) ? expo[u] : ZERO_ROW_EXP32;
                            }
                        }
                        tc_fence_before();
                    }
                    __syncwarp();
                    if (t + 1 < steps && lane == 0) mbar_arrive(&empty[g]);
                }
            }
        }
        // a bulk copy that was issued but never consumed must land before exit
        if (ew == 0 && lane == 0 && pload_issued) {
            const long long t0 = clock64();
            while (!mbar_try_wait(pload, (pload_issued - 1) & 1u) && clock64() - t0 < SPIN_LIMIT_CYCLES) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(C::TMEM_COLS)
                     : "memory");
    }
}

template <int KP, int PREC, int G, int E>
cudaError_t launch_tc_t(int n_prop, int n_chunks, int renorm, int K, const ConstLayout &lay,
                        const float *cblock, const ChunkDesc *chunks, const float2 *packed, float *A0,
                        int32_t *e0, unsigned *status, cudaStream_t st) {
    using C = TcCfg<KP, PREC, G, E>;
    auto kern = chunk_tc_kernel<KP, PREC, G, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_item = G * C::CPG;
    const long long n_items = (long long)n_prop * ((n_chunks + per_item - 1) / per_item);
    const int grid = (int)(n_items < sms ? n_items : sms);
    kern<<<grid, C::THREADS, C::SMEM, st>>>(n_prop, n_chunks, renorm, K, lay, cblock, chunks, packed, A0, e0,
                                             status);
    return cudaGetLastError();
}

}  // namespace

bool chunk_tc_supported(int K, int precision) {
    if (precision != HMM_PREC_TF32 && precision != HMM_PREC_TF32_SPLIT && precision != HMM_PREC_BF16) return false;
    return K >= 1 && K <= 32;
}

int chunk_tc_chunks_per_item(int KP) { return 8 * (TC_M / KP); }

cudaError_t launch_chunk_tc(int n_prop, int n_chunks, int L, int renorm, int precision,
                            const ConstLayout &lay, const float *cblock, const ChunkDesc *chunks,
                            const float2 *packed, float *A0, int32_t *e0, unsigned *status,
                            cudaStream_t st) {
    (void)L;
    if (n_chunks == 0 || n_prop == 0) return cudaSuccess;
    const int K = 0;
#define HMM_TC_CASE(KPV, PRECV)                                                                    \
    if (lay.KP == KPV && precision == PRECV)                                                        \
        return launch_tc_t<KPV, PRECV, 8, 2>(n_prop, n_chunks, renorm, K, lay, cblock, chunks, packed, \
                                              A0, e0, status, st);
    HMM_TC_CASE(16, HMM_PREC_TF32)
    HMM_TC_CASE(32, HMM_PREC_TF32)
    HMM_TC_CASE(16, HMM_PREC_TF32_SPLIT)
    HMM_TC_CASE(32, HMM_PREC_TF32_SPLIT)
    HMM_TC_CASE(16, HMM_PREC_BF16)
    HMM_TC_CASE(32, HMM_PREC_BF16)
#undef HMM_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace hmm
