// Chunk products on the tensor cores for wide state spaces (K = 33..80, padded
// to KP = 48, 64 or 80).
//
// The same computation as the K <= 32 kernel (Section "The likelihood
// algorithm", steps 1-3 fused): each chunk's running product advances by
// "multiply by P, then scale column j by the emission D_t[j]", with exact
// power-of-two renormalisation. The mapping changes with the width:
//   * the chunks of a work item are packed densely over the rows of its G
//     128-row MMA operands (row R of the item, R = 128 g + TMEM lane, is
//     start state R mod KP of chunk R / KP), so a chunk may straddle two
//     groups and only the rows past the item's last chunk are padding that
//     the tensor core multiplies along and nobody reads (KP = 80, G = 3: four
//     chunks in 384 rows, where one chunk per group would use 240);
//   * the MMA is M = 128, N = KP, with KP / 8 (TF32) or KP / 16 (BF16)
//     K-steps per pass over P;
//   * a row of KP values is handled in passes of 16 TMEM columns, so the
//     registers of an epilogue thread do not grow with K. On a step that
//     renormalises (every R steps, or when a chunk ends) the row is read
//     twice: once for its maximum, once to scale, round and store it;
//   * each epilogue warp computes the emissions of the (one or two) chunks its
//     32 rows belong to, all KP states of each (several states per lane);
//   * the TMEM lane quadrants that hold only padding rows have no epilogue
//     work; the `empty` barriers count only the quadrants that do.
//
// Warp roles, P and the observation windows by TMA bulk copies, TMEM-resident
// A and D, bounded waits and the abort protocol are those of the K <= 32
// kernel.
#include "hmm_tc_common.cuh"

namespace hmm {

namespace {

template <int KP, int PREC, int G, int E>
struct WideCfg {
    static constexpr int ESZ = PREC == HMM_PREC_BF16 ? 2 : 4;
    static constexpr int KSTEP = 32 / ESZ;                      // K per MMA instruction
    static constexpr int NKS = KP / KSTEP;                      // MMAs per pass over K
    static constexpr int NIMG = PREC == HMM_PREC_TF32 ? 1 : 2;  // P (hi) or P hi + lo
    static constexpr int PI = G * TC_M / KP;                    // chunks per work item
    static constexpr int ROWS = PI * KP;                        // rows of an item that belong to a chunk
    static constexpr int GPW = G / E;                           // groups per epilogue warp
    static constexpr int SBO = KP * ESZ * 8;
    static constexpr int KA = KP * ESZ / 4;                     // TMEM columns of one A row
    static constexpr int NPASS = KP / 16;                       // 16-column passes per row
    static constexpr int KAP = 16 * ESZ / 4;                    // A columns per pass (16 or 8)
    static constexpr int NV = (KP + 31) / 32;                   // states per lane (emission)
    static constexpr int P_BYTES = KP * KP * ESZ * NIMG;
    static constexpr int WIN = 64;                              // observation window (steps)
    static constexpr int CPW = 2;                               // chunk slots per warp (at most)
    static constexpr int EPI_WARPS = 4 * E;
    static constexpr int THREADS = 32 * (NISS + EPI_WARPS);
    static constexpr int TMEM_USED = G * (KP + KA);
    static constexpr int TMEM_COLS = 512;
    static constexpr int A_COL0 = G * KP;
    static constexpr int OFF_P = 0;
    static constexpr int OFF_OBS = OFF_P + ((P_BYTES + 127) / 128) * 128;
    static constexpr int OBS_BYTES = EPI_WARPS * GPW * CPW * 2 * WIN * 8;
    static constexpr int OFF_D = OFF_OBS + OBS_BYTES;
    static constexpr int D_BYTES = EPI_WARPS * GPW * CPW * KP * 4;
    static constexpr int OFF_BAR = OFF_D + D_BYTES;
    // full[G], empty[G], pload, drain[NISS], then two observation-window
    // barriers per epilogue warp (one per buffer)
    static constexpr int NBAR = 2 * G + 1 + NISS + 2 * EPI_WARPS;
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
    static constexpr int SMEM = OFF_MISC + 16 + 1024;
    static_assert(KP == 48 || KP == 64 || KP == 80, "wide tiles cover KP = 48, 64, 80");
    static_assert(G % E == 0, "groups must split evenly over epilogue teams");
    static_assert(GPW == 1, "one group per epilogue warp: the warp's rows are fixed for the kernel");
    static_assert(ROWS > (G - 1) * TC_M, "every group holds chunk rows");
    static_assert(TMEM_USED <= TMEM_COLS, "TMEM holds 512 32-bit columns");
    static_assert(THREADS <= 1024, "threads per CTA");
    static_assert(SMEM <= 232448, "shared memory per CTA");
    static_assert(KP % KSTEP == 0 && KP % 16 == 0, "K tiling");
};

template <int KP, int PREC, int G, int E>
__global__ void __launch_bounds__(WideCfg<KP, PREC, G, E>::THREADS, 1)
chunk_tc_wide_kernel(int n_prop, int n_chunks, int renorm, ConstLayout lay, const float *__restrict__ cblock,
                     const ChunkDesc *__restrict__ chunks, const float2 *__restrict__ packed,
                     float *__restrict__ A0, int32_t *__restrict__ e0, unsigned *__restrict__ status) {
    using C = WideCfg<KP, PREC, G, E>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *full = bars;
    uint64_t *empty = bars + G;
    uint64_t *pload = bars + 2 * G;
    uint64_t *drain = bars + 2 * G + 1;
    uint64_t *obar = drain + NISS;  // [epilogue warp][buffer]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + C::OFF_MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + C::OFF_MISC + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int per_item = C::PI;
    const int items_per_prop = (n_chunks + per_item - 1) / per_item;
    const int n_items = n_prop * items_per_prop;

    if (threadIdx.x == 0) {
        for (int g = 0; g < G; ++g) {
            mbar_init(&full[g], 1);
            // one arrival per quadrant warp that holds chunk rows
            mbar_init(&empty[g], (min(TC_M, C::ROWS - g * TC_M) + 31) / 32);
        }
        mbar_init(pload, 1);
        for (int w = 0; w < NISS; ++w) mbar_init(&drain[w], 1);
        for (int w = 0; w < 2 * C::EPI_WARPS; ++w) mbar_init(&obar[w], 1);
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

    if (warp < NISS) {
        // ---------------- MMA issuers (issuer w serves groups g = w mod 4) ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc<PREC>(KP);
            const uint32_t p_base = smem_u32(smem + C::OFF_P);
            uint32_t empty_par = 0, pload_par = 0;
            bool ok = true, issued = false;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const int b = item % items_per_prop;
                const int steps = item_steps(b);
                const int live_rows = min(per_item, n_chunks - b * per_item) * KP;
                const int live_groups = min(G, (live_rows + TC_M - 1) / TC_M);
                ok = mbar_wait(pload, pload_par, abort_flag, status);
                pload_par ^= 1;
                for (int t = 0; t < steps && ok; ++t) {
                    for (int g = warp; g < live_groups && ok; g += NISS) {
                        ok = mbar_wait(&empty[g], (empty_par >> g) & 1u, abort_flag, status);
                        if (!ok) break;
                        empty_par ^= 1u << g;
                        tc_fence_after();
                        const uint32_t d_tmem = tmem_base + (uint32_t)(g * KP);
                        const uint32_t a_tmem = tmem_base + (uint32_t)(C::A_COL0 + g * C::KA);
#pragma unroll
                        for (int img = 0; img < C::NIMG; ++img) {
#pragma unroll
                            for (int ks = 0; ks < C::NKS; ++ks) {
                                const uint64_t bd = smem_desc(p_base + img * (KP * KP * C::ESZ) + ks * 256, 128, C::SBO);
                                mma_ts<PREC>(d_tmem, a_tmem + ks * 8, bd, idesc, (img | ks) != 0);
                            }
                        }
                        mma_commit(&full[g]);
                        issued = true;
                    }
                }
            }
            if (issued) {
                mma_commit(&drain[warp]);
                const long long t0 = clock64();
                while (!mbar_try_wait(&drain[warp], 0) && clock64() - t0 < SPIN_LIMIT_CYCLES) {
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        const int ew = warp - NISS;
        const int quad = warp & 3;                 // TMEM lane quadrant
        const int team = ew >> 2;
        const int R0 = team * TC_M + quad * 32;    // first row of this warp within the item
        const int R = R0 + lane;                   // this thread's row of the item
        // (KP = 64 tiles every group exactly: every row belongs to a chunk)
        constexpr bool EXACT = (C::ROWS == G * TC_M);
        const bool active = EXACT || R0 < C::ROWS;  // this quadrant holds chunk rows
        const bool vrow = EXACT || R < C::ROWS;     // this row belongs to a chunk
        const int cs = vrow ? R / KP : 0;          // chunk slot of the row within the item
        const int i = (EXACT ? quad * 32 + lane : R) % KP;  // start state of the row
        const int c0 = R0 / KP;                    // first chunk slot of this warp
        const int nch = active ? min(C::PI - 1, (R0 + 31) / KP) - c0 + 1 : 0;
        const int sl = cs - c0;                    // the row's chunk among the warp's
        float2 *sObs = reinterpret_cast<float2 *>(smem + C::OFF_OBS) + (size_t)ew * C::GPW * C::CPW * 2 * C::WIN;
        float *sD = reinterpret_cast<float *>(smem + C::OFF_D) + (size_t)ew * C::GPW * C::CPW * KP;
        const uint32_t tm_row = tmem_base + ((uint32_t)(quad * 32) << 16);
        const int nthr_epi = 32 * C::EPI_WARPS;
        uint32_t full_par = 0, pload_issued = 0;
        int cur_q = -1;
        // emission constants of the states this lane evaluates: lane + 32 v
        float mux[C::NV], muy[C::NV], qa[C::NV], qb[C::NV], qc[C::NV], ctr[C::NV], cno[C::NV];
        // TF32 (one image of P): the running product goes to the tensor core
        // as raw FP32 bits, which it truncates to TF32; every step's emission
        // factors carry the mean-loss compensation 1/(1 - c) (c in
        // hmm_tc_common.cuh), and a chunk's first step, which multiplies the
        // exact identity, has its compensation taken back when the chunk is
        // written. TF32-split rounds to nearest instead.
        constexpr bool TRUNC = (PREC == HMM_PREC_TF32);
        constexpr float TRUNC_COMP = TRUNC ? TF32_TRUNC_COMP_LOG2 : 0.0f;
        const float uncomp = TRUNC ? ex2_approx(-TF32_TRUNC_COMP_LOG2) : 1.0f;

        auto win_ptr = [&](int u, int slot, int bsel) {
            return sObs + (((size_t)u * C::CPW + slot) * 2 + bsel) * C::WIN;
        };
        // per group slot u and chunk slot c (of this warp): start and length
        int64_t pstart[C::GPW][C::CPW];
        int len[C::GPW][C::CPW];
        // Observations arrive by 1-D bulk copies (TMA), one window of WIN steps
        // per chunk slot into one of two buffers, issued by lane 0 with one
        // arrival carrying the byte count on the warp's barrier of that buffer.
        // Chunks start on 64-step boundaries of the packed sequence, so every
        // window starts 512-byte aligned and stays inside its segment's padded
        // region (the K <= 32 kernel relies on the same layout).
        uint64_t *wbar = obar + 2 * ew;
        uint32_t opar = 0, opend = 0;  // per buffer: phase parity, copies pending
        auto win_issue = [&](int wdw, int bsel) {
            if (lane == 0) {
                const int s0 = wdw * C::WIN;
                uint32_t bytes = 0;
#pragma unroll
                for (int u = 0; u < C::GPW; ++u)
#pragma unroll
                    for (int c = 0; c < C::CPW; ++c) bytes += (s0 < len[u][c]) ? (uint32_t)(C::WIN * 8) : 0u;
                fence_proxy_async_smem();  // this buffer's earlier reads come first
                mbar_arrive_expect_tx(&wbar[bsel], bytes);
#pragma unroll
                for (int u = 0; u < C::GPW; ++u)
#pragma unroll
                    for (int c = 0; c < C::CPW; ++c)
                        if (s0 < len[u][c])
                            bulk_g2s(win_ptr(u, c, bsel), packed + pstart[u][c] + s0, C::WIN * 8, &wbar[bsel]);
            }
            opend |= 1u << bsel;
        };
        auto win_wait = [&](int bsel) {
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&wbar[bsel], (opar >> bsel) & 1u, abort_flag, status));
            if (ok) {
                opar ^= 1u << bsel;
                opend &= ~(1u << bsel);
            }
            return ok;
        };
        auto win_drain = [&]() {
#pragma unroll
            for (int bsel = 0; bsel < 2; ++bsel)
                if (opend >> bsel & 1u) {
                    mbar_drain(&wbar[bsel], (opar >> bsel) & 1u);
                    opar ^= 1u << bsel;
                }
            opend = 0;
        };

        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
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
            if (!active) continue;
            if (q != cur_q) {
                const float *em = cblock + (size_t)q * lay.stride + lay.off_emis;
#pragma unroll
                for (int v = 0; v < C::NV; ++v) {
                    const int s = lane + 32 * v;
                    const bool in = s < KP;
                    mux[v] = in ? em[EM_MUX * KP + s] : 0.f;
                    muy[v] = in ? em[EM_MUY * KP + s] : 0.f;
                    qa[v] = in ? em[EM_QA * KP + s] : 0.f;
                    qb[v] = in ? em[EM_QB * KP + s] : 0.f;
                    qc[v] = in ? em[EM_QC * KP + s] : 0.f;
                    ctr[v] = in ? em[EM_CTR * KP + s] + TRUNC_COMP : -INFINITY;
                    cno[v] = in ? em[EM_CNO * KP + s] + TRUNC_COMP : -INFINITY;
                }
                cur_q = q;
            }
            int expo[C::GPW];
            uint32_t glive = 0;
#pragma unroll
            for (int u = 0; u < C::GPW; ++u) {
                const int g = team + E * u;
                const int jg = b * per_item;
                if (jg + (g * TC_M) / KP < n_chunks) glive |= 1u << u;
                expo[u] = 0;
#pragma unroll
                for (int c = 0; c < C::CPW; ++c) {
                    const int j = jg + c0 + c;
                    const bool in = c < nch && j < n_chunks;
                    pstart[u][c] = in ? chunks[j].pstart : 0;
                    len[u][c] = in ? chunks[j].len : 0;
                }
                if (!(glive >> u & 1u)) continue;
                // running product starts as the identity row e_i (padding rows: zero)
#pragma unroll
                for (int p = 0; p < C::NPASS; ++p) {
                    uint32_t w[C::KAP];
#pragma unroll
                    for (int c = 0; c < C::KAP; ++c) {
                        if constexpr (C::ESZ == 4) {
                            w[c] = (vrow && p * 16 + c == i) ? 0x3f800000u : 0u;
                        } else {
                            const int k0 = p * 16 + 2 * c;
                            w[c] = !vrow ? 0u : (k0 == i) ? 0x00003f80u : (k0 + 1 == i) ? 0x3f800000u : 0u;
                        }
                    }
                    tmem_st_row<C::KAP>(tm_row + C::A_COL0 + g * C::KA + p * C::KAP, w);
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[g]);
            }
            // observation windows 0 and 1 of every chunk slot
            win_issue(0, 0);
            win_issue(1, 1);

            int rcount = renorm;
            for (int t = 0; t < steps; ++t) {
                const bool rn_step = (--rcount == 0);
                if (rn_step) rcount = renorm;
                const int w = t % C::WIN;
                const int bsel = (t / C::WIN) & 1;
                if (w == 0) {
                    if (t > 0) {
                        // the other buffer (window t/WIN - 1) is consumed: refill it
                        __syncwarp();
                        win_issue(t / C::WIN + 1, bsel ^ 1);
                    }
                    if (!win_wait(bsel)) break;
                }
                // Step 1 fused: all KP emissions of each chunk of this warp at step t,
                // prescaled by the nearest power of two of the best one
                int Et[C::GPW][C::CPW];
#pragma unroll
                for (int u = 0; u < C::GPW; ++u) {
#pragma unroll
                    for (int c = 0; c < C::CPW; ++c) {
                        Et[u][c] = 0;
                        if (c >= nch) continue;
                        const float2 o = win_ptr(u, c, bsel)[w];
                        const bool none = isnan(o.x);
                        float l[C::NV];
                        float m = -INFINITY;
#pragma unroll
                        for (int v = 0; v < C::NV; ++v) {
                            const float dx = o.x - mux[v], dy = o.y - muy[v];
                            const float lt = fmaf(qa[v] * dx, dx, fmaf(qb[v] * dx, dy, fmaf(qc[v] * dy, dy, ctr[v])));
                            l[v] = none ? cno[v] : lt;
                            m = fmaxf(m, l[v]);
                        }
                        m = chunk_max<32>(m, lane);
                        float mf;
                        const int e = round_to_int(m, mf);
                        const bool ok = m >= -(float)EXP_LIMIT;
                        Et[u][c] = ok ? e : 0;
                        if (!ok && m != -INFINITY && t < len[u][c]) atomicOr(status, ST_ENUMERIC);
                        float *dst = sD + ((size_t)u * C::CPW + c) * KP;
#pragma unroll
                        for (int v = 0; v < C::NV; ++v) {
                            const int s = lane + 32 * v;
                            if (s < KP) dst[s] = ok ? ex2_approx(l[v] - mf) : 0.0f;
                        }
                    }
                }
                __syncwarp();
                const bool more = t + 1 < steps;
#pragma unroll
                for (int u = 0; u < C::GPW; ++u) {
                    const int g = team + E * u;
                    if (!(glive >> u & 1u)) continue;
                    const bool okw = __all_sync(0xffffffffu, mbar_wait(&full[g], (full_par >> g) & 1u, abort_flag, status));
                    full_par ^= 1u << g;
                    // (two-way selects keep the small per-slot arrays in registers)
                    const int my_len = !vrow ? 0 : (sl == 0 ? len[u][0] : len[u][C::CPW - 1]);
                    const bool last = vrow && t + 1 == my_len;
                    if (okw) {
                        tc_fence_after();
                        const float *drow = sD + ((size_t)u * C::CPW + (vrow && sl > 0 ? 1 : 0)) * KP;
                        if (vrow && t < my_len) expo[u] += (sl == 0 ? Et[u][0] : Et[u][C::CPW - 1]);
                        // the row is renormalised on the R-th step and when its chunk ends
                        const bool two = rn_step || __any_sync(0xffffffffu, last);
                        float scl = 1.0f, mx = 0.0f;
                        if (two) {
#pragma unroll
                            for (int p = 0; p < C::NPASS; ++p) {
                                float a[16];
                                tmem_ld16(tm_row + g * KP + p * 16, a);
                                tmem_wait_ld();
                                scale_row<16>(a, drow + p * 16);
                                float m4[4];
#pragma unroll
                                for (int j = 0; j < 4; ++j) m4[j] = max3f(max3f(a[4 * j], a[4 * j + 1], a[4 * j + 2]), a[4 * j + 3], 0.0f);
                                mx = max3f(mx, max3f(m4[0], m4[1], m4[2]), m4[3]);
                            }
                            if (mx > 0.0f) {
                                if (!isfinite(mx) && vrow && t < my_len) atomicOr(status, ST_ENUMERIC);
                                int rr = float_exponent(mx);
                                rr = rr < -126 ? -126 : (rr > 126 ? 126 : rr);
                                scl = pow2f(-rr);
                                expo[u] += rr;
                            }
                        }
                        const size_t jj = (size_t)q * n_chunks + (size_t)b * per_item + cs;
#pragma unroll
                        for (int p = 0; p < C::NPASS; ++p) {
                            float a[16];
                            tmem_ld16(tm_row + g * KP + p * 16, a);
                            tmem_wait_ld();
                            scale_row<16>(a, drow + p * 16);
                            if (two) {
#pragma unroll
                                for (int j = 0; j < 16; ++j) a[j] *= scl;
                            }
                            if (last) {
                                float4 *dst = reinterpret_cast<float4 *>(A0 + jj * KP * KP + (size_t)i * KP + p * 16);
#pragma unroll
                                for (int j4 = 0; j4 < 4; ++j4)
                                    dst[j4] = make_float4(a[4 * j4] * uncomp, a[4 * j4 + 1] * uncomp,
                                                          a[4 * j4 + 2] * uncomp, a[4 * j4 + 3] * uncomp);
                            }
                            if (more) {
                                uint32_t wv[C::KAP];
                                if constexpr (TRUNC) {
#pragma unroll
                                    for (int c = 0; c < 16; ++c) wv[c] = __float_as_uint(a[c]);
                                } else if constexpr (C::ESZ == 4) {
#pragma unroll
                                    for (int c = 0; c < 16; ++c) wv[c] = to_tf32_bits(a[c]);
                                } else {
#pragma unroll
                                    for (int c = 0; c < 8; ++c) {
                                        __nv_bfloat162 bb = __floats2bfloat162_rn(a[2 * c], a[2 * c + 1]);
                                        wv[c] = *reinterpret_cast<uint32_t *>(&bb);
                                    }
                                }
                                tmem_st_row<C::KAP>(tm_row + C::A_COL0 + g * C::KA + p * C::KAP, wv);
                            }
                        }
                        if (last) e0[jj * KP + i] = (mx > 0.0f) ? expo[u] : ZERO_ROW_EXP32;
                        if (more) tmem_wait_st();
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (more && lane == 0) mbar_arrive(&empty[g]);
                }
            }
            // copies issued but not consumed land before the buffers are reused
            win_drain();
        }
        if (ew == 0 && lane == 0 && pload_issued) {
            const long long t0 = clock64();
            while (!mbar_try_wait(pload, (pload_issued - 1) & 1u) && clock64() - t0 < SPIN_LIMIT_CYCLES) {
            }
        }
        win_drain();
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
cudaError_t launch_wide_t(int n_prop, int n_chunks, int renorm, const ConstLayout &lay, const float *cblock,
                          const ChunkDesc *chunks, const float2 *packed, float *A0, int32_t *e0, unsigned *status,
                          cudaStream_t st) {
    using C = WideCfg<KP, PREC, G, E>;
    auto kern = chunk_tc_wide_kernel<KP, PREC, G, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_item = C::PI;
    const long long n_items = (long long)n_prop * ((n_chunks + per_item - 1) / per_item);
    const int grid = (int)(n_items < sms ? n_items : sms);
    kern<<<grid, C::THREADS, C::SMEM, st>>>(n_prop, n_chunks, renorm, lay, cblock, chunks, packed, A0, e0, status);
    return cudaGetLastError();
}

// groups in flight G (TMEM: G (KP + KA) <= 512 columns) and epilogue teams E
template <int KP, int PREC>
struct WideTile;
template <> struct WideTile<48, HMM_PREC_TF32> { static constexpr int G = 5, E = 5; };
template <> struct WideTile<48, HMM_PREC_TF32_SPLIT> { static constexpr int G = 5, E = 5; };
template <> struct WideTile<48, HMM_PREC_BF16> { static constexpr int G = 7, E = 7; };
template <> struct WideTile<64, HMM_PREC_TF32> { static constexpr int G = 4, E = 4; };
template <> struct WideTile<64, HMM_PREC_TF32_SPLIT> { static constexpr int G = 4, E = 4; };
template <> struct WideTile<64, HMM_PREC_BF16> { static constexpr int G = 5, E = 5; };
template <> struct WideTile<80, HMM_PREC_TF32> { static constexpr int G = 3, E = 3; };
template <> struct WideTile<80, HMM_PREC_TF32_SPLIT> { static constexpr int G = 3, E = 3; };
template <> struct WideTile<80, HMM_PREC_BF16> { static constexpr int G = 4, E = 4; };

}  // namespace

int chunk_tc_wide_chunks_per_item(int KP, int precision) {
#define HMM_WIDE_PER_ITEM(KPV, PRECV) \
    if (KP == KPV && precision == PRECV) return WideTile<KPV, PRECV>::G * TC_M / KPV;
    HMM_WIDE_PER_ITEM(48, HMM_PREC_TF32)
    HMM_WIDE_PER_ITEM(64, HMM_PREC_TF32)
    HMM_WIDE_PER_ITEM(80, HMM_PREC_TF32)
    HMM_WIDE_PER_ITEM(48, HMM_PREC_TF32_SPLIT)
    HMM_WIDE_PER_ITEM(64, HMM_PREC_TF32_SPLIT)
    HMM_WIDE_PER_ITEM(80, HMM_PREC_TF32_SPLIT)
    HMM_WIDE_PER_ITEM(48, HMM_PREC_BF16)
    HMM_WIDE_PER_ITEM(64, HMM_PREC_BF16)
    HMM_WIDE_PER_ITEM(80, HMM_PREC_BF16)
#undef HMM_WIDE_PER_ITEM
    return 0;
}

cudaError_t launch_chunk_tc_wide(int n_prop, int n_chunks, int renorm, int precision, const ConstLayout &lay,
                                 const float *cblock, const ChunkDesc *chunks, const float2 *packed, float *A0,
                                 int32_t *e0, unsigned *status, cudaStream_t st) {
    if (n_chunks == 0 || n_prop == 0) return cudaSuccess;
#define HMM_WIDE_CASE(KPV, PRECV)                                                                         \
    if (lay.KP == KPV && precision == PRECV)                                                               \
        return launch_wide_t<KPV, PRECV, WideTile<KPV, PRECV>::G, WideTile<KPV, PRECV>::E>(                \
            n_prop, n_chunks, renorm, lay, cblock, chunks, packed, A0, e0, status, st);
    HMM_WIDE_CASE(48, HMM_PREC_TF32)
    HMM_WIDE_CASE(64, HMM_PREC_TF32)
    HMM_WIDE_CASE(80, HMM_PREC_TF32)
    HMM_WIDE_CASE(48, HMM_PREC_TF32_SPLIT)
    HMM_WIDE_CASE(64, HMM_PREC_TF32_SPLIT)
    HMM_WIDE_CASE(80, HMM_PREC_TF32_SPLIT)
    HMM_WIDE_CASE(48, HMM_PREC_BF16)
    HMM_WIDE_CASE(64, HMM_PREC_BF16)
    HMM_WIDE_CASE(80, HMM_PREC_BF16)
#undef HMM_WIDE_CASE
    return cudaErrorInvalidValue;
}

}  // namespace hmm
