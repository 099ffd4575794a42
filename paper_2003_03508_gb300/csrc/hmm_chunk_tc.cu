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
// Both A and the FP32 accumulator D live in tensor memory (TMEM): with N = KP
// as small as 32, an A operand in shared memory would be re-read by every MMA
// and rewritten by every epilogue, and shared-memory bandwidth, not the tensor
// core, would set the pace. P (the B operand, canonical K-major no-swizzle
// layout) arrives in shared memory by a TMA bulk copy. A CTA keeps G such
// 128-row groups in flight so the tensor core works on one group while the
// epilogue warps scale and write back the others.
//
// Warp roles: warp 0 allocates TMEM; lane 0 of warps 0..3 issue the MMAs
// (issuer w serves groups g = w mod 4); warps 4..4+4E-1 are the epilogue
// (warp w reads TMEM lanes 32*(w%4)..+31 and owns those rows of groups
// g = team, team+E, ...).
//
// Every wait is bounded: a wait that runs out sets the context's ETIMEOUT
// status bit and an abort flag; all warps then drain (in-flight copies and
// MMAs) and return, and the TMEM is freed.
#include <type_traits>

#include "hmm_tc_common.cuh"

namespace hmm {

namespace {

template <int KP, int PREC, int G, int E>
struct TcCfg {
    static constexpr int ESZ = PREC == HMM_PREC_BF16 ? 2 : 4;  // bytes per operand element
    static constexpr int KSTEP = 32 / ESZ;                      // K per MMA instruction
    static constexpr int NKS = KP / KSTEP;                      // MMAs per pass over K
    static constexpr int NIMG = PREC == HMM_PREC_TF32 ? 1 : 2;  // P (hi) or P hi + lo
    static constexpr int CPW = 32 / KP;                         // chunks per warp
    static constexpr int CPG = TC_M / KP;                       // chunks per group
    static constexpr int GPW = G / E;                           // groups per epilogue warp
    static constexpr int SBO = KP * ESZ * 8;                    // bytes between 8-row groups of P
    static constexpr int KA = KP * ESZ / 4;                     // TMEM columns of one A row
    static constexpr int P_BYTES = KP * KP * ESZ * NIMG;
    static constexpr int WIN = KP == 32 ? 64 : 32;              // observation window (steps)
    static constexpr int EPI_WARPS = 4 * E;
    static constexpr int THREADS = 32 * (4 + EPI_WARPS);
    // TMEM: G accumulators D (KP columns each), then G running products A (KA columns each)
    static constexpr int TMEM_USED = G * (KP + KA);
    static constexpr int TMEM_COLS = (TMEM_USED <= 32) ? 32 : (TMEM_USED <= 64) ? 64 : (TMEM_USED <= 128) ? 128
                                     : (TMEM_USED <= 256) ? 256 : 512;
    static constexpr int A_COL0 = G * KP;
    // shared memory carve (bytes)
    static constexpr int OFF_P = 0;
    static constexpr int OFF_OBS = OFF_P + ((P_BYTES + 127) / 128) * 128;
    static constexpr int OBS_BYTES = EPI_WARPS * GPW * CPW * 2 * WIN * 8;  // double buffered
    static constexpr int OFF_D = OFF_OBS + OBS_BYTES;
    static constexpr int D_BYTES = EPI_WARPS * GPW * 32 * 4;
    static constexpr int OFF_BAR = OFF_D + D_BYTES;
    // full[G], empty[G], pload, drain[4], then two observation-window
    // barriers per epilogue warp (one per buffer)
    static constexpr int NBAR = 2 * G + 1 + 4 + 2 * EPI_WARPS;
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
    static constexpr int SMEM = OFF_MISC + 16 + 1024;  // + slack for 1 KB alignment
    static_assert(G % E == 0, "groups must split evenly over epilogue teams");
    static_assert(KP == 16 || KP == 32, "this tile shape covers KP = 16 and 32");
    static_assert(TMEM_USED <= 512, "TMEM holds 512 32-bit columns");
    static_assert(G <= 32, "group bitmasks are 32-bit");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

template <int KP, int PREC, int G, int E>
__global__ void __launch_bounds__(TcCfg<KP, PREC, G, E>::THREADS, 1)
chunk_tc_kernel(int n_prop, int n_chunks, int renorm, ConstLayout lay, const float *__restrict__ cblock,
                const ChunkDesc *__restrict__ chunks, const float2 *__restrict__ packed,
                float *__restrict__ A0, int32_t *__restrict__ e0, unsigned *__restrict__ status) {
    using C = TcCfg<KP, PREC, G, E>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    uint64_t *full = bars;
    uint64_t *empty = bars + G;
    uint64_t *pload = bars + 2 * G;
    uint64_t *drain = bars + 2 * G + 1;  // one per issuer
    uint64_t *obar = drain + NISS;       // [epilogue warp][buffer]
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
        for (int w = 0; w < NISS; ++w) mbar_init(&drain[w], 1);
        // one arrival per chunk of the warp (its first lane issues the copies)
        for (int w = 0; w < 2 * C::EPI_WARPS; ++w) mbar_init(&obar[w], C::CPW);
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
        // ---------------- MMA issuers ----------------
        // One thread issues a tcgen05.mma only every few tens of cycles, far less
        // work than one M=128, N=KP MMA holds, so four warps (one per SM
        // sub-partition) issue in parallel; issuer w owns groups g = w (mod 4)
        // and serves them in order.
        if (lane == 0) {
            const uint32_t idesc = instr_desc<PREC>(KP);
            const uint32_t p_base = smem_u32(smem + C::OFF_P);
            // B descriptors of every MMA of a group-step (P's images never move)
            uint64_t bd[C::NIMG * C::NKS];
#pragma unroll
            for (int img = 0; img < C::NIMG; ++img)
#pragma unroll
                for (int ks = 0; ks < C::NKS; ++ks)
                    bd[img * C::NKS + ks] = smem_desc(p_base + img * (KP * KP * C::ESZ) + ks * 256, 128, C::SBO);
            uint32_t empty_par = 0, pload_par = 0;
            bool ok = true, issued = false;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const int b = item % items_per_prop;
                const int steps = item_steps(b);
                const int live_groups = min(G, (n_chunks - b * per_item + C::CPG - 1) / C::CPG);
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
                        // one MMA consumes 32 bytes of K: 8 TMEM columns of A
                        mma_group<PREC, C::NIMG, C::NKS>(d_tmem, a_tmem, bd, idesc);
                        mma_commit(&full[g]);
                        issued = true;
                    }
                }
            }
            if (issued) {
                // every MMA this thread issued completes before the TMEM is freed
                mma_commit(&drain[warp]);
                const long long t0 = clock64();
                while (!mbar_try_wait(&drain[warp], 0) && clock64() - t0 < SPIN_LIMIT_CYCLES) {
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
        float2 *sObs = reinterpret_cast<float2 *>(smem + C::OFF_OBS) + (size_t)ew * C::GPW * C::CPW * 2 * C::WIN;
        float *sD = reinterpret_cast<float *>(smem + C::OFF_D) + ew * C::GPW * 32;
        const uint32_t tm_row = tmem_base + ((uint32_t)(quad * 32) << 16);
        const int nthr_epi = 32 * C::EPI_WARPS;
        uint32_t full_par = 0, pload_issued = 0;
        int cur_q = -1;
        float mux = 0.f, muy = 0.f, qa = 0.f, qb = 0.f, qc = 0.f, ctr = -INFINITY, cno = -INFINITY;

        // window buffer for (group slot u, buffer b) of this lane's chunk
        auto win_ptr = [&](int u, int bsel) {
            return sObs + (((size_t)u * C::CPW + half) * 2 + bsel) * C::WIN;
        };
        // Observations arrive by 1-D bulk copies (TMA), one window of WIN steps
        // per chunk into one of two buffers, completion counted on the warp's
        // barrier of that buffer. Every chunk starts on a 64-step boundary of
        // the packed sequence (segments are laid out on 64-step boundaries and
        // chunk lengths are multiples of 64), so every window starts 256-byte
        // aligned, and a window that runs past its chunk's end stays inside the
        // segment's padded region. The first lane of each chunk issues its
        // copies and one arrival with the byte count (zero when the chunk has
        // no step left in that window).
        uint64_t *wbar = obar + 2 * ew;
        uint32_t opar = 0, opend = 0;  // per buffer: phase parity, copies pending
        int64_t pstart[C::GPW];        // per group slot: this lane's chunk's first step
        int len[C::GPW];               // and its length (0: no chunk)
        auto win_issue = [&](int wdw, int bsel) {
            if (jl == 0) {
                const int s0 = wdw * C::WIN;
                uint32_t bytes = 0;
#pragma unroll
                for (int u = 0; u < C::GPW; ++u) bytes += (s0 < len[u]) ? (uint32_t)(C::WIN * 8) : 0u;
                fence_proxy_async_smem();  // this buffer's earlier reads come first
                mbar_arrive_expect_tx(&wbar[bsel], bytes);
#pragma unroll
                for (int u = 0; u < C::GPW; ++u)
                    if (s0 < len[u]) bulk_g2s(win_ptr(u, bsel), packed + pstart[u] + s0, C::WIN * 8, &wbar[bsel]);
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
            int expo[C::GPW];
            uint32_t glive = 0;
#pragma unroll
            for (int u = 0; u < C::GPW; ++u) {
                const int g = team + E * u;
                const int jg = b * per_item + g * C::CPG;
                if (jg < n_chunks) glive |= 1u << u;
                const int j = jg + cs;
                expo[u] = 0;
                pstart[u] = j < n_chunks ? chunks[j].pstart : 0;
                len[u] = j < n_chunks ? chunks[j].len : 0;
                if (!(glive >> u & 1u)) continue;
                // running product starts as the identity row e_i (in TMEM)
                {
                    uint32_t w[C::KA];
#pragma unroll
                    for (int c = 0; c < C::KA; ++c) {
                        if constexpr (C::ESZ == 4) w[c] = (c == i) ? 0x3f800000u : 0u;  // 1.0f
                        else w[c] = (c == i / 2) ? ((i & 1) ? 0x3f800000u : 0x00003f80u) : 0u;  // bf16 1.0
                    }
                    tmem_st_row<C::KA>(tm_row + C::A_COL0 + g * C::KA, w);
                    tmem_wait_st();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[g]);
            }
            // observation windows 0 and 1 of every chunk
            win_issue(0, 0);
            win_issue(1, 1);

            // The fast path covers the default renormalisation interval for every
            // tensor-core precision; the general path below takes any other.
            const bool fast = (renorm == FAST_R);
            bool bad = false;
            if (fast) {
                // ---- fast path: trips of four steps, renormalisation on the fourth ----
                // TMEM is read and written in the 16x256b fragment, kept as
                // 64-bit pairs of adjacent columns: this thread holds rows
                // 8*rho + g8 (rho = 0..3) of its warp's 32 lanes, columns
                // 8m + 2*qd + {0, 1} (m < NB), so it needs only 2*NB of the KP
                // emission factors of a step, read as 16-byte words from a
                // permuted copy in shared memory; the four threads of a quad
                // share a row and combine their row maxima by two shuffles.
                constexpr int NB = KP / 8;
                constexpr int NP = 4 * NB;  // pairs per thread (both halves)
                const int g8 = lane >> 2, qd = lane & 3;
                int lenw[C::GPW][C::CPW];
#pragma unroll
                for (int u = 0; u < C::GPW; ++u)
#pragma unroll
                    for (int cw = 0; cw < C::CPW; ++cw) lenw[u][cw] = __shfl_sync(0xffffffffu, len[u], cw * KP);
                int ex[C::GPW][4];
                int esum[C::GPW];
                uint32_t gbit[C::GPW];
#pragma unroll
                for (int u = 0; u < C::GPW; ++u) {
                    esum[u] = 0;
                    gbit[u] = 1u << (team + E * u);
#pragma unroll
                    for (int rho = 0; rho < 4; ++rho) ex[u][rho] = 0;
                }
                // this lane's emission factor goes to position pd of its chunk's factors
                const int pd = half * KP + (2 * NB) * ((jl >> 1) & 3) + 2 * (jl >> 3) + (jl & 1);
                // TF32 (one image of P): the tensor core truncates the running
                // product to its top 19 bits; the mean relative loss per step
                // is restored by scaling every step's emissions by 1/(1 - c)
                // (c in hmm_tc_common.cuh). A chunk's first step multiplies the
                // exact identity, so its compensation is taken back when the
                // chunk is written.
                constexpr bool TRUNC = (PREC == HMM_PREC_TF32);
                const float ctr_s = ctr + (TRUNC ? TF32_TRUNC_COMP_LOG2 : 0.0f);
                const float cno_s = cno + (TRUNC ? TF32_TRUNC_COMP_LOG2 : 0.0f);
                const float uncomp = TRUNC ? ex2_approx(-TF32_TRUNC_COMP_LOG2) : 1.0f;
                // smallest finite best-state log2 emission of the live steps
                // (below -EXP_LIMIT is out of range; checked once per item)
                float mlow = 0.0f;
                const float2 *wbase[C::GPW];

                auto step = [&](int t, int rr, auto SPEC) {
                    constexpr bool spec = decltype(SPEC)::value;
                    const int w = t & (C::WIN - 1);
                    int Et[C::GPW];
#pragma unroll
                    for (int u = 0; u < C::GPW; ++u) {
                        // Step 1 fused: log2 emission of this lane's state (Eq.
                        // "emission-matrix"), the chunk's best state, the
                        // power-of-two prescale and the factor D_t
                        const float2 o = wbase[u][w];
                        const float dx = o.x - mux, dy = o.y - muy;
                        const float l2 = fmaf(fmaf(qa, dx, qb * dy), dx, fmaf(qc * dy, dy, ctr_s));
                        const float l = isnan(o.x) ? cno_s : l2;
                        const float m = chunk_max<KP>(l, lane);
                        if (t < len[u] && m > -INFINITY) mlow = fminf(mlow, m);
                        float mf;
                        Et[u] = round_to_int(fmaxf(m, -(float)EXP_LIMIT), mf);
                        sD[u * 32 + pd] = ex2_approx(l - mf);
                        esum[u] += Et[u];
                    }
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < C::GPW; ++u) {
                        const int g = team + E * u;
                        if (!(glive >> u & 1u)) continue;
                        const bool okw =
                            __all_sync(0xffffffffu, mbar_wait(&full[g], (full_par & gbit[u]) ? 1u : 0u, abort_flag, status));
                        full_par ^= gbit[u];
                        if (!okw) {
                            bad = true;
                            return;
                        }
                        tc_fence_after();
                        unsigned long long pr[NP];
                        tmem_ld_pairs<NB>(tm_row + g * KP, tm_row + (16u << 16) + g * KP, pr);
                        // Step 2 fused: column scale by D_t, paired multiplies
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int cw = (KP == 32) ? 0 : h;
                            const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(sD + u * 32 + cw * KP + 2 * NB * qd);
#pragma unroll
                            for (int k = 0; k < NB / 2; ++k) {
                                const ulonglong2 dd = src[k];
#pragma unroll
                                for (int j = 0; j < 2; ++j) {
                                    pr[h * 2 * NB + 4 * k + j] = mul2(pr[h * 2 * NB + 4 * k + j], dd.x);
                                    pr[h * 2 * NB + 4 * k + 2 + j] = mul2(pr[h * 2 * NB + 4 * k + 2 + j], dd.y);
                                }
                            }
                        }
                        // per-row power-of-two renormalisation, and a chunk's final write-out
                        bool fin[4];
#pragma unroll
                        for (int rho = 0; rho < 4; ++rho) fin[rho] = spec && (t + 1 == lenw[u][(KP == 32) ? 0 : (rho >> 1)]);
                        const bool any_rn = (rr == FAST_R - 1) || (spec && (fin[0] || fin[1] || fin[2] || fin[3]));
                        if (any_rn) {
                            int es[C::CPW];
#pragma unroll
                            for (int cw = 0; cw < C::CPW; ++cw) es[cw] = spec ? __shfl_sync(0xffffffffu, esum[u], cw * KP) : 0;
                            bool nonfinite = false;
#pragma unroll
                            for (int rho = 0; rho < 4; ++rho) {
                                const int h = rho >> 1, j = rho & 1;
                                const int cw = (KP == 32) ? 0 : h;
                                float mx = 0.0f;
#pragma unroll
                                for (int mm = 0; mm < NB; ++mm) {
                                    float a0, a1;
                                    unpack2(pr[h * 2 * NB + 2 * mm + j], a0, a1);
                                    mx = max3f(mx, a0, a1);
                                }
                                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
                                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
                                if (!((rr == FAST_R - 1) || fin[rho])) continue;
                                uint32_t eb = __float_as_uint(mx) & 0x7f800000u;
                                nonfinite |= (t < lenw[u][cw]) && eb == 0x7f800000u;
                                eb = min(max(eb, 0x00800000u), 0x7e800000u);  // exponent in [-126, 126]
                                const float sc = __uint_as_float(0x7f000000u - eb);
                                ex[u][rho] += (int)(eb >> 23) - 127;
                                const unsigned long long s2 = pack2(sc, sc);
#pragma unroll
                                for (int mm = 0; mm < NB; ++mm)
                                    pr[h * 2 * NB + 2 * mm + j] = mul2(pr[h * 2 * NB + 2 * mm + j], s2);
                                if (spec && fin[rho]) {
                                    // this row's chunk ends here: write the row and its exponent
                                    const int row = (KP == 32) ? 8 * rho + g8 : 8 * j + g8;
                                    const size_t jj = (size_t)q * n_chunks + (size_t)b * per_item + g * C::CPG +
                                                      quad * C::CPW + cw;
                                    unsigned long long *dst =
                                        reinterpret_cast<unsigned long long *>(A0 + jj * KP * KP + (size_t)row * KP + 2 * qd);
                                    const unsigned long long un = pack2(uncomp, uncomp);
#pragma unroll
                                    for (int mm = 0; mm < NB; ++mm) dst[4 * mm] = mul2(pr[h * 2 * NB + 2 * mm + j], un);
                                    if (qd == 0) e0[jj * KP + row] = (mx > 0.0f) ? ex[u][rho] + es[cw] : ZERO_ROW_EXP32;
                                }
                            }
                            if (nonfinite) atomicOr(status, ST_ENUMERIC);
                        }
                        if (t + 1 < steps) {
                            // next A operand (TF32: the raw FP32 bits, truncated by the
                            // tensor core; TF32-split: rounded to nearest first, both
                            // halves of a pair in one add: values are non-negative, so
                            // the low half never carries; BF16: rounded to nearest and
                            // packed two per column)
                            const uint32_t a0 = tm_row + C::A_COL0 + g * C::KA, a1 = a0 + (16u << 16);
                            if constexpr (PREC == HMM_PREC_BF16) {
                                tmem_st_bf16_pairs<NB>(a0, a1, pr);
                            } else {
                                if constexpr (!TRUNC) {
#pragma unroll
                                    for (int k = 0; k < NP; ++k) pr[k] += 0x0000100000001000ull;
                                }
                                tmem_st_pairs<NB>(a0, a1, pr);
                            }
                            tmem_wait_st();
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (t + 1 < steps && lane == 0) mbar_arrive(&empty[g]);
                    }
                };

                for (int t0 = 0; t0 < steps && !bad; t0 += FAST_R) {
                    const int bsel = (t0 / C::WIN) & 1;
                    if ((t0 & (C::WIN - 1)) == 0) {
                        if (t0 > 0) {
                            // the other buffer (window t0/WIN - 1) is consumed: refill it
                            __syncwarp();
                            win_issue(t0 / C::WIN + 1, bsel ^ 1);
                        }
                        if (!win_wait(bsel)) {
                            bad = true;
                            break;
                        }
#pragma unroll
                        for (int u = 0; u < C::GPW; ++u) wbase[u] = win_ptr(u, bsel);
                    }
                    // a trip in which a chunk of this warp ends, or the item's last
                    // trip, takes the per-row checks; every other trip runs without
                    bool spec = t0 + FAST_R >= steps;
#pragma unroll
                    for (int u = 0; u < C::GPW; ++u)
#pragma unroll
                        for (int cw = 0; cw < C::CPW; ++cw)
                            spec |= (unsigned)(lenw[u][cw] - 1 - t0) < (unsigned)FAST_R;
                    if (!spec) {
#pragma unroll
                        for (int rr = 0; rr < FAST_R; ++rr) {
                            step(t0 + rr, rr, std::integral_constant<bool, false>());
                            if (bad) break;
                        }
                    } else {
                        for (int rr = 0; rr < FAST_R && t0 + rr < steps; ++rr) {
                            step(t0 + rr, rr, std::integral_constant<bool, true>());
                            if (bad) break;
                        }
                    }
                }
                if (mlow < -(float)EXP_LIMIT) atomicOr(status, ST_ENUMERIC);
            }
            int rcount = renorm;
            for (int t = 0; t < steps && !fast; ++t) {
                const bool rn_step = (--rcount == 0);
                if (rn_step) rcount = renorm;
                const int w = t % C::WIN;
                const int bsel = (t / C::WIN) & 1;
                if (w == 0) {
                    if (t > 0) {
                        // refill the buffer that window t/WIN - 1 used with window t/WIN + 1
                        __syncwarp();
                        win_issue(t / C::WIN + 1, bsel ^ 1);
                    }
                    if (!win_wait(bsel)) break;
                }
                // Step 1 fused: emissions of every group's chunk at step t (log2),
                // prescale exponent, D_t into shared memory
                int Et[C::GPW];
#pragma unroll
                for (int u = 0; u < C::GPW; ++u) {
                    const float2 o = win_ptr(u, bsel)[w];
                    float l;
                    if (isnan(o.x)) {
                        l = cno;
                    } else {
                        const float dx = o.x - mux, dy = o.y - muy;
                        l = fmaf(qa * dx, dx, fmaf(qb * dx, dy, fmaf(qc * dy, dy, ctr)));
                    }
                    const float m = chunk_max<KP>(l, lane);
                    float d;
                    Et[u] = 0;
                    if (m >= -(float)EXP_LIMIT) {
                        // prescale by the nearest power of two: the best state's
                        // factor lies in [2^-0.5, 2^0.5]
                        float mf;
                        Et[u] = round_to_int(m, mf);
                        d = ex2_approx(l - mf);
                    } else {
                        if (m != -INFINITY && t < len[u]) atomicOr(status, ST_ENUMERIC);
                        d = 0.0f;
                    }
                    sD[u * 32 + lane] = d;
                }
                __syncwarp();
                // products of this step, group by group
#pragma unroll
                for (int u = 0; u < C::GPW; ++u) {
                    const int g = team + E * u;
                    if (!(glive >> u & 1u)) continue;
                    const bool okw = __all_sync(0xffffffffu, mbar_wait(&full[g], (full_par >> g) & 1u, abort_flag, status));
                    full_par ^= 1u << g;
                    float a[KP];
                    if (okw) {
                        tc_fence_after();
                        tmem_ld_row<KP>(tm_row + g * KP, a);
                        tmem_wait_ld();
                    }
                    if (okw && t < len[u]) {
                        // Step 2 fused: column scale by D_t (pairs)
                        scale_row<KP>(a, sD + u * 32 + half * KP);
                        expo[u] += Et[u];
                        const bool last = (t + 1 == len[u]);
                        if (rn_step || last) {
                            const float mx = renorm_row<KP>(a, expo[u], true, status);
                            if (last) {
                                const size_t jj = (size_t)q * n_chunks + (size_t)b * per_item + (team + E * u) * C::CPG + cs;
                                float4 *dst = reinterpret_cast<float4 *>(A0 + jj * KP * KP + (size_t)i * KP);
#pragma unroll
                                for (int j4 = 0; j4 < KP / 4; ++j4)
                                    dst[j4] = make_float4(a[4 * j4], a[4 * j4 + 1], a[4 * j4 + 2], a[4 * j4 + 3]);
                                e0[jj * KP + i] = (mx > 0.0f) ? expo[u] : ZERO_ROW_EXP32;
                            }
                        }
                    }
                    // next A operand row, rounded to the operand type, into TMEM. The
                    // store is warp-wide: rows whose chunk has ended (or ends now) write
                    // whatever they hold, which only ever feeds their own ignored rows.
                    if (okw && __any_sync(0xffffffffu, t + 1 < len[u])) {
                        uint32_t *w = reinterpret_cast<uint32_t *>(a);  // converted in place
                        if constexpr (C::ESZ == 4) {
#pragma unroll
                            for (int c = 0; c < KP; ++c) w[c] = to_tf32_bits(a[c]);
                        } else {
#pragma unroll
                            for (int c = 0; c < KP / 2; ++c) {
                                __nv_bfloat162 bb = __floats2bfloat162_rn(a[2 * c], a[2 * c + 1]);
                                w[c] = *reinterpret_cast<uint32_t *>(&bb);
                            }
                        }
                        tmem_st_row<C::KA>(tm_row + C::A_COL0 + g * C::KA, w);
                        tmem_wait_st();
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (t + 1 < steps && lane == 0) mbar_arrive(&empty[g]);
                }
            }
            // copies issued but not consumed (a window past the item's last step,
            // or an abort) land before the buffers are reused
            win_drain();
        }
        // a bulk copy that was issued but never consumed must land before exit
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
cudaError_t launch_tc_t(int n_prop, int n_chunks, int renorm, const ConstLayout &lay, const float *cblock,
                        const ChunkDesc *chunks, const float2 *packed, float *A0, int32_t *e0, unsigned *status,
                        cudaStream_t st) {
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
    kern<<<grid, C::THREADS, C::SMEM, st>>>(n_prop, n_chunks, renorm, lay, cblock, chunks, packed, A0, e0, status);
    return cudaGetLastError();
}

// tile configuration per (KP, precision): groups in flight G, epilogue teams E
template <int KP, int PREC>
struct TcTile;
template <> struct TcTile<32, HMM_PREC_TF32> { static constexpr int G = 8, E = 4; };
template <> struct TcTile<32, HMM_PREC_TF32_SPLIT> { static constexpr int G = 8, E = 4; };
template <> struct TcTile<32, HMM_PREC_BF16> { static constexpr int G = 8, E = 4; };
template <> struct TcTile<16, HMM_PREC_TF32> { static constexpr int G = 16, E = 4; };
template <> struct TcTile<16, HMM_PREC_TF32_SPLIT> { static constexpr int G = 16, E = 4; };
template <> struct TcTile<16, HMM_PREC_BF16> { static constexpr int G = 16, E = 4; };

}  // namespace

bool chunk_tc_supported(int K, int precision) {
    if (precision != HMM_PREC_TF32 && precision != HMM_PREC_TF32_SPLIT && precision != HMM_PREC_BF16) return false;
    return K >= 1 && K <= 80;
}

int chunk_tc_chunks_per_item(int KP, int precision) {
    if (KP > 32) return chunk_tc_wide_chunks_per_item(KP, precision);
#define HMM_TC_PER_ITEM(KPV, PRECV) \
    if (KP == KPV && precision == PRECV) return TcTile<KPV, PRECV>::G * (TC_M / KPV);
    HMM_TC_PER_ITEM(16, HMM_PREC_TF32)
    HMM_TC_PER_ITEM(32, HMM_PREC_TF32)
    HMM_TC_PER_ITEM(16, HMM_PREC_TF32_SPLIT)
    HMM_TC_PER_ITEM(32, HMM_PREC_TF32_SPLIT)
    HMM_TC_PER_ITEM(16, HMM_PREC_BF16)
    HMM_TC_PER_ITEM(32, HMM_PREC_BF16)
#undef HMM_TC_PER_ITEM
    return 32;
}

cudaError_t launch_chunk_tc(int n_prop, int n_chunks, int L, int renorm, int precision,
                            const ConstLayout &lay, const float *cblock, const ChunkDesc *chunks,
                            const float2 *packed, float *A0, int32_t *e0, unsigned *status,
                            cudaStream_t st) {
    // the observation windows are bulk copies that need every chunk to start
    // on a 64-step (512-byte) boundary of the packed sequence: chunk lengths
    // are multiples of 64 (segments are laid out on such boundaries)
    if (L <= 0 || L % 64 != 0) return cudaErrorInvalidValue;
    if (n_chunks == 0 || n_prop == 0) return cudaSuccess;
    if (lay.KP > 32)
        return launch_chunk_tc_wide(n_prop, n_chunks, renorm, precision, lay, cblock, chunks, packed, A0, e0,
                                    status, st);
#define HMM_TC_CASE(KPV, PRECV)                                                                              \
    if (lay.KP == KPV && precision == PRECV)                                                                  \
        return launch_tc_t<KPV, PRECV, TcTile<KPV, PRECV>::G, TcTile<KPV, PRECV>::E>(n_prop, n_chunks, renorm, \
                                                                                   lay, cblock, chunks,       \
                                                                                   packed, A0, e0, status, st);
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
