// Inline-PTX wrappers shared by the tensor-core chunk kernels: mbarriers with
// bounded waits, tcgen05 (MMA, commit, TMEM loads and stores, fences), shared
// memory descriptors, cp.async, and the small arithmetic helpers of the
// epilogue (TF32 rounding, nearest-integer split, ex2, row renormalisation).
#pragma once

#include <cuda_bf16.h>

#include "hmm_internal.cuh"

namespace hmm {

namespace {

constexpr int TC_M = 128;
constexpr int NISS = 4;  // MMA issuer warps (warps 0..3)
constexpr int FAST_R = 4;  // renormalisation interval of the unrolled fast path
constexpr long long SPIN_LIMIT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz
// A TF32 operand read from FP32 bits keeps the top 10 mantissa bits: the
// dropped part is a fraction U * 2^-10 / m of the value (U uniform in [0, 1),
// m in [1, 2) the mantissa), whose mean over log-uniformly spread mantissas
// is c = 2^-11 * E[1/m] = 2^-11 / (2 ln 2). Multiplying a step's emission
// factors by 1 / (1 - c), i.e. adding -log2(1 - c) to their log2, restores
// the mean loss of the truncated step.
constexpr float TF32_TRUNC_COMP_LOG2 = 5.0823623e-4f;

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

// non-blocking probe of one phase (never suspends the thread)
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
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
                                          unsigned *status, long long limit = SPIN_LIMIT_CYCLES) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            atomicOr(status, ST_ETIMEOUT);
            return false;
        }
    }
}

// 1-D bulk copy (TMA) of `bytes` from global to shared memory, its completion
// counted in bytes on `bar` (both addresses 16-byte aligned, bytes a multiple
// of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Wait for a phase that completes by itself (copies already in flight),
// bounded, whatever the abort flag says: used to let copies land before their
// buffer is reused or the CTA exits.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity) && clock64() - t0 < SPIN_LIMIT_CYCLES) {
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

// D (TMEM) = A (TMEM) x B (shared memory), or D += A x B
template <int PREC>
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    if constexpr (PREC == HMM_PREC_BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
            "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
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

// 32 lanes x 32 columns of 32-bit TMEM data into 32 registers per thread
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// one thread's row of NC consecutive 32-bit TMEM columns (NC = 16 or 32)
template <int NC>
__device__ __forceinline__ void tmem_ld_row(uint32_t taddr, float *v) {
    static_assert(NC == 16 || NC == 32, "row width");
    if constexpr (NC == 32) tmem_ld32(taddr, v);
    else tmem_ld16(taddr, v);
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 registers per thread into 32 lanes x 16 columns of TMEM
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// one thread's row of NC consecutive 32-bit TMEM columns (NC = 8, 16 or 32)
template <int NC>
__device__ __forceinline__ void tmem_st_row(uint32_t taddr, const uint32_t *r) {
    static_assert(NC == 8 || NC == 16 || NC == 32, "row width");
    if constexpr (NC == 8) tmem_st8(taddr, r);
    else if constexpr (NC == 16) tmem_st16(taddr, r);
    else tmem_st32(taddr, r);
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---- 16x256b access: 16 TMEM lanes x 8 32-bit columns per repetition ----
// Thread t of the warp holds, for repetition m (columns 8m .. 8m+7 from the
// address's column), registers 4m+0/1 = lane (t/4), columns 8m + 2(t%4) + 0/1
// and registers 4m+2/3 = lane (t/4 + 8), the same columns. A row of 8 columns
// is therefore spread over the four threads of a quad, and each thread needs
// only 2 of every 8 column factors.
template <int NB>
__device__ __forceinline__ void tmem_ld_16x256b(uint32_t taddr, float *v) {
    static_assert(NB == 2 || NB == 4, "16x256b repetitions");
    uint32_t r[4 * NB];
    if constexpr (NB == 4) {
        asm volatile(
            "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
              "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    } else {
        asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7])
                     : "r"(taddr));
    }
#pragma unroll
    for (int i = 0; i < 4 * NB; ++i) v[i] = __uint_as_float(r[i]);
}

template <int NB>
__device__ __forceinline__ void tmem_st_16x256b(uint32_t taddr, const uint32_t *r) {
    static_assert(NB == 2 || NB == 4, "16x256b repetitions");
    if constexpr (NB == 4) {
        asm volatile(
            "tcgen05.st.sync.aligned.16x256b.x4.b32 [%0], "
            "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
            "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
            "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
            : "memory");
    } else {
        asm volatile("tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                     "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                     : "memory");
    }
}

// Both 16-lane halves of a warp's quadrant in the 16x256b fragment (t0: lanes
// 0-15, t1: lanes 16-31 of the quadrant), as 64-bit pairs of adjacent columns:
// pair h*2NB + 2m + j holds registers 4m + 2j and 4m + 2j + 1 of half h, i.e.
// row 8j + lane/4 (+16h), columns 8m + 2(lane%4) + {0, 1}. Keeping the data in
// pairs from the load, through the paired multiplies, to the store lets the
// register allocator keep each pair in place. The load waits for completion.
template <int NB>
__device__ __forceinline__ void tmem_ld_pairs(uint32_t t0, uint32_t t1, unsigned long long *p);
template <int NB>
__device__ __forceinline__ void tmem_st_pairs(uint32_t t0, uint32_t t1, const unsigned long long *p);

template <>
__device__ __forceinline__ void tmem_ld_pairs<4>(uint32_t t0, uint32_t t1, unsigned long long *p) {
    asm volatile("{\n\t.reg .b32 r<32>;\n\t"
                 "tcgen05.ld.sync.aligned.16x256b.x4.b32 {r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15}, [%16];\n\t"
                 "tcgen05.ld.sync.aligned.16x256b.x4.b32 {r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31}, [%17];\n\t"
                 "tcgen05.wait::ld.sync.aligned;\n\t"
                 "mov.b64 %0, {r0, r1};\n\t"
                 "mov.b64 %1, {r2, r3};\n\t"
                 "mov.b64 %2, {r4, r5};\n\t"
                 "mov.b64 %3, {r6, r7};\n\t"
                 "mov.b64 %4, {r8, r9};\n\t"
                 "mov.b64 %5, {r10, r11};\n\t"
                 "mov.b64 %6, {r12, r13};\n\t"
                 "mov.b64 %7, {r14, r15};\n\t"
                 "mov.b64 %8, {r16, r17};\n\t"
                 "mov.b64 %9, {r18, r19};\n\t"
                 "mov.b64 %10, {r20, r21};\n\t"
                 "mov.b64 %11, {r22, r23};\n\t"
                 "mov.b64 %12, {r24, r25};\n\t"
                 "mov.b64 %13, {r26, r27};\n\t"
                 "mov.b64 %14, {r28, r29};\n\t"
                 "mov.b64 %15, {r30, r31};\n\t"
                 "}"
                 : "=l"(p[0]), "=l"(p[1]), "=l"(p[2]), "=l"(p[3]), "=l"(p[4]), "=l"(p[5]), "=l"(p[6]), "=l"(p[7]), "=l"(p[8]), "=l"(p[9]), "=l"(p[10]), "=l"(p[11]), "=l"(p[12]), "=l"(p[13]), "=l"(p[14]), "=l"(p[15])
                 : "r"(t0), "r"(t1) : "memory");
}

template <>
__device__ __forceinline__ void tmem_ld_pairs<2>(uint32_t t0, uint32_t t1, unsigned long long *p) {
    asm volatile("{\n\t.reg .b32 r<16>;\n\t"
                 "tcgen05.ld.sync.aligned.16x256b.x2.b32 {r0,r1,r2,r3,r4,r5,r6,r7}, [%8];\n\t"
                 "tcgen05.ld.sync.aligned.16x256b.x2.b32 {r8,r9,r10,r11,r12,r13,r14,r15}, [%9];\n\t"
                 "tcgen05.wait::ld.sync.aligned;\n\t"
                 "mov.b64 %0, {r0, r1};\n\t"
                 "mov.b64 %1, {r2, r3};\n\t"
                 "mov.b64 %2, {r4, r5};\n\t"
                 "mov.b64 %3, {r6, r7};\n\t"
                 "mov.b64 %4, {r8, r9};\n\t"
                 "mov.b64 %5, {r10, r11};\n\t"
                 "mov.b64 %6, {r12, r13};\n\t"
                 "mov.b64 %7, {r14, r15};\n\t"
                 "}"
                 : "=l"(p[0]), "=l"(p[1]), "=l"(p[2]), "=l"(p[3]), "=l"(p[4]), "=l"(p[5]), "=l"(p[6]), "=l"(p[7])
                 : "r"(t0), "r"(t1) : "memory");
}

template <>
__device__ __forceinline__ void tmem_st_pairs<4>(uint32_t t0, uint32_t t1, const unsigned long long *p) {
    asm volatile("{\n\t.reg .b32 r<32>;\n\t"
                 "mov.b64 {r0, r1}, %2;\n\t"
                 "mov.b64 {r2, r3}, %3;\n\t"
                 "mov.b64 {r4, r5}, %4;\n\t"
                 "mov.b64 {r6, r7}, %5;\n\t"
                 "mov.b64 {r8, r9}, %6;\n\t"
                 "mov.b64 {r10, r11}, %7;\n\t"
                 "mov.b64 {r12, r13}, %8;\n\t"
                 "mov.b64 {r14, r15}, %9;\n\t"
                 "mov.b64 {r16, r17}, %10;\n\t"
                 "mov.b64 {r18, r19}, %11;\n\t"
                 "mov.b64 {r20, r21}, %12;\n\t"
                 "mov.b64 {r22, r23}, %13;\n\t"
                 "mov.b64 {r24, r25}, %14;\n\t"
                 "mov.b64 {r26, r27}, %15;\n\t"
                 "mov.b64 {r28, r29}, %16;\n\t"
                 "mov.b64 {r30, r31}, %17;\n\t"
                 "tcgen05.st.sync.aligned.16x256b.x4.b32 [%0], {r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15};\n\t"
                 "tcgen05.st.sync.aligned.16x256b.x4.b32 [%1], {r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31};\n\t"
                 "}"
                 :: "r"(t0), "r"(t1), "l"(p[0]), "l"(p[1]), "l"(p[2]), "l"(p[3]), "l"(p[4]), "l"(p[5]), "l"(p[6]), "l"(p[7]), "l"(p[8]), "l"(p[9]), "l"(p[10]), "l"(p[11]), "l"(p[12]), "l"(p[13]), "l"(p[14]), "l"(p[15]) : "memory");
}

template <>
__device__ __forceinline__ void tmem_st_pairs<2>(uint32_t t0, uint32_t t1, const unsigned long long *p) {
    asm volatile("{\n\t.reg .b32 r<16>;\n\t"
                 "mov.b64 {r0, r1}, %2;\n\t"
                 "mov.b64 {r2, r3}, %3;\n\t"
                 "mov.b64 {r4, r5}, %4;\n\t"
                 "mov.b64 {r6, r7}, %5;\n\t"
                 "mov.b64 {r8, r9}, %6;\n\t"
                 "mov.b64 {r10, r11}, %7;\n\t"
                 "mov.b64 {r12, r13}, %8;\n\t"
                 "mov.b64 {r14, r15}, %9;\n\t"
                 "tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {r0,r1,r2,r3,r4,r5,r6,r7};\n\t"
                 "tcgen05.st.sync.aligned.16x256b.x2.b32 [%1], {r8,r9,r10,r11,r12,r13,r14,r15};\n\t"
                 "}"
                 :: "r"(t0), "r"(t1), "l"(p[0]), "l"(p[1]), "l"(p[2]), "l"(p[3]), "l"(p[4]), "l"(p[5]), "l"(p[6]), "l"(p[7]) : "memory");
}

// All MMAs of one group-step (NIMG images of P x NKS slices of K), the first
// overwriting D, the rest accumulating; B descriptors precomputed.
template <int PREC, int NIMG, int NKS>
__device__ __forceinline__ void mma_group(uint32_t d_tmem, uint32_t a_tmem, const uint64_t *bd, uint32_t idesc) {
#pragma unroll
    for (int img = 0; img < NIMG; ++img)
#pragma unroll
        for (int ks = 0; ks < NKS; ++ks) mma_ts<PREC>(d_tmem, a_tmem + ks * 8, bd[img * NKS + ks], idesc, (img | ks) != 0);
}


// FP32 -> TF32 operand, round to nearest with ties away from zero: add half a
// TF32 unit in the last place to the bit pattern (integer pipe; overflow
// rounds to infinity as it should). The tensor core reads a TF32 operand from
// the top 19 bits and ignores the 13 low bits, so they need not be cleared;
// the parity tests pin this (identical results with and without the mask).
__device__ __forceinline__ uint32_t to_tf32_bits(float x) {
    return __float_as_uint(x) + 0x1000u;
}

// nearest integer to m (|m| < 2^22) and the same value as a float, without
// the conversion pipe: add and subtract 1.5 * 2^23
__device__ __forceinline__ int round_to_int(float m, float &mf) {
    const float magic = 12582912.0f;
    const float t = __fadd_rn(m, magic);
    mf = __fsub_rn(t, magic);
    return __float_as_int(t) - 0x4B400000;
}

// 2^x on the special-function unit (FTZ: results below 2^-126 flush to 0)
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
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

// packed FP32 pair helpers (sm_100+ f32x2 arithmetic)
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// The same pairs rounded to BF16 and stored as the BF16 A operand (two
// K-adjacent elements per 32-bit TMEM column, the even one in the low half):
// pair h*2NB + 2m + j (row 8j + lane/4 + 16h, columns 8m + 2(lane%4) + {0, 1})
// becomes the word at column 4m + lane%4 of that row, which is register
// 2m + j of the 16x128b fragment (thread t: lane t/4 and t/4 + 8, column t%4
// of each 4-column repetition).
template <int NB>
__device__ __forceinline__ void tmem_st_bf16_pairs(uint32_t t0, uint32_t t1, const unsigned long long *p) {
    static_assert(NB == 2 || NB == 4, "16x128b repetitions");
    uint32_t w[4 * NB];
#pragma unroll
    for (int k = 0; k < 4 * NB; ++k) {
        float a0, a1;
        unpack2(p[k], a0, a1);
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w[k]) : "f"(a1), "f"(a0));
    }
    if constexpr (NB == 4) {
        asm volatile("tcgen05.st.sync.aligned.16x128b.x4.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(t0), "r"(w[0]),
                     "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                     : "memory");
        asm volatile("tcgen05.st.sync.aligned.16x128b.x4.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(t1), "r"(w[8]),
                     "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
                     : "memory");
    } else {
        asm volatile("tcgen05.st.sync.aligned.16x128b.x2.b32 [%0], {%1,%2,%3,%4};" ::"r"(t0), "r"(w[0]), "r"(w[1]),
                     "r"(w[2]), "r"(w[3])
                     : "memory");
        asm volatile("tcgen05.st.sync.aligned.16x128b.x2.b32 [%0], {%1,%2,%3,%4};" ::"r"(t1), "r"(w[4]), "r"(w[5]),
                     "r"(w[6]), "r"(w[7])
                     : "memory");
    }
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// maximum over the KP lanes of each chunk (KP = 32: whole warp, KP = 16: halves)
template <int KP>
__device__ __forceinline__ float chunk_max(float v, int lane) {
    if constexpr (KP == 32) {
        float m;
        asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(m) : "f"(v));
        return m;
    } else {
        float lo = lane < 16 ? v : -INFINITY, hi = lane < 16 ? -INFINITY : v, m0, m1;
        asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(m0) : "f"(lo));
        asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(m1) : "f"(hi));
        return lane < 16 ? m0 : m1;
    }
}

// Per-row power-of-two renormalisation of one row of KP values: the row
// maximum is brought into [1, 2) and its exponent added to `expo`. Returns
// the maximum before scaling (0 for an all-zero row). A non-finite maximum
// of a live row raises ENUMERIC.
template <int KP>
__device__ __forceinline__ float renorm_row(float *a, int &expo, bool live, unsigned *status) {
    float m4[KP / 4];
#pragma unroll
    for (int j = 0; j < KP / 4; ++j) m4[j] = max3f(max3f(a[4 * j], a[4 * j + 1], a[4 * j + 2]), a[4 * j + 3], 0.0f);
#pragma unroll
    for (int s = KP / 8; s > 0; s >>= 1)
#pragma unroll
        for (int j = 0; j < s; ++j) m4[j] = fmaxf(m4[j], m4[j + s]);
    const float mx = m4[0];
    if (mx > 0.0f) {
        if (!isfinite(mx) && live) atomicOr(status, ST_ENUMERIC);
        int rr = float_exponent(mx);
        rr = rr < -126 ? -126 : (rr > 126 ? 126 : rr);
        const unsigned long long s2 = pack2(pow2f(-rr), pow2f(-rr));
#pragma unroll
        for (int j = 0; j < KP / 2; ++j) {
            unsigned long long pp = mul2(pack2(a[2 * j], a[2 * j + 1]), s2);
            unpack2(pp, a[2 * j], a[2 * j + 1]);
        }
        expo += rr;
    }
    return mx;
}

// column scale of one row by the step's emission factors (KP values in shared
// memory). Scalar multiplies: they issue to both FP32 pipes, where the paired
// f32x2 form measured slower here.
template <int KP>
__device__ __forceinline__ void scale_row(float *a, const float *d) {
    const float4 *dv = reinterpret_cast<const float4 *>(d);
#pragma unroll
    for (int j4 = 0; j4 < KP / 4; ++j4) {
        const float4 dd = dv[j4];
        a[4 * j4] *= dd.x;
        a[4 * j4 + 1] *= dd.y;
        a[4 * j4 + 2] *= dd.z;
        a[4 * j4 + 3] *= dd.w;
    }
}

}  // namespace

}  // namespace hmm
