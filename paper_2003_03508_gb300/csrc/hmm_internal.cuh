// Internal declarations shared by the library's translation units.
//
// Data layout in HBM (per call, carved out of one context-owned workspace):
//   cblock  [n_prop][cstride] f32  per-proposal constants written by the prep
//                                  kernel: emission coefficients (log2 domain,
//                                  8 x KP SoA), P padded to KP x KP in FP32,
//                                  and the tensor-core operand images of P.
//   packed  [n_packed] float2      chain observations x_1..x_{T-1} of every
//                                  segment, each segment starting on a
//                                  64-step boundary; x = NaN marks "no tremor".
//   head    [n_seg] float2         first observation x_0 of each segment.
//   chunks  [n_chunks] ChunkDesc   chunk table shared by all proposals.
//   A0/e0   [n_prop][n_chunks]     chunk products (KP x KP f32) and per-row
//                                  int32 power-of-two exponents.
//   A_l/e_l levels of the product tree (int64 exponents).
//   qtab/qexp [n_prop][nb] run-length shortcut table (KP x KP f32 and KP int32
//                                  row exponents per power), only when it is on.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hmm_gb300.h"

namespace hmm {

// device status word bits
enum : unsigned {
    ST_EINVAL = 1u,
    ST_ENUMERIC = 2u,
    ST_ETIMEOUT = 4u,
};

// emission coefficient rows in the const block (each row is KP floats)
enum {
    EM_MUX = 0,
    EM_MUY = 1,
    EM_QA = 2,   // -0.5 log2(e) syy / det
    EM_QB = 3,   //      log2(e) sxy / det
    EM_QC = 4,   // -0.5 log2(e) sxx / det
    EM_CTR = 5,  // log2 p - log2(2 pi) - 0.5 log2 det
    EM_CNO = 6,  // log2 (1 - p)
    EM_ROWS = 8,
};

// a step whose best state has log2-emission below -EXP_LIMIT is not representable
// (keeps a chunk's exponent sum, <= 16384 steps, inside int32)
constexpr int EXP_LIMIT = 1 << 16;
// exponent recorded for an all-zero row (its scale is irrelevant); the tree
// aligns rows to the largest exponent, so zero rows must never win that max
constexpr int32_t ZERO_ROW_EXP32 = INT32_MIN;
constexpr long long ZERO_ROW_EXP64 = -(1LL << 62);
constexpr int MAX_LEVELS = 10;
constexpr int TREE_GROUP = 16;
constexpr int OBS_WIN = 64;   // steps per observation window; chunk lengths are multiples

struct ChunkDesc {
    int64_t pstart;  // index of the chunk's first step in `packed`
    int32_t len;     // steps in this chunk (1..L)
    int32_t seg;     // segment it belongs to
};

struct ConstLayout {
    int KP;         // padded state count used by the chunk kernel
    int off_emis;   // EM_ROWS * KP floats
    int off_p32;    // KP * KP floats, row-major, zero padded
    int off_tc;     // tensor-core B-operand images (path dependent)
    int tc_floats;  // size of the tensor-core section
    int stride;     // floats per proposal (multiple of 32)
};

struct TreeGroup {
    int32_t src;  // first matrix (index within one proposal's level buffer)
    int32_t cnt;  // matrices to multiply, in order
    int32_t dst;  // output index in the next level
    int32_t pad;
};

struct SegFinal {
    int64_t T;      // observations in the segment
    int32_t level;  // level holding the segment's product (-1: no product)
    int32_t idx;    // index within one proposal's slice of that level
};

struct LevelPtrs {
    float *A[MAX_LEVELS];
    void *e[MAX_LEVELS];     // level 0: int32, others: int64
    int32_t n[MAX_LEVELS];   // matrices per proposal at each level
};

// ---------------- small device helpers ----------------

// floor(log2(m)) for a positive normal float, as the exponent field.
__device__ __forceinline__ int float_exponent(float m) {
    return ((__float_as_int(m) >> 23) & 0xff) - 127;
}

// 2^k as a float for k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) {
    return __int_as_float((k + 127) << 23);
}

// log2 of the emission of state k for observation (x, y) (Eq. "emission-matrix").
__device__ __forceinline__ float log2_emission(const float *__restrict__ em, int KP, int k,
                                               float x, float y, bool tremor) {
    if (!tremor) return em[EM_CNO * KP + k];
    float dx = x - em[EM_MUX * KP + k];
    float dy = y - em[EM_MUY * KP + k];
    float acc = em[EM_CTR * KP + k];
    acc = fmaf(em[EM_QC * KP + k] * dy, dy, acc);
    acc = fmaf(em[EM_QB * KP + k] * dx, dy, acc);
    acc = fmaf(em[EM_QA * KP + k] * dx, dx, acc);
    return acc;
}

// ---------------- launchers (host side, one per translation unit) ----------------

ConstLayout make_layout(int K, int precision);

cudaError_t launch_prep(int n_prop, int K, const ConstLayout &lay, int precision, int init_mode,
                        const float *pi, const float *P, const float *p, const float *mu,
                        const float *cov, float *cblock, int *prop_bad, unsigned *status,
                        cudaStream_t st);

cudaError_t launch_pack(int n_seg, const int64_t *d_offsets, const int64_t *d_pbase,
                        int64_t T_total, const float *xy, const uint8_t *tremor, float2 *packed,
                        float2 *head, int *obs_bad, unsigned *status, cudaStream_t st);

cudaError_t launch_chunk_simt(int n_prop, int n_chunks, int L, int renorm, const ConstLayout &lay,
                              const float *cblock, const ChunkDesc *chunks, const float2 *packed,
                              float *A0, int32_t *e0, unsigned *status, cudaStream_t st);

// run-length shortcut (FP32 on the CUDA cores): table of M_0^(2^b), b < nb,
// then chunk products that apply runs of >= min_run no-tremor steps from it
int rle_levels(int L);
cudaError_t launch_rle_table(int n_prop, int nb, const ConstLayout &lay, const float *cblock, float *qtab,
                             int32_t *qexp, unsigned *status, cudaStream_t st);
cudaError_t launch_chunk_rle(int n_prop, int n_chunks, int renorm, int min_run, int nb, const ConstLayout &lay,
                             const float *cblock, const float *qtab, const int32_t *qexp, const ChunkDesc *chunks,
                             const float2 *packed, float *A0, int32_t *e0, unsigned *status, cudaStream_t st);

bool chunk_tc_supported(int K, int precision);
int chunk_tc_chunks_per_item(int KP, int precision);
cudaError_t launch_posterior(int K, int KP, int init_mode, int n_chunks, int L, const ChunkDesc *chunks,
                             const float *pi, const float *P, const float *em, const float2 *head,
                             const float2 *packed, const float *A0, const int32_t *e0, float *fvec, float *bvec,
                             float *gamma, double *stats_part, double *g0, double *stats, cudaStream_t st);
int chunk_tc_wide_chunks_per_item(int KP, int precision);
cudaError_t launch_viterbi(int K, int init_mode, int n_chunks, int L, const ConstLayout &lay, const ChunkDesc *chunks,
                           const float *pi, const float *P, const float *cblock, const float2 *head,
                           const float2 *packed, float *V, double *voff, int32_t *ptr, int32_t *bstate, uint8_t *bp,
                           int32_t *path, double *score, cudaStream_t st);
cudaError_t launch_chunk_tc_wide(int n_prop, int n_chunks, int renorm, int precision, const ConstLayout &lay,
                                 const float *cblock, const ChunkDesc *chunks, const float2 *packed, float *A0,
                                 int32_t *e0, unsigned *status, cudaStream_t st);
cudaError_t launch_chunk_tc(int n_prop, int n_chunks, int L, int renorm, int precision,
                            const ConstLayout &lay, const float *cblock, const ChunkDesc *chunks,
                            const float2 *packed, float *A0, int32_t *e0, unsigned *status,
                            cudaStream_t st);

// Fisher-identity gradient and EM M-step from the E-step statistics (hmm_grad.cu)
cudaError_t launch_fisher_grad(int K, int init_mode, const float *pi, const float *P, const float *p, const float *mu,
                               const float *cov, const double *stats, double *grad, cudaStream_t st);
cudaError_t launch_em_mstep(int K, const float *pi, const float *P, const float *p, const float *mu, const float *cov,
                            const double *stats, float *pi_out, float *P_out, float *p_out, float *mu_out,
                            float *cov_out, cudaStream_t st);

cudaError_t launch_tree_level(int n_prop, int KP, int level, int n_groups, const TreeGroup *groups,
                              const LevelPtrs &lv, unsigned *status, cudaStream_t st);

cudaError_t launch_final(int n_prop, int K, int init_mode, int n_seg, const SegFinal *segs,
                         const float2 *head, const LevelPtrs &lv, int KP, const float *pi,
                         const float *P, const float *p, const float *mu, const float *cov,
                         const int *prop_bad, const int *obs_bad, double *out, cudaStream_t st);

}  // namespace hmm
