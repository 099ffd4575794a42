// hmm_loglik_noalloc: the single-sequence FP32 likelihood without any device
// allocation.
//
// Some callers cannot allocate device memory while they run: code inside a
// framework that owns every device allocation itself, code whose memory is
// fixed up front (long-running services that must not fragment or grow their
// footprint), or code that must never synchronise the device, which
// cudaMalloc/cudaFree can do. hmm_loglik, by contrast, allocates through its
// context. This entry point runs the same kernels (prep, pack, FP32-SIMT
// chunk products, product tree, FP64 combine) with all of their scratch in
// one file-scope __device__ array of fixed size, allocated when the library
// is loaded and held by every GPU that loads it until the process exits.
//
// The address of that array is looked up once per device (with the device
// current) by cudaGetSymbolAddress; the first call on a device does it, so
// that first call should come before any stream capture. Every call reuses
// the same array and overwrites what the previous call left there; the parts
// that must start at zero are cleared on the call's stream. Calls whose work
// overlaps on the GPU (different streams, or different host threads, without
// ordering between them) race on the array: order them or use hmm_loglik.
//
// Without a context there is no hmm_status() to read the device status word,
// so the call's last kernel reads it on the stream and turns a failed call
// into a NaN result: invalid parameters or flagged observations (already NaN
// from the combine), a value that left the representable range (an emission
// below 2^-65536 of the step's best state, or a non-finite product), or a
// bounded device wait that ran out.
#include <algorithm>
#include <mutex>

#include "hmm_internal.cuh"

namespace hmm {
namespace {

constexpr int NA_KP = 32;        // SIMT padding for K <= 32
constexpr int NA_L = 1024;       // fixed chunk length
constexpr int NA_MAX_DEVICES = 64;

// Layout of the scratch array for the largest allowed problem.
struct NaLayout {
    size_t cblock, flags, packed, head, offs, pbase, chunks, segs, groups, A[4], e[4], total;
    int n_levels;
    int level_n[4];
    int n_groups[3];
};

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

NaLayout na_layout(int64_t T) {
    NaLayout L{};
    const int64_t steps = T > 1 ? T - 1 : 0;
    const int C = (int)((steps + NA_L - 1) / NA_L);
    L.level_n[0] = C;
    L.n_levels = 0;
    int n = C;
    while (n > 1 && L.n_levels < 3) {
        const int ng = (n + TREE_GROUP - 1) / TREE_GROUP;
        L.n_groups[L.n_levels] = ng;
        L.level_n[L.n_levels + 1] = ng;
        n = ng;
        ++L.n_levels;
    }
    size_t o = 0;
    const ConstLayout lay = make_layout(NA_KP, HMM_PREC_FP32_SIMT);
    L.cblock = o; o = al256(o + sizeof(float) * lay.stride);
    L.flags = o;  o = al256(o + 4 * sizeof(int));  // prop_bad, obs_bad, status
    L.packed = o; o = al256(o + sizeof(float2) * (size_t)std::max<int64_t>(OBS_WIN, (steps + OBS_WIN - 1) / OBS_WIN * OBS_WIN));
    L.head = o;   o = al256(o + sizeof(float2));
    L.offs = o;   o = al256(o + 2 * sizeof(int64_t));
    L.pbase = o;  o = al256(o + sizeof(int64_t));
    L.chunks = o; o = al256(o + sizeof(ChunkDesc) * (size_t)std::max(1, C));
    L.segs = o;   o = al256(o + sizeof(SegFinal));
    L.groups = o; o = al256(o + sizeof(TreeGroup) * (size_t)(L.n_groups[0] + L.n_groups[1] + L.n_groups[2] + 3));
    for (int l = 0; l <= L.n_levels; ++l) {
        const size_t m = (size_t)std::max(1, L.level_n[l]);
        L.A[l] = o; o = al256(o + sizeof(float) * m * NA_KP * NA_KP);
        L.e[l] = o; o = al256(o + (l == 0 ? 4 : 8) * m * NA_KP);
    }
    L.total = o;
    return L;
}

}  // namespace

// 12.6 MiB: the layout above at T = HMM_NOALLOC_MAX_T (checked at run time)
constexpr size_t NA_SCRATCH_BYTES = (size_t)13 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

namespace {

std::mutex g_na_mutex;
void *g_na_ptr[NA_MAX_DEVICES] = {};

// Fills the chunk table, the tree groups and the segment record for one
// sequence of T observations (the same plan the context path builds on the
// host, computed here so nothing has to be copied in).
__global__ void noalloc_plan_kernel(int64_t T, int C, int n_levels, int ng0, int ng1, int ng2,
                                    ChunkDesc *chunks, TreeGroup *groups, SegFinal *seg, int64_t *offs,
                                    int64_t *pbase) {
    const int64_t steps = T > 1 ? T - 1 : 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        ChunkDesc d;
        d.pstart = (int64_t)c * NA_L;
        d.len = (int)min((int64_t)NA_L, steps - (int64_t)c * NA_L);
        d.seg = 0;
        chunks[c] = d;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int ng[3] = {ng0, ng1, ng2};
        int n = C, base = 0;
        for (int l = 0; l < n_levels; ++l) {
            for (int g = 0; g < ng[l]; ++g) {
                TreeGroup tg;
                tg.src = g * TREE_GROUP;
                tg.cnt = min(TREE_GROUP, n - g * TREE_GROUP);
                tg.dst = g;
                tg.pad = 0;
                groups[base + g] = tg;
            }
            base += ng[l];
            n = ng[l];
        }
        SegFinal s;
        s.T = T;
        s.level = C >= 1 ? n_levels : -1;
        s.idx = 0;
        *seg = s;
        offs[0] = 0;
        offs[1] = T;
        *pbase = 0;
    }
}

// the status word as the result: any failure bit makes log L NaN
__global__ void noalloc_status_kernel(const unsigned *status, double *out) {
    if (*status & (ST_EINVAL | ST_ENUMERIC | ST_ETIMEOUT)) *out = __longlong_as_double(0x7ff8000000000000LL);
}

}  // namespace
}  // namespace hmm

using namespace hmm;

extern "C" int hmm_loglik_noalloc(const hmm_params *prm, const hmm_obs *obs, double *out_dev,
                                  void *stream) {
    if (!prm || !obs || !out_dev) return HMM_EINVAL;
    const int K = prm->K;
    const int64_t T = obs->T;
    if (K < 1 || K > HMM_NOALLOC_MAX_K) return HMM_EINVAL;
    if (T < 0 || T > HMM_NOALLOC_MAX_T) return HMM_EINVAL;
    if (!prm->pi || !prm->P || !prm->p_tremor || !prm->mu || !prm->cov) return HMM_EINVAL;
    if (T > 0 && (!obs->xy || !obs->tremor)) return HMM_EINVAL;
    if (obs->xy && ((uintptr_t)obs->xy & 7)) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return HMM_ECUDA;
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return HMM_ECUDA;
            }
            g_na_ptr[dev] = p;
        }
        base = static_cast<unsigned char *>(g_na_ptr[dev]);
    }
    const NaLayout L = na_layout(T);
    if (L.total > NA_SCRATCH_BYTES) return HMM_EINVAL;

    const ConstLayout lay = make_layout(K, HMM_PREC_FP32_SIMT);
    float *cblock = reinterpret_cast<float *>(base + L.cblock);
    int *flags = reinterpret_cast<int *>(base + L.flags);
    int *prop_bad = flags, *obs_bad = flags + 1;
    unsigned *status = reinterpret_cast<unsigned *>(flags + 2);
    float2 *packed = reinterpret_cast<float2 *>(base + L.packed);
    float2 *head = reinterpret_cast<float2 *>(base + L.head);
    int64_t *offs = reinterpret_cast<int64_t *>(base + L.offs);
    int64_t *pbase = reinterpret_cast<int64_t *>(base + L.pbase);
    ChunkDesc *chunks = reinterpret_cast<ChunkDesc *>(base + L.chunks);
    SegFinal *segs = reinterpret_cast<SegFinal *>(base + L.segs);
    TreeGroup *groups = reinterpret_cast<TreeGroup *>(base + L.groups);
    LevelPtrs lv{};
    for (int l = 0; l <= L.n_levels; ++l) {
        lv.A[l] = reinterpret_cast<float *>(base + L.A[l]);
        lv.e[l] = base + L.e[l];
        lv.n[l] = L.level_n[l];
    }
    const int C = L.level_n[0];

    // the flags must start at zero; everything else is written before it is read
    e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), st);
    if (e == cudaSuccess) {
        noalloc_plan_kernel<<<std::max(1, std::min(64, (C + 255) / 256)), 256, 0, st>>>(
            T, C, L.n_levels, L.n_groups[0], L.n_groups[1], L.n_groups[2], chunks, groups, segs, offs, pbase);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_prep(1, K, lay, HMM_PREC_FP32_SIMT, 0, prm->pi, prm->P, prm->p_tremor, prm->mu, prm->cov,
                        cblock, prop_bad, status, st);
    if (e == cudaSuccess && T > 0)
        e = launch_pack(1, offs, pbase, T, obs->xy, obs->tremor, packed, head, obs_bad, status, st);
    if (e == cudaSuccess && C > 0)
        e = launch_chunk_simt(1, C, NA_L, 4, lay, cblock, chunks, packed, lv.A[0], (int32_t *)lv.e[0], status, st);
    int gbase = 0;
    for (int l = 0; l < L.n_levels && e == cudaSuccess; ++l) {
        e = launch_tree_level(1, lay.KP, l, L.n_groups[l], groups + gbase, lv, status, st);
        gbase += L.n_groups[l];
    }
    if (e == cudaSuccess)
        e = launch_final(1, K, HMM_INIT_EMIT_FIRST, 1, segs, head, lv, lay.KP, prm->pi, prm->P, prm->p_tremor,
                         prm->mu, prm->cov, prop_bad, obs_bad, out_dev, st);
    if (e == cudaSuccess) {
        noalloc_status_kernel<<<1, 1, 0, st>>>(status, out_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HMM_ECUDA;
    }
    return HMM_OK;
}
