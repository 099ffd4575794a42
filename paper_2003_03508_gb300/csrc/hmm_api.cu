// C ABI: context, workspace, planning and the launch sequence.
//
// One call of hmm_loglik_batched is (Section "The likelihood algorithm"):
//   prep   -> per-proposal constants (and parameter checks)
//   pack   -> observations into 64-step aligned windows
//   chunk  -> every chunk's product of P D_t (steps 1-3, fused)
//   tree   -> ordered products of the chunk products, level by level
//   final  -> head vector pi0 D_0 times the product, log L in FP64, summed
//             over segments in order
// Every launch goes to the caller's stream; nothing synchronises unless the
// caller asks (hmm_status, or the _host entry point).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "hmm_internal.cuh"

using namespace hmm;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct Plan {
    bool valid = false;
    int K = 0, n_prop = 0, n_seg = 0, precision = -1, L = 0;
    std::vector<int64_t> offsets;
    // derived
    ConstLayout lay{};
    int64_t n_packed = 0;
    int n_chunks = 0;
    int n_levels = 0;  // number of tree levels that run (level l -> l+1)
    std::vector<int32_t> level_n;           // matrices per proposal at each level
    std::vector<std::vector<TreeGroup>> groups;
    std::vector<SegFinal> segfinal;
    std::vector<int64_t> pbase;
    std::vector<ChunkDesc> chunks;
    // device copies (inside plan_buf)
    ChunkDesc *d_chunks = nullptr;
    TreeGroup *d_groups[MAX_LEVELS] = {};
    SegFinal *d_segs = nullptr;
    int64_t *d_offsets = nullptr;
    int64_t *d_pbase = nullptr;
};

}  // namespace

struct hmm_ctx {
    int device = 0;
    char err[512] = {0};
    DevBuf work;       // per-call workspace
    DevBuf planbuf;    // plan tables
    DevBuf stage;      // staging area for the _host entry point
    DevBuf fb;         // boundary vectors (and partial statistics) of hmm_posterior
    DevBuf gam;        // posterior vectors of hmm_expected_stats
    DevBuf stats;      // E-step statistics of hmm_loglik_grad / hmm_em_step
    unsigned *d_status = nullptr;
    Plan plan;
    int last_launches = 0;
    int last_L = 0;
    int n_sms = 0;
    // phase timing
    bool prof_on = false;
    bool prof_pending = false;
    cudaEvent_t ev[HMM_PHASE_COUNT + 1] = {};
    double prof_ms[HMM_PHASE_COUNT] = {};
    int prof_calls = 0;
    // the batched call's launch sequence as an instantiated CUDA graph
    bool graphs_on = true;
    cudaStream_t cap_stream = nullptr;  // captures run here: the legacy default stream cannot be captured
    cudaGraphExec_t call_exec = nullptr;
    std::vector<uint64_t> call_key;     // what the graph's launches depend on
    std::vector<uint64_t> seen_key;     // the previous direct call's (a repeat is captured)
    int call_launches = 0;
    int last_graph = 0;                 // 0 direct, 1 captured and launched, 2 replayed
    uint64_t plan_version = 0;          // advances whenever the plan tables are uploaded
};

static void drop_call_graph(hmm_ctx *c) {
    if (c->call_exec) cudaGraphExecDestroy(c->call_exec);
    c->call_exec = nullptr;
    c->call_key.clear();
    c->seen_key.clear();
}

// fold the events of the previous recorded call into the totals
static void prof_collect(hmm_ctx *c) {
    if (!c->prof_pending) return;
    cudaEventSynchronize(c->ev[HMM_PHASE_COUNT]);
    for (int i = 0; i < HMM_PHASE_COUNT; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]) == cudaSuccess) c->prof_ms[i] += ms;
    }
    cudaGetLastError();
    c->prof_calls += 1;
    c->prof_pending = false;
}

static void prof_mark(hmm_ctx *c, int i, cudaStream_t st) {
    if (c->prof_on) cudaEventRecord(c->ev[i], st);
}

static int fail(hmm_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

static int cuda_fail(hmm_ctx *c, cudaError_t e, const char *what) {
    return fail(c, HMM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static int ensure(hmm_ctx *c, DevBuf &b, size_t bytes) {
    if (b.cap >= bytes) return HMM_OK;
    if (b.p) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaDeviceSynchronize");
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = bytes + bytes / 8 + 4096;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(c, HMM_ENOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    b.cap = want;
    return HMM_OK;
}

// simple bump carve of an existing buffer
struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base((char *)b) {}
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T *r = (T *)(base + off);
        off += n * sizeof(T);
        return r;
    }
};

static int choose_chunk_len(int precision, int n_prop, int KP, int64_t steps_total, int n_sms) {
    if (precision != HMM_PREC_FP32_SIMT) {
        // persistent tensor-core kernel: one work item = chunks_per_item chunks of
        // one proposal on one SM; minimise the critical path, waves x (chunk
        // length + per-item start-up, about 64 steps), plus the product tree
        // (one K^3 product per chunk, about 1/16 of a chunk step per chunk on
        // the whole GPU), preferring longer chunks on ties
        const int per_item = chunk_tc_chunks_per_item(KP, precision);
        int64_t best_cost = INT64_MAX;
        int best_L = OBS_WIN;
        for (int L = OBS_WIN; L <= 16384; L += OBS_WIN) {
            int64_t C = (steps_total + L - 1) / L;
            if (C < 1) C = 1;
            int64_t items = (int64_t)n_prop * ((C + per_item - 1) / per_item);
            int64_t waves = (items + n_sms - 1) / n_sms;
            int64_t cost = waves * (L + 64) + (int64_t)n_prop * C / (16 * n_sms);
            if (cost <= best_cost) {
                best_cost = cost;
                best_L = L;
            }
            if (C == 1) break;
        }
        return best_L;
    }
    // enough independent rows to fill the GPU a few times over, chunk length
    // a multiple of the 64-step observation window
    double rows_target = (double)n_sms * 2048.0;
    double chunks_target = rows_target / ((double)n_prop * KP);
    if (chunks_target < 1.0) chunks_target = 1.0;
    double L = (double)steps_total / chunks_target;
    int64_t Li = ((int64_t)L + 63) / 64 * 64;
    if (Li < 64) Li = 64;
    if (Li > 16384) Li = 16384;
    return (int)Li;
}

// ---- chunk-length tuning ----
//
// The tuner measures a handful of chunk lengths around the cost model's
// choice and remembers the fastest per shape. The tile shapes are fixed by
// the hardware mapping (M = 128 TMEM lanes, N = the padded state count), so
// the chunk length is the schedule's free parameter: it sets the number of
// work items, the waves the GPU runs them in, and the size of the tree.

constexpr int TUNE_L_MAX = 16384;
constexpr int TUNE_MAX_CANDIDATES = 16;

static int round_to_win(double L) {
    int64_t r = (int64_t)(L / OBS_WIN + 0.5) * OBS_WIN;
    return (int)std::min<int64_t>(TUNE_L_MAX, std::max<int64_t>(OBS_WIN, r));
}

// waves of the persistent tensor-core kernel at chunk length L
static int64_t tc_waves(int per_item, int n_prop, int64_t steps_total, int L, int n_sms) {
    int64_t C = std::max<int64_t>(1, (steps_total + L - 1) / L);
    int64_t items = (int64_t)n_prop * ((C + per_item - 1) / per_item);
    return (items + n_sms - 1) / n_sms;
}

// Candidate chunk lengths: the cost model's choice, its neighbours at factors
// 2^(j/2) (j = -3..3) and, on the tensor-core path, the shortest chunk length
// that fits each wave count next to the model's. Ascending, distinct, multiples
// of OBS_WIN in [OBS_WIN, min(16384, steps rounded up)].
static std::vector<int> tune_candidates(int precision, int n_prop, int K, int64_t steps_total, int n_sms) {
    const ConstLayout lay = make_layout(K, precision);
    const int L0 = choose_chunk_len(precision, n_prop, lay.KP, steps_total, n_sms);
    const int64_t Lcap = std::min<int64_t>(
        TUNE_L_MAX, std::max<int64_t>(OBS_WIN, (steps_total + OBS_WIN - 1) / OBS_WIN * OBS_WIN));
    std::vector<int> c;
    auto add = [&](int L) { c.push_back((int)std::min<int64_t>(Lcap, L)); };
    add(L0);
    for (int j = -3; j <= 3; ++j)
        if (j) add(round_to_win(L0 * std::pow(2.0, 0.5 * j)));
    if (precision != HMM_PREC_FP32_SIMT) {
        const int per_item = chunk_tc_chunks_per_item(lay.KP, precision);
        const int64_t w0 = tc_waves(per_item, n_prop, steps_total, L0, n_sms);
        for (int64_t w = std::max<int64_t>(1, w0 - 2); w <= w0 + 2; ++w) {
            for (int L = OBS_WIN; L <= Lcap; L += OBS_WIN) {
                if (tc_waves(per_item, n_prop, steps_total, L, n_sms) <= w) {
                    add(L);
                    break;
                }
            }
        }
    }
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    if ((int)c.size() > TUNE_MAX_CANDIDATES) {
        // keep the ones nearest the model's choice (in log distance)
        std::stable_sort(c.begin(), c.end(), [&](int a, int b) {
            return std::fabs(std::log((double)a / L0)) < std::fabs(std::log((double)b / L0));
        });
        c.resize(TUNE_MAX_CANDIDATES);
        std::sort(c.begin(), c.end());
    }
    return c;
}

struct TuneKey {
    int32_t n_sms, K, precision, n_prop, n_seg, runlen_min;
    int64_t steps;
    bool operator==(const TuneKey &o) const {
        return n_sms == o.n_sms && K == o.K && precision == o.precision && n_prop == o.n_prop &&
               n_seg == o.n_seg && runlen_min == o.runlen_min && steps == o.steps;
    }
};

struct TuneEntry {
    TuneKey key;
    int32_t L;
    double ms;
};

// process-wide table of tuned chunk lengths
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;

static int tune_get(const TuneKey &k) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry &t : g_tune)
        if (t.key == k) return t.L;
    return 0;
}

static void tune_put_locked(const TuneEntry &e) {
    for (TuneEntry &t : g_tune)
        if (t.key == e.key) {
            t = e;
            return;
        }
    g_tune.push_back(e);
}

static bool tune_entry_valid(const TuneEntry &e) {
    const TuneKey &k = e.key;
    const bool prec_ok = k.precision == HMM_PREC_FP32_SIMT || k.precision == HMM_PREC_TF32 ||
                         k.precision == HMM_PREC_BF16 || k.precision == HMM_PREC_TF32_SPLIT;
    return k.n_sms > 0 && k.K >= 1 && k.K <= 80 && prec_ok && k.n_prop >= 1 && k.n_seg >= 1 &&
           k.runlen_min >= 0 && k.runlen_min <= 16384 && k.steps >= 0 && e.L >= OBS_WIN &&
           e.L <= TUNE_L_MAX && e.L % OBS_WIN == 0 && e.ms >= 0.0;
}

static void build_plan(Plan &pl, int K, int n_prop, int n_seg, const int64_t *offs, int precision,
                       int L) {
    pl.K = K;
    pl.n_prop = n_prop;
    pl.n_seg = n_seg;
    pl.precision = precision;
    pl.L = L;
    pl.offsets.assign(offs, offs + n_seg + 1);
    pl.lay = make_layout(K, precision);
    pl.pbase.assign(n_seg, 0);
    pl.chunks.clear();
    std::vector<int> C(n_seg), first(n_seg);
    int64_t pb = 0;
    for (int s = 0; s < n_seg; ++s) {
        int64_t T = offs[s + 1] - offs[s];
        int64_t steps = T > 1 ? T - 1 : 0;
        pl.pbase[s] = pb;
        pb += (steps + OBS_WIN - 1) / OBS_WIN * OBS_WIN;
        C[s] = (int)((steps + L - 1) / L);
        first[s] = (int)pl.chunks.size();
        for (int c = 0; c < C[s]; ++c) {
            ChunkDesc d;
            d.pstart = pl.pbase[s] + (int64_t)c * L;
            d.len = (int)std::min<int64_t>(L, steps - (int64_t)c * L);
            d.seg = s;
            pl.chunks.push_back(d);
        }
    }
    pl.n_packed = pb > 0 ? pb : OBS_WIN;
    pl.n_chunks = (int)pl.chunks.size();
    // tree levels
    pl.level_n.assign(1, pl.n_chunks);
    pl.groups.clear();
    pl.segfinal.assign(n_seg, SegFinal{});
    std::vector<int> cnt(C), base(first);
    for (int s = 0; s < n_seg; ++s) {
        pl.segfinal[s].T = offs[s + 1] - offs[s];
        pl.segfinal[s].level = cnt[s] >= 1 ? 0 : -1;
        pl.segfinal[s].idx = base[s];
    }
    int level = 0;
    for (;;) {
        bool any = false;
        for (int s = 0; s < n_seg; ++s) any = any || cnt[s] > 1;
        if (!any) break;
        std::vector<TreeGroup> gs;
        int nout = 0;
        for (int s = 0; s < n_seg; ++s) {
            if (cnt[s] <= 1) continue;
            int ng = (cnt[s] + TREE_GROUP - 1) / TREE_GROUP;
            for (int g = 0; g < ng; ++g) {
                TreeGroup tg;
                tg.src = base[s] + g * TREE_GROUP;
                tg.cnt = std::min(TREE_GROUP, cnt[s] - g * TREE_GROUP);
                tg.dst = nout + g;
                tg.pad = 0;
                gs.push_back(tg);
            }
            base[s] = nout;
            cnt[s] = ng;
            nout += ng;
            pl.segfinal[s].level = level + 1;
            pl.segfinal[s].idx = base[s];
        }
        pl.groups.push_back(gs);
        pl.level_n.push_back(nout);
        ++level;
    }
    pl.n_levels = level;
    pl.valid = true;
}

static bool plan_matches(const Plan &pl, int K, int n_prop, int n_seg, const int64_t *offs,
                         int precision, int L) {
    if (!pl.valid || pl.K != K || pl.n_prop != n_prop || pl.n_seg != n_seg ||
        pl.precision != precision || pl.L != L)
        return false;
    return std::equal(pl.offsets.begin(), pl.offsets.end(), offs);
}

static int upload_plan(hmm_ctx *c, cudaStream_t st) {
    ++c->plan_version;
    Plan &pl = c->plan;
    size_t bytes = 0;
    auto add = [&](size_t b) { bytes += (b + 255) & ~(size_t)255; };
    add(sizeof(ChunkDesc) * std::max<size_t>(1, pl.chunks.size()));
    for (auto &g : pl.groups) add(sizeof(TreeGroup) * std::max<size_t>(1, g.size()));
    add(sizeof(SegFinal) * pl.segfinal.size());
    add(sizeof(int64_t) * pl.offsets.size());
    add(sizeof(int64_t) * pl.pbase.size());
    int rc = ensure(c, c->planbuf, bytes + 4096);
    if (rc) return rc;
    Carve cv(c->planbuf.p);
    pl.d_chunks = cv.take<ChunkDesc>(std::max<size_t>(1, pl.chunks.size()));
    for (int l = 0; l < pl.n_levels; ++l) pl.d_groups[l] = cv.take<TreeGroup>(std::max<size_t>(1, pl.groups[l].size()));
    pl.d_segs = cv.take<SegFinal>(pl.segfinal.size());
    pl.d_offsets = cv.take<int64_t>(pl.offsets.size());
    pl.d_pbase = cv.take<int64_t>(pl.pbase.size());
    cudaError_t e = cudaSuccess;
    if (!pl.chunks.empty())
        e = cudaMemcpyAsync(pl.d_chunks, pl.chunks.data(), sizeof(ChunkDesc) * pl.chunks.size(), cudaMemcpyHostToDevice, st);
    for (int l = 0; l < pl.n_levels && e == cudaSuccess; ++l)
        e = cudaMemcpyAsync(pl.d_groups[l], pl.groups[l].data(), sizeof(TreeGroup) * pl.groups[l].size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl.d_segs, pl.segfinal.data(), sizeof(SegFinal) * pl.segfinal.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl.d_offsets, pl.offsets.data(), sizeof(int64_t) * pl.offsets.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl.d_pbase, pl.pbase.data(), sizeof(int64_t) * pl.pbase.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors may change after return
    if (e != cudaSuccess) {
        pl.valid = false;
        return cuda_fail(c, e, "plan upload");
    }
    return HMM_OK;
}

extern "C" {

void hmm_opts_default(hmm_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = HMM_PREC_FP32_SIMT;
    o->init_mode = HMM_INIT_EMIT_FIRST;
    o->chunk_len = 0;
    o->renorm_every = 0;
}

int hmm_create(hmm_ctx **out, int device) {
    if (!out) return HMM_EINVAL;
    *out = nullptr;
    hmm_ctx *c = new (std::nothrow) hmm_ctx();
    if (!c) return HMM_ENOMEM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        int rc = e == cudaErrorMemoryAllocation ? HMM_ENOMEM : HMM_ECUDA;
        cudaGetLastError();
        delete c;
        return rc;
    }
    *out = c;
    return HMM_OK;
}

int hmm_destroy(hmm_ctx *c) {
    if (!c) return HMM_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->work.p) cudaFree(c->work.p);
    if (c->planbuf.p) cudaFree(c->planbuf.p);
    if (c->stage.p) cudaFree(c->stage.p);
    if (c->fb.p) cudaFree(c->fb.p);
    if (c->gam.p) cudaFree(c->gam.p);
    if (c->stats.p) cudaFree(c->stats.p);
    if (c->d_status) cudaFree(c->d_status);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    drop_call_graph(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return HMM_OK;
}

const char *hmm_last_error(const hmm_ctx *c) { return c ? c->err : "null context"; }

int hmm_last_launch_count(const hmm_ctx *c) { return c ? c->last_launches : -1; }

int hmm_last_chunk_len(const hmm_ctx *c) { return c ? c->last_L : -1; }

int hmm_set_call_graphs(hmm_ctx *c, int on) {
    if (!c) return HMM_EINVAL;
    c->graphs_on = on != 0;
    if (!c->graphs_on) {
        cudaSetDevice(c->device);
        drop_call_graph(c);
    }
    return HMM_OK;
}

int hmm_last_call_graph(const hmm_ctx *c) { return c ? c->last_graph : -1; }

int hmm_profile_enable(hmm_ctx *c, int on) {
    if (!c) return HMM_EINVAL;
    cudaSetDevice(c->device);
    prof_collect(c);
    if (on && !c->ev[0]) {
        for (auto &e : c->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(c, r, "cudaEventCreate");
        }
    }
    c->prof_on = on != 0;
    if (on) {
        for (double &m : c->prof_ms) m = 0.0;
        c->prof_calls = 0;
    }
    return HMM_OK;
}

int hmm_profile_read(hmm_ctx *c, double *ms_out, int *n_calls) {
    if (!c || !ms_out) return HMM_EINVAL;
    cudaSetDevice(c->device);
    prof_collect(c);
    for (int i = 0; i < HMM_PHASE_COUNT; ++i) ms_out[i] = c->prof_ms[i];
    if (n_calls) *n_calls = c->prof_calls;
    return HMM_OK;
}

int hmm_status(hmm_ctx *c, void *stream) {
    if (!c) return HMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "hmm_status");
    if (h & ST_EINVAL) return fail(c, HMM_EINVAL, "a parameter set or a flagged observation failed its checks");
    if (h & ST_ENUMERIC) return fail(c, HMM_ENUMERIC, "a scaled value left the representable range");
    if (h & ST_ETIMEOUT) return fail(c, HMM_ETIMEOUT, "a bounded device wait expired");
    return HMM_OK;
}

// The per-call workspace, in carving order (sizes only when base is null).
struct WorkPtrs {
    float *cblock = nullptr;
    int *prop_bad = nullptr, *obs_bad = nullptr;
    float2 *packed = nullptr, *head = nullptr;
    LevelPtrs lv{};
};

static size_t carve_work(void *base, int n_prop, int n_seg, const ConstLayout &lay, const Plan &pl, WorkPtrs *w) {
    const int KP = lay.KP;
    Carve cv(base);
    w->cblock = cv.take<float>((size_t)n_prop * lay.stride);
    w->prop_bad = cv.take<int>(n_prop);
    w->obs_bad = cv.take<int>(1);
    w->packed = cv.take<float2>(pl.n_packed);
    w->head = cv.take<float2>(n_seg);
    w->lv = LevelPtrs{};
    for (int l = 0; l <= pl.n_levels; ++l) {
        w->lv.A[l] = cv.take<float>((size_t)n_prop * std::max(1, pl.level_n[l]) * KP * KP);
        if (l == 0) w->lv.e[l] = cv.take<int32_t>((size_t)n_prop * std::max(1, pl.level_n[l]) * KP);
        else w->lv.e[l] = cv.take<long long>((size_t)n_prop * std::max(1, pl.level_n[l]) * KP);
        w->lv.n[l] = pl.level_n[l];
    }
    return cv.off;
}

int hmm_loglik_batched(hmm_ctx *c, int32_t n_prop, int32_t K, const float *pi, const float *P,
                       const float *p, const float *mu, const float *cov, int32_t n_seg,
                       const int64_t *offs, const float *xy, const uint8_t *tremor,
                       const hmm_opts *opts_in, double *out, void *stream) {
    if (!c) return HMM_EINVAL;
    c->last_launches = 0;
    hmm_opts opts;
    if (opts_in) opts = *opts_in; else hmm_opts_default(&opts);
    if (K < 1 || K > 80) return fail(c, HMM_EINVAL, "K=%d outside 1..80", K);
    if (n_prop < 1) return fail(c, HMM_EINVAL, "n_prop=%d < 1", n_prop);
    if (n_seg < 1 || !offs) return fail(c, HMM_EINVAL, "need n_seg >= 1 and seg_offsets");
    if (!pi || !P || !p || !mu || !cov || !out) return fail(c, HMM_EINVAL, "null parameter or output pointer");
    if (offs[0] != 0) return fail(c, HMM_EINVAL, "seg_offsets[0] must be 0");
    for (int s = 0; s < n_seg; ++s)
        if (offs[s + 1] < offs[s]) return fail(c, HMM_EINVAL, "seg_offsets must be non-decreasing");
    const int64_t T_total = offs[n_seg];
    if (T_total > 0 && (!xy || !tremor)) return fail(c, HMM_EINVAL, "null observation pointer");
    if (xy && ((uintptr_t)xy & 7)) return fail(c, HMM_EINVAL, "xy must be 8-byte aligned");
    if (opts.init_mode != HMM_INIT_EMIT_FIRST && opts.init_mode != HMM_INIT_TRANSITION_FIRST)
        return fail(c, HMM_EINVAL, "bad init_mode %d", opts.init_mode);
    if (opts.chunk_len < 0 || (opts.chunk_len % OBS_WIN) != 0)
        return fail(c, HMM_EINVAL, "chunk_len must be 0 or a positive multiple of %d", OBS_WIN);
    if (opts.renorm_every < 0 || opts.renorm_every > 64)
        return fail(c, HMM_EINVAL, "renorm_every must be 0..64");
    for (int r = 0; r < 2; ++r)
        if (opts.reserved[r]) return fail(c, HMM_EINVAL, "reserved option fields must be 0");
    const int min_run = opts.runlen_min;
    if (min_run < 0 || min_run > 16384) return fail(c, HMM_EINVAL, "runlen_min must be 0..16384");
    const int prec = opts.precision;
    if (prec != HMM_PREC_FP32_SIMT && prec != HMM_PREC_TF32 && prec != HMM_PREC_BF16 &&
        prec != HMM_PREC_TF32_SPLIT)
        return fail(c, HMM_EINVAL, "bad precision %d", prec);
    if (prec != HMM_PREC_FP32_SIMT && !chunk_tc_supported(K, prec))
        return fail(c, HMM_EUNSUPPORTED, "tensor-core path does not support K=%d precision %d", K, prec);
    if (min_run && prec != HMM_PREC_FP32_SIMT)
        return fail(c, HMM_EUNSUPPORTED, "the run-length shortcut runs on the FP32-SIMT path only");
    const int renorm = opts.renorm_every ? opts.renorm_every : 4;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");

    // ---- plan (cached while the shape is unchanged) ----
    ConstLayout lay = make_layout(K, prec);
    int64_t steps_total = 0;
    for (int s = 0; s < n_seg; ++s) steps_total += std::max<int64_t>(0, offs[s + 1] - offs[s] - 1);
    if (!c->n_sms) cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, c->device);
    int L = opts.chunk_len;
    if (!L) {
        // a tuned chunk length for this shape if the tuner stored one, else the cost model's
        const TuneKey key{c->n_sms, K, prec, n_prop, n_seg, min_run, steps_total};
        L = tune_get(key);
        if (!L) L = choose_chunk_len(prec, n_prop, lay.KP, steps_total, c->n_sms);
    }
    if (!plan_matches(c->plan, K, n_prop, n_seg, offs, prec, L)) {
        build_plan(c->plan, K, n_prop, n_seg, offs, prec, L);
        if (c->plan.n_levels + 1 > MAX_LEVELS) {
            c->plan.valid = false;
            return fail(c, HMM_EINVAL, "too many chunks for the tree (raise chunk_len)");
        }
        int rc = upload_plan(c, st);
        if (rc) return rc;
    }
    Plan &pl = c->plan;
    c->last_L = L;

    // ---- workspace ----
    const int KP = lay.KP;
    WorkPtrs wp;
    const size_t main_bytes = (carve_work(nullptr, n_prop, n_seg, lay, pl, &wp) + 255) & ~(size_t)255;
    // run-length table after the main carve (the other entry points never see it)
    const int nb = min_run ? rle_levels(L) : 0;
    const size_t qtab_bytes = ((size_t)n_prop * nb * KP * KP * sizeof(float) + 255) & ~(size_t)255;
    const size_t qexp_bytes = (size_t)n_prop * nb * KP * sizeof(int32_t);
    int rc = ensure(c, c->work, main_bytes + qtab_bytes + qexp_bytes + 4096);
    if (rc) return rc;
    carve_work(c->work.p, n_prop, n_seg, lay, pl, &wp);
    float *qtab = (float *)((char *)c->work.p + main_bytes);
    int32_t *qexp = (int32_t *)((char *)c->work.p + main_bytes + qtab_bytes);
    float *cblock = wp.cblock;
    int *prop_bad = wp.prop_bad;
    int *obs_bad = wp.obs_bad;
    float2 *packed = wp.packed;
    float2 *head = wp.head;
    LevelPtrs lv = wp.lv;

    // ---- launches ----
    // The whole sequence, on stream `s` (the caller's, or the capture stream).
    auto enqueue = [&](cudaStream_t s, int &launches) -> cudaError_t {
        launches = 0;
        prof_mark(c, HMM_PHASE_PREP, s);
        cudaError_t r = cudaMemsetAsync(obs_bad, 0, sizeof(int), s);
        if (r == cudaSuccess) { r = launch_prep(n_prop, K, lay, prec, opts.init_mode, pi, P, p, mu, cov, cblock, prop_bad, c->d_status, s); ++launches; }
        prof_mark(c, HMM_PHASE_PACK, s);
        if (r == cudaSuccess && T_total > 0) { r = launch_pack(n_seg, pl.d_offsets, pl.d_pbase, T_total, xy, tremor, packed, head, obs_bad, c->d_status, s); ++launches; }
        prof_mark(c, HMM_PHASE_CHUNK, s);
        if (r == cudaSuccess && pl.n_chunks > 0) {
            if (min_run) {
                r = launch_rle_table(n_prop, nb, lay, cblock, qtab, qexp, c->d_status, s);
                ++launches;
                if (r == cudaSuccess)
                    r = launch_chunk_rle(n_prop, pl.n_chunks, renorm, min_run, nb, lay, cblock, qtab, qexp, pl.d_chunks,
                                         packed, lv.A[0], (int32_t *)lv.e[0], c->d_status, s);
            } else if (prec == HMM_PREC_FP32_SIMT)
                r = launch_chunk_simt(n_prop, pl.n_chunks, L, renorm, lay, cblock, pl.d_chunks, packed, lv.A[0], (int32_t *)lv.e[0], c->d_status, s);
            else
                r = launch_chunk_tc(n_prop, pl.n_chunks, L, renorm, prec, lay, cblock, pl.d_chunks, packed, lv.A[0], (int32_t *)lv.e[0], c->d_status, s);
            ++launches;
        }
        prof_mark(c, HMM_PHASE_TREE, s);
        for (int l = 0; l < pl.n_levels && r == cudaSuccess; ++l) {
            r = launch_tree_level(n_prop, KP, l, (int)pl.groups[l].size(), pl.d_groups[l], lv, c->d_status, s);
            ++launches;
        }
        prof_mark(c, HMM_PHASE_FINAL, s);
        if (r == cudaSuccess) {
            r = launch_final(n_prop, K, opts.init_mode, n_seg, pl.d_segs, head, lv, KP, pi, P, p, mu, cov, prop_bad, obs_bad, out, s);
            ++launches;
        }
        prof_mark(c, HMM_PHASE_COUNT, s);
        return r;
    };

    prof_collect(c);
    c->last_graph = 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamIsCapturing");
    if (c->graphs_on && !c->prof_on && cap == cudaStreamCaptureStatusNone) {
        const std::vector<uint64_t> key = {
            (uint64_t)(uintptr_t)pi, (uint64_t)(uintptr_t)P, (uint64_t)(uintptr_t)p, (uint64_t)(uintptr_t)mu,
            (uint64_t)(uintptr_t)cov, (uint64_t)(uintptr_t)xy, (uint64_t)(uintptr_t)tremor, (uint64_t)(uintptr_t)out,
            (uint64_t)(uintptr_t)c->work.p, c->plan_version, (uint64_t)n_prop, (uint64_t)K, (uint64_t)n_seg,
            (uint64_t)prec, (uint64_t)opts.init_mode, (uint64_t)renorm, (uint64_t)min_run, (uint64_t)L,
            (uint64_t)T_total};
        if (c->call_exec && c->call_key == key) {
            e = cudaGraphLaunch(c->call_exec, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
            c->last_launches = c->call_launches;
            c->last_graph = 2;
            return HMM_OK;
        }
        if (c->call_exec) {
            // another configuration's graph: it goes, the remembered key stays
            cudaGraphExecDestroy(c->call_exec);
            c->call_exec = nullptr;
            c->call_key.clear();
        }
        if (c->seen_key != key) {
            // first call of this configuration: launch directly, capture on a repeat
            c->seen_key = key;
            int launches = 0;
            e = enqueue(st, launches);
            c->last_launches = launches;
            if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
            return HMM_OK;
        }
        if (!c->cap_stream) {
            e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamCreateWithFlags");
        }
        int launches = 0;
        e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            const cudaError_t eq = enqueue(c->cap_stream, launches);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(c->cap_stream, &g);
            if (eq != cudaSuccess) e = eq;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->call_exec, g, 0);
            if (g) cudaGraphDestroy(g);
        }
        if (e == cudaSuccess) {
            c->call_key = key;
            c->call_launches = launches;
            e = cudaGraphLaunch(c->call_exec, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
            c->last_launches = launches;
            c->last_graph = 1;
            return HMM_OK;
        }
        // the sequence could not be captured here: launch it directly (the
        // same kernels; a launch error shows up again below)
        drop_call_graph(c);
        cudaGetLastError();
    }
    int launches = 0;
    e = enqueue(st, launches);
    if (c->prof_on) c->prof_pending = true;
    c->last_launches = launches;
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    return HMM_OK;
}

int hmm_loglik(hmm_ctx *c, const hmm_params *prm, const hmm_obs *obs, const hmm_opts *opts,
               double *out, void *stream) {
    if (!c) return HMM_EINVAL;
    if (!prm || !obs) return fail(c, HMM_EINVAL, "null params or obs");
    if (obs->T < 0) return fail(c, HMM_EINVAL, "T < 0");
    int64_t offs[2] = {0, obs->T};
    return hmm_loglik_batched(c, 1, prm->K, prm->pi, prm->P, prm->p_tremor, prm->mu, prm->cov, 1,
                              offs, obs->xy, obs->tremor, opts, out, stream);
}

// the posterior (and optionally the E-step statistics) of one sequence
static int posterior_impl(hmm_ctx *c, const hmm_params *prm, const hmm_obs *obs, const hmm_opts *opts,
                          float *gamma, double *loglik, double *stats, void *stream) {
    if (!c) return HMM_EINVAL;
    if (!prm || !obs || !gamma || !loglik) return fail(c, HMM_EINVAL, "null argument");
    if (obs->T < 1) return fail(c, HMM_EINVAL, "T must be >= 1");
    int64_t offs[2] = {0, obs->T};
    hmm_opts o;
    if (opts) o = *opts; else hmm_opts_default(&o);
    if (o.chunk_len == 0) {
        // the boundary scans cost ~1.5 us per chunk in sequence and every chunk
        // ~0.5 us per step (all chunks in one wave): L ~ sqrt(3 T) balances them
        const int64_t Lp = ((int64_t)std::sqrt(3.0 * (double)obs->T) + OBS_WIN - 1) / OBS_WIN * OBS_WIN;
        o.chunk_len = (int32_t)std::min<int64_t>(16384, std::max<int64_t>(OBS_WIN, Lp));
    }
    // the likelihood path computes the chunk products (and log L)
    int rc = hmm_loglik_batched(c, 1, prm->K, prm->pi, prm->P, prm->p_tremor, prm->mu, prm->cov, 1, offs, obs->xy,
                                obs->tremor, &o, loglik, stream);
    if (rc) return rc;
    const Plan &pl = c->plan;
    const int K = prm->K, KP = pl.lay.KP, C = std::max(1, pl.n_chunks);
    WorkPtrs wp;
    carve_work(c->work.p, 1, 1, pl.lay, pl, &wp);
    size_t fb_bytes = sizeof(float) * 2 * (size_t)C * KP + 256;
    if (stats) fb_bytes += sizeof(double) * ((size_t)C * (K * K + 7 * K) + K) + 256;
    rc = ensure(c, c->fb, fb_bytes);
    if (rc) return rc;
    float *fvec = (float *)c->fb.p;
    float *bvec = fvec + (size_t)C * KP;
    double *part = nullptr, *g0 = nullptr;
    if (stats) {
        part = (double *)(((uintptr_t)(bvec + (size_t)C * KP) + 255) & ~(uintptr_t)255);
        g0 = part + (size_t)C * (K * K + 7 * K);
    }
    cudaError_t e = launch_posterior(K, KP, o.init_mode, pl.n_chunks, pl.L, pl.d_chunks, prm->pi, prm->P,
                                     wp.cblock + pl.lay.off_emis, wp.head, wp.packed, wp.lv.A[0],
                                     (const int32_t *)wp.lv.e[0], fvec, bvec, gamma, part, g0, stats,
                                     (cudaStream_t)stream);
    c->last_launches += 1 + (pl.n_chunks > 0 ? 1 : 0) + (stats && pl.n_chunks > 0 ? 1 : 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "posterior launch");
    return HMM_OK;
}

int hmm_posterior(hmm_ctx *c, const hmm_params *prm, const hmm_obs *obs, const hmm_opts *opts, float *gamma,
                  double *loglik, void *stream) {
    return posterior_impl(c, prm, obs, opts, gamma, loglik, nullptr, stream);
}

int hmm_expected_stats(hmm_ctx *c, const hmm_params *prm, const hmm_obs *obs, const hmm_opts *opts,
                       double *stats, double *loglik, void *stream) {
    if (!c) return HMM_EINVAL;
    if (!prm || !obs || !stats || !loglik) return fail(c, HMM_EINVAL, "null argument");
    if (obs->T < 2) return fail(c, HMM_EINVAL, "T must be >= 2");
    // the posterior vectors go to a context-owned buffer
    int rc = ensure(c, c->gam, sizeof(float) * (size_t)obs->T * prm->K + 256);
    if (rc) return rc;
    return posterior_impl(c, prm, obs, opts, (float *)c->gam.p, loglik, stats, stream);
}

int hmm_loglik_grad(hmm_ctx *c, const hmm_params *prm, const hmm_obs *obs, const hmm_opts *opts, double *grad,
                    double *loglik, void *stream) {
    if (!c) return HMM_EINVAL;
    if (!prm || !obs || !grad || !loglik) return fail(c, HMM_EINVAL, "null argument");
    if (prm->K < 1 || prm->K > 80) return fail(c, HMM_EINVAL, "K must be 1..80");
    int rc = ensure(c, c->stats, sizeof(double) * ((size_t)prm->K * prm->K + 8 * prm->K));
    if (rc) return rc;
    double *st = (double *)c->stats.p;
    rc = hmm_expected_stats(c, prm, obs, opts, st, loglik, stream);
    if (rc) return rc;
    const int init_mode = opts ? opts->init_mode : HMM_INIT_EMIT_FIRST;
    cudaError_t e = launch_fisher_grad(prm->K, init_mode, prm->pi, prm->P, prm->p_tremor, prm->mu, prm->cov, st, grad,
                                       (cudaStream_t)stream);
    c->last_launches += 1;
    return e == cudaSuccess ? HMM_OK : cuda_fail(c, e, "gradient launch");
}

int hmm_em_step(hmm_ctx *c, const hmm_params *prm, const hmm_obs *obs, const hmm_opts *opts, float *pi_out,
                float *P_out, float *p_out, float *mu_out, float *cov_out, double *loglik, void *stream) {
    if (!c) return HMM_EINVAL;
    if (!prm || !obs || !pi_out || !P_out || !p_out || !mu_out || !cov_out || !loglik)
        return fail(c, HMM_EINVAL, "null argument");
    if (prm->K < 1 || prm->K > 80) return fail(c, HMM_EINVAL, "K must be 1..80");
    if (opts && opts->init_mode != HMM_INIT_EMIT_FIRST)
        return fail(c, HMM_EUNSUPPORTED, "the EM update has a closed form for the emit-first convention only");
    int rc = ensure(c, c->stats, sizeof(double) * ((size_t)prm->K * prm->K + 8 * prm->K));
    if (rc) return rc;
    double *st = (double *)c->stats.p;
    rc = hmm_expected_stats(c, prm, obs, opts, st, loglik, stream);
    if (rc) return rc;
    cudaError_t e = launch_em_mstep(prm->K, prm->pi, prm->P, prm->p_tremor, prm->mu, prm->cov, st, pi_out, P_out,
                                    p_out, mu_out, cov_out, (cudaStream_t)stream);
    c->last_launches += 1;
    return e == cudaSuccess ? HMM_OK : cuda_fail(c, e, "EM launch");
}

int hmm_viterbi(hmm_ctx *c, const hmm_params *prm, const hmm_obs *obs, const hmm_opts *opts, int32_t *path,
                double *score, double *loglik, void *stream) {
    if (!c) return HMM_EINVAL;
    if (!prm || !obs || !path || !score || !loglik) return fail(c, HMM_EINVAL, "null argument");
    if (obs->T < 1) return fail(c, HMM_EINVAL, "T must be >= 1");
    if (prm->K > 255) return fail(c, HMM_EINVAL, "K must be <= 255");
    int64_t offs[2] = {0, obs->T};
    hmm_opts o;
    if (opts) o = *opts; else hmm_opts_default(&o);
    o.precision = HMM_PREC_FP32_SIMT;  // the max-plus chunks run on the CUDA cores
    if (o.chunk_len == 0) {
        const int64_t Lp = ((int64_t)std::sqrt(3.0 * (double)obs->T) + OBS_WIN - 1) / OBS_WIN * OBS_WIN;
        o.chunk_len = (int32_t)std::min<int64_t>(16384, std::max<int64_t>(OBS_WIN, Lp));
    }
    // parameters, observations and the chunk table (and log L) from the likelihood path
    int rc = hmm_loglik_batched(c, 1, prm->K, prm->pi, prm->P, prm->p_tremor, prm->mu, prm->cov, 1, offs, obs->xy,
                                obs->tremor, &o, loglik, stream);
    if (rc) return rc;
    const Plan &pl = c->plan;
    const int KP = pl.lay.KP, C = std::max(1, pl.n_chunks);
    WorkPtrs wp;
    carve_work(c->work.p, 1, 1, pl.lay, pl, &wp);
    Carve cv(nullptr);
    cv.take<float>((size_t)C * KP * KP);
    cv.take<double>((size_t)C * KP);
    cv.take<int32_t>((size_t)C * KP);
    cv.take<int32_t>((size_t)C + 1);
    cv.take<uint8_t>((size_t)C * pl.L * KP);
    rc = ensure(c, c->fb, cv.off + 1024);
    if (rc) return rc;
    Carve vc(c->fb.p);
    float *V = vc.take<float>((size_t)C * KP * KP);
    double *voff = vc.take<double>((size_t)C * KP);
    int32_t *ptr = vc.take<int32_t>((size_t)C * KP);
    int32_t *bstate = vc.take<int32_t>((size_t)C + 1);
    uint8_t *bp = vc.take<uint8_t>((size_t)C * pl.L * KP);
    cudaError_t e = launch_viterbi(prm->K, o.init_mode, pl.n_chunks, pl.L, pl.lay, pl.d_chunks, prm->pi, prm->P,
                                   wp.cblock, wp.head, wp.packed, V, voff, ptr, bstate, bp, path, score,
                                   (cudaStream_t)stream);
    c->last_launches += pl.n_chunks > 0 ? 3 : 2;
    if (e != cudaSuccess) return cuda_fail(c, e, "viterbi launch");
    return HMM_OK;
}

int hmm_loglik_batched_host(hmm_ctx *c, int32_t n_prop, int32_t K, const float *pi, const float *P,
                            const float *p, const float *mu, const float *cov, int32_t n_seg,
                            const int64_t *offs, const float *xy, const uint8_t *tremor,
                            const hmm_opts *opts, double *out_host, void *stream) {
    if (!c) return HMM_EINVAL;
    if (K < 1 || K > 80 || n_prop < 1 || n_seg < 1 || !offs || !out_host || !pi || !P || !p || !mu || !cov)
        return fail(c, HMM_EINVAL, "bad arguments");
    const int64_t T_total = offs[n_seg];
    if (T_total < 0) return fail(c, HMM_EINVAL, "bad seg_offsets");
    if (T_total > 0 && (!xy || !tremor)) return fail(c, HMM_EINVAL, "null observation pointer");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const size_t nk = (size_t)n_prop * K;
    size_t need = 0;
    auto add = [&](size_t b) { need += (b + 255) & ~(size_t)255; };
    add(4 * nk); add(4 * nk * K); add(4 * nk); add(8 * nk); add(12 * nk);
    add(8 * (size_t)T_total); add((size_t)T_total); add(8 * (size_t)n_prop);
    int rc = ensure(c, c->stage, need + 4096);
    if (rc) return rc;
    Carve cv(c->stage.p);
    float *dpi = cv.take<float>(nk), *dP = cv.take<float>(nk * K), *dp = cv.take<float>(nk);
    float *dmu = cv.take<float>(2 * nk), *dcov = cv.take<float>(3 * nk);
    float *dxy = cv.take<float>(2 * (size_t)T_total);
    uint8_t *dtr = cv.take<uint8_t>((size_t)T_total);
    double *dout = cv.take<double>(n_prop);
    struct { void *d; const void *h; size_t n; } cp[] = {
        {dpi, pi, 4 * nk}, {dP, P, 4 * nk * K}, {dp, p, 4 * nk}, {dmu, mu, 8 * nk},
        {dcov, cov, 12 * nk}, {dxy, xy, 8 * (size_t)T_total}, {dtr, tremor, (size_t)T_total}};
    for (auto &x : cp) {
        if (x.n == 0) continue;
        e = cudaMemcpyAsync(x.d, x.h, x.n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
    }
    rc = hmm_loglik_batched(c, n_prop, K, dpi, dP, dp, dmu, dcov, n_seg, offs,
                            T_total ? dxy : nullptr, T_total ? dtr : nullptr, opts, dout, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(out_host, dout, 8 * (size_t)n_prop, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
    return hmm_status(c, stream);
}


// ---- chunk-length tuning (see the header) ----

int32_t hmm_default_chunk_len(int32_t precision, int32_t n_prop, int32_t K, int64_t steps_total, int32_t n_sms) {
    if (K < 1 || K > 80 || n_prop < 1 || steps_total < 0 || n_sms < 1) return 0;
    if (precision != HMM_PREC_FP32_SIMT && !chunk_tc_supported(K, precision)) return 0;
    return choose_chunk_len(precision, n_prop, make_layout(K, precision).KP, steps_total, n_sms);
}

int hmm_tune_candidates(int32_t precision, int32_t n_prop, int32_t K, int64_t steps_total, int32_t n_sms,
                        int32_t *out, int32_t cap, int32_t *n_out) {
    if (!out || !n_out || cap < 1 || K < 1 || K > 80 || n_prop < 1 || steps_total < 0 || n_sms < 1)
        return HMM_EINVAL;
    if (precision != HMM_PREC_FP32_SIMT && !chunk_tc_supported(K, precision)) return HMM_EINVAL;
    const std::vector<int> c = tune_candidates(precision, n_prop, K, steps_total, n_sms);
    const int n = std::min<int>(cap, (int)c.size());
    for (int i = 0; i < n; ++i) out[i] = c[i];
    *n_out = n;
    return HMM_OK;
}

int hmm_autotune_batched(hmm_ctx *c, int32_t n_prop, int32_t K, const float *pi, const float *P,
                         const float *p, const float *mu, const float *cov, int32_t n_seg,
                         const int64_t *offs, const float *xy, const uint8_t *tremor,
                         const hmm_opts *opts_in, int32_t reps, double *out, int32_t *chunk_len_out,
                         double *ms_out, void *stream) {
    if (!c) return HMM_EINVAL;
    hmm_opts opts;
    if (opts_in) opts = *opts_in; else hmm_opts_default(&opts);
    if (opts.chunk_len != 0) return fail(c, HMM_EINVAL, "autotuning needs opts->chunk_len = 0");
    if (reps < 1 || reps > 100) return fail(c, HMM_EINVAL, "reps=%d outside 1..100", reps);
    if (K < 1 || K > 80 || n_prop < 1 || n_seg < 1 || !offs)
        return fail(c, HMM_EINVAL, "bad shape arguments");
    if (opts.precision != HMM_PREC_FP32_SIMT && !chunk_tc_supported(K, opts.precision))
        return fail(c, HMM_EUNSUPPORTED, "tensor-core path does not support K=%d precision %d", K, opts.precision);
    if (offs[0] != 0) return fail(c, HMM_EINVAL, "seg_offsets[0] must be 0");
    int64_t steps_total = 0;
    for (int s = 0; s < n_seg; ++s) {
        if (offs[s + 1] < offs[s]) return fail(c, HMM_EINVAL, "seg_offsets must be non-decreasing");
        steps_total += std::max<int64_t>(0, offs[s + 1] - offs[s] - 1);
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    if (!c->n_sms) cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, c->device);
    const std::vector<int> cand = tune_candidates(opts.precision, n_prop, K, steps_total, c->n_sms);

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, e, "cudaEventCreate");
    }
    // the tuner's own calls stay out of the phase profile
    const bool prof_was = c->prof_on;
    c->prof_on = false;
    int best_L = 0, rc = HMM_OK, last_rc = HMM_OK;
    double best_ms = 0.0;
    for (int L : cand) {
        hmm_opts o = opts;
        o.chunk_len = L;
        // warm-up: builds the plan and grows the workspace
        rc = hmm_loglik_batched(c, n_prop, K, pi, P, p, mu, cov, n_seg, offs, xy, tremor, &o, out, stream);
        if (rc == HMM_EINVAL || rc == HMM_ENOMEM) {
            // this chunk length does not fit (tree depth, memory): try the others
            last_rc = rc;
            rc = HMM_OK;
            continue;
        }
        if (rc) break;
        e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && e == cudaSuccess && rc == HMM_OK; ++r)
            rc = hmm_loglik_batched(c, n_prop, K, pi, P, p, mu, cov, n_seg, offs, xy, tremor, &o, out, stream);
        if (rc) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(c, e, "tuning events");
            break;
        }
        const double per = (double)ms / reps;
        if (!best_L || per < best_ms) {
            best_L = L;
            best_ms = per;
        }
    }
    c->prof_on = prof_was;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (!best_L) return fail(c, last_rc ? last_rc : HMM_EINVAL, "no candidate chunk length could be evaluated");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_put_locked(TuneEntry{TuneKey{c->n_sms, K, opts.precision, n_prop, n_seg, opts.runlen_min, steps_total},
                                  best_L, best_ms});
    }
    // leave the caller's output and the context's plan at the winner
    hmm_opts o = opts;
    o.chunk_len = best_L;
    rc = hmm_loglik_batched(c, n_prop, K, pi, P, p, mu, cov, n_seg, offs, xy, tremor, &o, out, stream);
    if (rc) return rc;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    if (chunk_len_out) *chunk_len_out = best_L;
    if (ms_out) *ms_out = best_ms;
    return HMM_OK;
}

int hmm_tune_lookup(int32_t n_sms, int32_t K, int32_t precision, int32_t n_prop, int32_t n_seg,
                    int64_t steps_total, int32_t runlen_min, int32_t *chunk_len) {
    if (!chunk_len) return HMM_EINVAL;
    *chunk_len = tune_get(TuneKey{n_sms, K, precision, n_prop, n_seg, runlen_min, steps_total});
    return HMM_OK;
}

int hmm_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    return HMM_OK;
}

int hmm_tune_save(const char *path) {
    if (!path) return HMM_EINVAL;
    std::vector<TuneEntry> snap;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        snap = g_tune;
    }
    FILE *f = fopen(path, "w");
    if (!f) return HMM_EINVAL;
    bool ok = fprintf(f, "# hmm_gb300 tuned chunk lengths: n_sms K precision n_prop n_seg steps_total "
                         "runlen_min chunk_len ms_per_call\n") > 0;
    for (const TuneEntry &t : snap)
        ok = ok && fprintf(f, "%d %d %d %d %d %lld %d %d %.6f\n", t.key.n_sms, t.key.K, t.key.precision,
                           t.key.n_prop, t.key.n_seg, (long long)t.key.steps, t.key.runlen_min, t.L, t.ms) > 0;
    ok = (fclose(f) == 0) && ok;
    return ok ? HMM_OK : HMM_EINVAL;
}

int hmm_tune_load(const char *path) {
    if (!path) return HMM_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f) return HMM_EINVAL;
    std::vector<TuneEntry> got;
    char line[512];
    bool ok = true;
    while (ok && fgets(line, sizeof(line), f)) {
        const size_t n = strlen(line);
        if (n == sizeof(line) - 1 && line[n - 1] != '\n') {  // over-long line
            ok = false;
            break;
        }
        const char *q = line;
        while (*q == ' ' || *q == '\t') ++q;
        if (*q == '#' || *q == '\n' || *q == '\r' || *q == '\0') continue;
        TuneEntry t{};
        long long steps = 0;
        int used = 0;
        const int m = sscanf(q, "%d %d %d %d %d %lld %d %d %lf %n", &t.key.n_sms, &t.key.K, &t.key.precision,
                             &t.key.n_prop, &t.key.n_seg, &steps, &t.key.runlen_min, &t.L, &t.ms, &used);
        t.key.steps = steps;
        if (m != 9 || q[used] != '\0' || !tune_entry_valid(t)) {
            ok = false;
            break;
        }
        got.push_back(t);
    }
    if (ferror(f)) ok = false;
    fclose(f);
    if (!ok) return HMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneEntry &t : got) tune_put_locked(t);
    return HMM_OK;
}

}  // extern "C"
