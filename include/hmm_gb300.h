/*
 * hmm_gb300.h -- C ABI of the GB300 (sm_103a) tremor-HMM likelihood library.
 *
 * What is computed (Section 2 of Stoltz et al., "A 1000-fold acceleration of
 * hidden Markov model fitting using GPUs"):
 *
 *   Eq. "emission-matrix": for an observation o and hidden state k the
 *   diagonal emission matrix D(o) has entries
 *       D(o)_kk = p_k * phi(o | mu_k, Sigma_k)   if a tremor is observed at o in R^2,
 *       D(o)_kk = 1 - p_k                         if no tremor is observed,
 *   phi being the bivariate normal density.
 *
 *   Eq. "likelihood func": L = pi^T D_1 P D_2 P ... P D_T 1 (emit-first, the
 *   default), or with HMM_INIT_TRANSITION_FIRST the printed form
 *   L = pi^T P D_1 P D_2 ... P D_T 1. P (the paper's Gamma) is the transition
 *   matrix, P[i*K+j] = Pr(i -> j); pi (the paper's delta) the initial vector.
 *
 *   Section "The likelihood algorithm", steps 1-3: the emissions are
 *   evaluated in parallel, the matrices M_t = P D_t are multiplied as a chain
 *   split into chunks, the chunk products are combined, and log L (not L) is
 *   returned, with scale coefficients keeping every partial product in range.
 *
 * Conventions for every entry point:
 *   - Every function returns an int status: HMM_OK (0) or one of HMM_E*.
 *     Nothing traps or aborts; hmm_last_error() describes the last failure.
 *   - Pointers are DEVICE pointers unless the name ends in _host. The caller
 *     owns every buffer it passes; the library never frees or keeps them
 *     past the call (results are written asynchronously on `stream`).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - K is 1..80. T (per segment) is >= 0; T = 0 gives log(sum_k pi_k).
 *   - Parameter checks that need the device data (rows of P and pi >= 0 and
 *     summing to 1 within 1e-5, 0 <= p_k <= 1, Sigma_k symmetric positive
 *     definite, finite means, finite xy wherever a tremor is flagged) run on
 *     the device: an invalid proposal's result is NaN and the context's
 *     status word records HMM_EINVAL; hmm_status() synchronises and reads it.
 *   - A true zero likelihood returns -INFINITY with HMM_OK.
 *   - Results are bit-for-bit reproducible for the same inputs, options and
 *     GPU model (fixed chunking, fixed reduction order, no atomics on data).
 *   - One context per host thread; contexts are independent.
 */
#ifndef HMM_GB300_H
#define HMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HMM_OK 0
#define HMM_EINVAL 1       /* bad argument (host check) or bad parameter data (device check) */
#define HMM_ECUDA 2        /* a CUDA runtime call failed; see hmm_last_error() */
#define HMM_ENOMEM 3       /* workspace allocation failed */
#define HMM_ENUMERIC 4     /* a value left the representable range (see hmm_status) */
#define HMM_ETIMEOUT 5     /* a bounded device wait expired (kernel returned early) */
#define HMM_EUNSUPPORTED 6 /* option not available for this K / device */

/* ---- arithmetic of the chunk products (Step 3) ---- */
#define HMM_PREC_FP32_SIMT 0  /* FP32 FFMA on the CUDA cores ("plain GPU") */
#define HMM_PREC_TF32 1       /* tcgen05 tensor cores, TF32 operands, FP32 accumulation */
#define HMM_PREC_BF16 2       /* tcgen05 tensor cores, BF16 running product, P as BF16 hi+lo */
#define HMM_PREC_TF32_SPLIT 3 /* tcgen05 TF32 with P as TF32 hi+lo (two MMAs) */

/* ---- where pi enters ---- */
#define HMM_INIT_EMIT_FIRST 0       /* L = pi^T D_1 P D_2 ... (pi = law of the first state) */
#define HMM_INIT_TRANSITION_FIRST 1 /* L = pi^T P D_1 P D_2 ... (Eq. "likelihood func", Algorithm 1) */

typedef struct hmm_ctx hmm_ctx;

/* One parameter set (Section 2: pi, P, and per state p_k, mu_k, Sigma_k). All float32, device. */
typedef struct {
    int32_t K;
    const float *pi;       /* [K]                                        */
    const float *P;        /* [K*K] row-major, P[i*K+j] = Pr(i -> j)      */
    const float *p_tremor; /* [K]  probability of observing a tremor      */
    const float *mu;       /* [K*2] (x, y) mean location                  */
    const float *cov;      /* [K*3] (sxx, sxy, syy) covariance             */
} hmm_params;

/* One observation sequence x_0..x_{T-1} (Section 2: each is "no tremor" or a point in R^2). */
typedef struct {
    int64_t T;
    const float *xy;        /* [T*2] (x, y); ignored where tremor == 0 */
    const uint8_t *tremor;  /* [T]   1 = tremor observed at xy, 0 = none */
} hmm_obs;

typedef struct {
    int32_t precision;    /* HMM_PREC_*                                           */
    int32_t init_mode;    /* HMM_INIT_*                                           */
    int32_t chunk_len;    /* steps per chunk product (multiple of 64); 0 = tuned or cost model (below) */
    int32_t renorm_every; /* per-row power-of-two renormalisation interval; 0 = 4 */
    int32_t recheck_fp32; /* samplers only (see hmm_sampler_create); ignored here  */
    int32_t runlen_min;   /* run-length shortcut, FP32-SIMT only; 0 = off (below)  */
    int32_t reserved[2];  /* must be 0                                             */
} hmm_opts;

/*
 * Run-length shortcut (opts->runlen_min = n_min >= 1). Every step without a
 * tremor has the same matrix M_0 = P diag(1 - p_k) (Eq. "emission-matrix"),
 * so a run of n of them inside a chunk contributes M_0^n. With the shortcut
 * on, the library first builds, per proposal, M_0^(2^b) for b = 0 ..
 * floor(log2(chunk length)) by repeated squaring (each row a float row plus
 * its own power-of-two exponent), and every run of at least n_min
 * no-tremor steps is applied as the product of the powers of its length's
 * set bits: popcount(n) matrix products instead of n. The result is the same
 * likelihood up to rounding; the work, and therefore the speed, depends on
 * the run lengths of the data. FP32-SIMT only (another precision with the
 * shortcut returns HMM_EUNSUPPORTED); n_min in 1..16384, else HMM_EINVAL.
 * Not part of the paper's algorithm.
 */

/* Default options: FP32-SIMT, emit-first, automatic chunking, renorm every 4. */
void hmm_opts_default(hmm_opts *opts);

/* Create a context bound to CUDA device `device` (it becomes current on the calling thread). */
int hmm_create(hmm_ctx **ctx, int device);

/* Free the context's device workspace. NULL is accepted. */
int hmm_destroy(hmm_ctx *ctx);

/* Text of the last error on this context (never NULL). */
const char *hmm_last_error(const hmm_ctx *ctx);

/*
 * Synchronise `stream`, read and clear the context's device status word.
 * Returns HMM_OK, HMM_EINVAL (a parameter set or a flagged observation failed
 * its checks), HMM_ENUMERIC or HMM_ETIMEOUT.
 */
int hmm_status(hmm_ctx *ctx, void *stream);

/*
 * Posterior state probabilities of one sequence: the smoothing step that
 * follows the likelihood when tremor episodes are classified by hidden state
 * (the forward-backward algorithm; Rabiner, Proc. IEEE 1989, Section III-A).
 * gamma (device, T x K floats, row-major) receives
 * gamma[t][k] = P(s_t = k | o_0 .. o_{T-1}); *loglik (device double)
 * receives log L. Computed on the chunk structure of hmm_loglik, with the
 * same options (opts->precision chooses the chunk products): two scans over
 * the chunk products give the forward vector entering and the backward
 * vector leaving every chunk, then every chunk recomputes its steps in FP32
 * from both, normalising each vector every step. T >= 1. A zero likelihood
 * gives NaN rows.
 */
int hmm_posterior(hmm_ctx *ctx, const hmm_params *params, const hmm_obs *obs, const hmm_opts *opts,
                  float *gamma, double *loglik, void *stream);

/*
 * The most probable hidden path of one sequence (Viterbi; Rabiner 1989,
 * Section III-B) on the chunk structure: every chunk's max-plus product
 * (best log2 score from each entering to each leaving state, CUDA cores),
 * a scan over chunk boundaries in FP64 with back-pointers, then every chunk
 * re-runs its recursion from its entering state and traces the path back
 * from its leaving state. path (device, T int32) receives the states;
 * *score (device double) log p(path, o) (natural log, -inf if every path has
 * probability zero); *loglik (device double) log L. Ties go to the smallest
 * state; paths whose scores differ only by FP32 rounding may differ from an
 * FP64 evaluation. T >= 1, K <= 80. opts->precision is ignored.
 */
int hmm_viterbi(hmm_ctx *ctx, const hmm_params *params, const hmm_obs *obs, const hmm_opts *opts,
                int32_t *path, double *score, double *loglik, void *stream);

/*
 * Expected sufficient statistics of the hidden chain (the E-step of EM,
 * Baum-Welch; Rabiner 1989, Section III-C), from the same chunked forward-
 * backward pass as hmm_posterior, into `stats` (device, K*K + 8*K doubles):
 *   N[i][j] = sum_{t>=1} P(s_{t-1}=i, s_t=j | o)  (K*K, row-major)
 *   G0[k] = P(s_0 = k | o); Gs[k] = sum_t gamma_t(k);
 *   Gr[k] = sum over tremor steps of gamma_t(k);
 *   Sx, Sy, Sxx, Sxy, Syy [k] = the same sums weighted by x, y, x^2, xy, y^2
 * (K each, in this order after N). With the Fisher identity they give the
 * gradient of log L with respect to every parameter (for gradient-based
 * samplers), and an EM update. Chunk partial sums are added in chunk order
 * in FP64 (deterministic). *loglik (device) receives log L. T >= 2.
 */
int hmm_expected_stats(hmm_ctx *ctx, const hmm_params *params, const hmm_obs *obs, const hmm_opts *opts,
                       double *stats, double *loglik, void *stream);

/*
 * Gradient of log L with respect to every parameter of one parameter set,
 * for gradient-based fitting and samplers, by the Fisher identity: the
 * posterior expectation of the gradient of the complete-data log likelihood
 * of Section 2 (hidden path, transitions P, emissions of Eq.
 * "emission-matrix"), formed in FP64 on the device from the statistics of
 * hmm_expected_stats (same options, same chunked forward-backward pass).
 * grad (device, K*K + 7*K doubles) receives, in the order of hmm_params,
 *   d/dpi [K], d/dP [K*K] (row-major), d/dp_tremor [K], d/dmu [K*2],
 *   d/dcov [K*3] (sxx, sxy, syy; sxy enters both off-diagonal entries),
 * with pi and P differentiated as free entries (no simplex constraint) and
 * opts->init_mode choosing where pi enters; *loglik (device double) receives
 * log L. Terms whose expected count is zero contribute zero. T >= 2.
 */
int hmm_loglik_grad(hmm_ctx *ctx, const hmm_params *params, const hmm_obs *obs, const hmm_opts *opts,
                    double *grad, double *loglik, void *stream);

/*
 * One EM (Baum-Welch) iteration: the E-step statistics of hmm_expected_stats
 * and the M-step that maximises the expected complete-data log likelihood,
 *   P_ij = N_ij / sum_j N_ij, pi = G0 / sum G0, p_k = Gr_k / Gs_k,
 *   mu_k = (Sx_k, Sy_k) / Gr_k, Sigma_k = (second moments) / Gr_k - mu_k mu_k^T,
 * written as float32 parameters to pi_out [K], P_out [K*K], p_out [K],
 * mu_out [K*2], cov_out [K*3] (device; may not alias the inputs); a row of P
 * or a state whose expected count is zero keeps its input value. *loglik
 * (device double) receives log L of the INPUT parameters; the likelihood of
 * the output is never lower (EM's monotonicity), up to the arithmetic's
 * rounding. Emit-first convention only (HMM_EUNSUPPORTED otherwise). T >= 2.
 */
int hmm_em_step(hmm_ctx *ctx, const hmm_params *params, const hmm_obs *obs, const hmm_opts *opts, float *pi_out,
                float *P_out, float *p_out, float *mu_out, float *cov_out, double *loglik, void *stream);

/*
 * log L for one parameter set and one sequence (Eq. "likelihood func",
 * computed as Section "The likelihood algorithm" restructures it).
 * out_dev: device pointer to one double.
 */
int hmm_loglik(hmm_ctx *ctx, const hmm_params *params, const hmm_obs *obs,
               const hmm_opts *opts, double *out_dev, void *stream);

/*
 * Many proposals, many segments, one call (MCMC batch evaluation).
 *   n_prop parameter sets, stacked: pi [n_prop*K], P [n_prop*K*K], p_tremor
 *   [n_prop*K], mu [n_prop*K*2], cov [n_prop*K*3] (device).
 *   n_seg independent observation segments, shared by every proposal:
 *   segment s is xy/tremor[seg_offsets[s] .. seg_offsets[s+1]) and starts
 *   from pi. seg_offsets is a HOST array of n_seg+1 non-decreasing int64,
 *   seg_offsets[0] = 0.
 *   out_dev[q] (device, n_prop doubles) = sum over s of log L(q | segment s),
 *   summed in segment order.
 */
int hmm_loglik_batched(hmm_ctx *ctx, int32_t n_prop, int32_t K, const float *pi,
                       const float *P, const float *p_tremor, const float *mu,
                       const float *cov, int32_t n_seg, const int64_t *seg_offsets,
                       const float *xy, const uint8_t *tremor, const hmm_opts *opts,
                       double *out_dev, void *stream);

/*
 * hmm_loglik_batched with HOST buffers: copies the inputs into the context's
 * device staging area on `stream`, evaluates, copies out_host[n_prop] back
 * and synchronises `stream` before returning (pinned host memory makes the
 * copies asynchronous up to that point). Returns the device status as
 * hmm_status() would.
 */
int hmm_loglik_batched_host(hmm_ctx *ctx, int32_t n_prop, int32_t K, const float *pi,
                            const float *P, const float *p_tremor, const float *mu,
                            const float *cov, int32_t n_seg, const int64_t *seg_offsets,
                            const float *xy, const uint8_t *tremor, const hmm_opts *opts,
                            double *out_host, void *stream);

/*
 * Number of kernel launches the last hmm_loglik / hmm_loglik_batched call
 * issued on its stream (for launch accounting in benchmarks).
 */
int hmm_last_launch_count(const hmm_ctx *ctx);

/*
 * Chunk length the last call used (after automatic selection).
 */
int hmm_last_chunk_len(const hmm_ctx *ctx);

/*
 * Graph replay of the batched call (the schedule of Section "The likelihood
 * algorithm" as one CUDA graph; the paper has no counterpart). With it on
 * (the default), hmm_loglik_batched (and hmm_loglik) captures its launch
 * sequence into a CUDA graph on a stream of the context's own and launches
 * the graph into the caller's stream; a later call with the same shape,
 * segment offsets, options, parameter/observation/output pointers and
 * workspace replays that graph instead of launching the kernels one by one.
 * The inputs' contents may change between calls (the kernels read them when
 * the graph runs). Calls made while the caller's stream is itself being
 * captured, and calls with phase profiling on, launch directly. Results are
 * identical either way. `on` = 0 turns it off (and frees the graph);
 * returns HMM_OK or HMM_EINVAL for a null context.
 */
int hmm_set_call_graphs(hmm_ctx *ctx, int on);

/*
 * How the last hmm_loglik / hmm_loglik_batched call ran: 0 = kernels launched
 * directly, 1 = captured into a new graph and launched, 2 = an existing graph
 * replayed; -1 for a null context.
 */
int hmm_last_call_graph(const hmm_ctx *ctx);

/* ---- chunk-length tuning of the batched schedule ----
 *
 * Section "The likelihood algorithm" splits the matrix chain into chunks
 * without fixing their length. The chunk length L sets the schedule of
 * hmm_loglik_batched: how many chunk products (work items of the persistent
 * chunk kernels) there are, how many waves of them the GPU runs, and the size
 * of the product tree. The tile shapes are fixed by the hardware mapping
 * (M = 128 rows of tensor memory, N = the padded state count), so L is the
 * schedule's free parameter. With opts->chunk_len = 0 the library uses, in
 * this order: a chunk length the tuner stored for the call's shape, else
 * its cost model's choice. The result depends on L only through rounding;
 * for a fixed table it is bit-for-bit reproducible like every other call.
 *
 * The shape key of a stored entry is (device multiprocessor count, K,
 * precision, n_prop, n_seg, total chain steps = sum over segments of
 * max(0, T_s - 1), runlen_min). The table is process-wide and guarded by a
 * lock, so every context (and thread) sees the same entries.
 */

/*
 * The cost model's chunk length for a shape (what chunk_len = 0 uses when
 * nothing is stored): a multiple of 64 in [64, 16384]. Host computation
 * only; 0 for arguments out of range (K in 1..80, n_prop >= 1,
 * steps_total >= 0, n_sms >= 1, a precision the library offers for K).
 */
int32_t hmm_default_chunk_len(int32_t precision, int32_t n_prop, int32_t K, int64_t steps_total,
                              int32_t n_sms);

/*
 * The chunk lengths hmm_autotune_batched measures for a shape: the cost
 * model's choice, its neighbours at factors 2^(j/2) (j = -3..3) and, for the
 * tensor-core precisions, the shortest chunk length that fits each wave count
 * within two of the model's. Ascending, distinct multiples of 64 in
 * [64, min(16384, steps_total rounded up to 64)], at most 16. Writes at most
 * `cap` of them to out (host) and their number to *n_out. Host computation
 * only; HMM_EINVAL for arguments out of range (as above, cap >= 1).
 */
int hmm_tune_candidates(int32_t precision, int32_t n_prop, int32_t K, int64_t steps_total,
                        int32_t n_sms, int32_t *out, int32_t cap, int32_t *n_out);

/*
 * Measures hmm_loglik_batched at every candidate chunk length for this
 * call's shape and stores the fastest. The arguments are those of
 * hmm_loglik_batched (device pointers, host seg_offsets), with
 * opts->chunk_len = 0 (else HMM_EINVAL). Per candidate: one untimed call
 * (it builds the plan and grows the workspace), then `reps` (1..100) calls
 * between two CUDA events on `stream`; the time is their mean, without an
 * L2 flush. A candidate whose call fails with HMM_EINVAL or HMM_ENOMEM (too
 * many chunks for the tree, or no memory) is skipped; any other error
 * ends the tuning and is returned. The winner is stored in the table, then
 * evaluated once more, so out_dev (n_prop doubles) holds log L computed at
 * the winner and hmm_last_chunk_len() returns it. *chunk_len_out and
 * *ms_out (host, may be NULL) receive the winner and its milliseconds per
 * call. The context keeps the largest workspace any candidate needed.
 * Synchronises `stream`; do not call it during stream capture.
 */
int hmm_autotune_batched(hmm_ctx *ctx, int32_t n_prop, int32_t K, const float *pi, const float *P,
                         const float *p_tremor, const float *mu, const float *cov, int32_t n_seg,
                         const int64_t *seg_offsets, const float *xy, const uint8_t *tremor,
                         const hmm_opts *opts, int32_t reps, double *out_dev, int32_t *chunk_len_out,
                         double *ms_out, void *stream);

/* The stored chunk length for a shape key, or 0 in *chunk_len if none. Host only. */
int hmm_tune_lookup(int32_t n_sms, int32_t K, int32_t precision, int32_t n_prop, int32_t n_seg,
                    int64_t steps_total, int32_t runlen_min, int32_t *chunk_len);

/* Forget every stored chunk length. Host only. */
int hmm_tune_clear(void);

/*
 * Write the table to a text file: a '#' comment line, then one entry per
 * line, "n_sms K precision n_prop n_seg steps_total runlen_min chunk_len
 * ms_per_call". HMM_EINVAL if the file cannot be written.
 */
int hmm_tune_save(const char *path);

/*
 * Read such a file and add its entries (an entry replaces a stored one with
 * the same key). Blank lines and lines starting with '#' are skipped. The
 * file is checked whole first: a malformed line or an entry out of range
 * (chunk_len not a multiple of 64 in [64, 16384], K outside 1..80, an
 * unknown precision, ...) or an unreadable path gives HMM_EINVAL and loads
 * nothing.
 */
int hmm_tune_load(const char *path);

/* ---- per-phase device timing (benchmarks) ---- */
#define HMM_PHASE_PREP 0   /* parameter checks and constants          */
#define HMM_PHASE_PACK 1   /* observation packing                      */
#define HMM_PHASE_CHUNK 2  /* chunk products (Section "Step 3")        */
#define HMM_PHASE_TREE 3   /* combining the chunk products             */
#define HMM_PHASE_FINAL 4  /* head vector, FP64 log L, segment sum     */
#define HMM_PHASE_COUNT 5

/*
 * on != 0: every later call records CUDA events on its stream around each
 * phase and accumulates the elapsed milliseconds (the event reads
 * synchronise on those events at the start of the next call and in
 * hmm_profile_read). on == 0: stop recording. Enabling resets the totals.
 */
int hmm_profile_enable(hmm_ctx *ctx, int on);

/*
 * Accumulated milliseconds per phase (ms_out[HMM_PHASE_COUNT]) and the number
 * of calls recorded (*n_calls). Waits for the recorded events.
 */
int hmm_profile_read(hmm_ctx *ctx, double *ms_out, int *n_calls);

/* ---- Bayesian fitting: random-walk Metropolis-Hastings (Section "Monte Carlo Markov Chains") ---- */

/*
 * Prior settings (Section "Model priors", Appendix A, as read here):
 * Dirichlet(alpha_P) on every row of P, Dirichlet(alpha_pi) on pi,
 * Gamma(shape m^2/v, rate m/v) truncated to (0,1) on p_k with m = p_mean_lo
 * for k < K/2 and p_mean_hi otherwise, v = p_var; means uniform on the box
 * [box[0], box[1]] x [box[2], box[3]]; Sigma_k inverse-Wishart(iw_df, I_2).
 */
typedef struct {
    float alpha_P, alpha_pi;
    float p_mean_lo, p_mean_hi, p_var;
    float box[4];
    float iw_df;
} hmm_prior;

/* alpha_P = 0.01, alpha_pi = 1, means 0.1 / 0.9, variance 0.001, box [0,300]x[0,150] km, df = K */
void hmm_prior_default(hmm_prior *prior, int32_t K);

/*
 * Dimension of the unconstrained state theta for K states: K^2 + 6K - 1.
 * Layout: K(K-1) reference logits of the rows of P (row i, columns j != i,
 * the diagonal being the reference), K-1 reference logits of pi (state 0 the
 * reference), K logits of p_k, 2K means (x, y), 2K (log sigma_x, log
 * sigma_y), K atanh(rho).
 */
int32_t hmm_theta_dim(int32_t K);

/*
 * theta [n][D] (device, float) -> parameters in the layout hmm_loglik_batched
 * takes (device, float) and logprior[n] (device, double) = log prior density
 * + log Jacobian of the map (up to a theta-independent constant; -INFINITY
 * when a mean lies outside the box). prior may be NULL (defaults). 2 <= K <= 80.
 */
int hmm_theta_to_params(int32_t n, int32_t K, const float *theta, const hmm_prior *prior, float *pi,
                        float *P, float *p_tremor, float *mu, float *cov, double *logprior, void *stream);

typedef struct hmm_sampler hmm_sampler;

/*
 * n_chains independent random-walk Metropolis-Hastings chains on one GPU.
 * theta0: device [n_chains][D] starting states; step: device [D] proposal
 * standard deviations (theta' = theta + step * N(0, I)); seed keys the
 * Philox4x32-10 counter-based generator. The observations (device, as for
 * hmm_loglik_batched; seg_offsets is a host array and is copied) must stay
 * valid while the sampler lives. opts selects the likelihood precision the
 * Metropolis-Hastings rule works in; every acceptance ratio compares two
 * values of that one precision. With opts->recheck_fp32 != 0 and a
 * tensor-core precision, every hmm_mcmc_step call ends by re-evaluating the
 * chains' current states (the proposals they last accepted) with FP32-SIMT
 * chunk products into a separate FP32 report (hmm_sampler_fp32_report); the
 * stored values the chains compare are not replaced. The sampler owns its
 * device state and two private contexts on `device`.
 */
int hmm_sampler_create(hmm_sampler **sampler, int device, int32_t n_chains, int32_t K,
                       const hmm_prior *prior, const float *theta0, const float *step, uint64_t seed,
                       int32_t n_seg, const int64_t *seg_offsets, const float *xy,
                       const uint8_t *tremor, const hmm_opts *opts, void *stream);

int hmm_sampler_destroy(hmm_sampler *sampler);

/*
 * n_iter iterations of every chain (Section "Monte Carlo Markov Chains": a
 * proposal is accepted with probability min(1, ratio of likelihood x prior),
 * times the proposal's Hastings factor where it is not symmetric): propose,
 * evaluate the batched likelihood of all proposals, accept or reject
 * (log u < log posterior ratio, u from Philox). After the first iteration the
 * sampler runs each iteration as one CUDA graph replay. trace_logpost (device [n_iter][n_chains] float) and
 * trace_theta (device [n_iter][n_chains][D] float) receive the state after
 * each iteration when not NULL. Asynchronous on `stream`, except for a short
 * synchronisation at the start of the call.
 */
int hmm_mcmc_step(hmm_sampler *sampler, int32_t n_iter, float *trace_logpost, float *trace_theta,
                  void *stream);

/*
 * FP32 recheck of the accepted proposals: re-evaluates every chain's current
 * state (its last accepted proposal) with FP32-SIMT chunk products now, on
 * `stream`. loglik_fp32_out (device, n_chains doubles) receives those log
 * likelihoods and *max_abs_diff_dev (device double) the largest
 * |FP32 value - stored value| over the chains; either may be NULL. The
 * stored values (hmm_sampler_state's log likelihood and log posterior) are
 * not changed, so later acceptance ratios stay in the sampler's precision.
 */
int hmm_sampler_recheck(hmm_sampler *sampler, double *loglik_fp32_out, double *max_abs_diff_dev, void *stream);

/*
 * The most recent FP32 recheck (the automatic one at the end of an
 * hmm_mcmc_step call with opts->recheck_fp32, or hmm_sampler_recheck), copied
 * without evaluating anything; NaN before the first recheck. Arguments as for
 * hmm_sampler_recheck.
 */
int hmm_sampler_fp32_report(hmm_sampler *sampler, double *loglik_fp32_out, double *max_abs_diff_dev,
                            void *stream);

/*
 * Checkpoints. hmm_sampler_save writes, after the sampler's queued work and
 * `stream` have finished, everything the chains' future depends on to the
 * file `path`: the states theta, their log posteriors, log likelihoods and
 * log priors, acceptance counts, the proposal step sizes, the Philox seed and
 * iteration counter, the proposal kind, the t-walk's second points, the FP32
 * report and, with the learned proposal, the network's parameters,
 * standardisation, scale, lam and drift. hmm_sampler_load restores such a
 * file into a sampler created with the same n_chains, K and observation
 * layout (n_seg and total length are checked; the data themselves are the
 * caller's); with the learned proposal the sampler must already use a
 * network of the saved shape, which is overwritten. After a load the sampler
 * continues bit for bit as the saved one would have. HMM_EINVAL for an
 * unreadable or unwritable path, a file that is not a checkpoint, or a
 * mismatch; both synchronise `stream`.
 */
int hmm_sampler_save(hmm_sampler *sampler, const char *path, void *stream);
int hmm_sampler_load(hmm_sampler *sampler, const char *path, void *stream);

/* Copy the current states: theta [n_chains][D] (float), log posterior,
 * log likelihood (double), accepted-proposal counts (uint64); all device
 * pointers, each may be NULL. */
int hmm_sampler_state(hmm_sampler *sampler, float *theta_out, double *logpost_out, double *loglik_out,
                      unsigned long long *n_accept_out, void *stream);

/* Kernel launches per iteration (the CUDA graph's node count of kernels). */
int hmm_sampler_launches_per_iter(const hmm_sampler *sampler);

/* 1 when iterations replay a captured CUDA graph, 0 when they are launched
 * directly (before the second iteration, or if capture failed). */
int hmm_sampler_graph_active(const hmm_sampler *sampler);

/* ---- learned proposal (a small MLP trained on the random walk's history) ---- */

#define HMM_PROPOSAL_RW 0   /* theta' = theta + step * N(0, I)                        */
#define HMM_PROPOSAL_MLP 1  /* theta' ~ q(. | theta) given by an hmm_mlp (see below)   */
#define HMM_PROPOSAL_TWALK 2 /* the t-walk: two points per chain (hmm_sampler_set_twalk) */

typedef struct hmm_mlp hmm_mlp;

/*
 * The network: x = (theta - mean) / in_scale (d inputs) -> relu(W1 x + b1)
 * (hidden) -> relu(W2 h1 + b2) (hidden) -> W3 h2 + b3 = (f_mu, f_sig) (2d).
 * The proposal it defines is
 *   q(theta' | theta) = N(theta + lam scale gamma f_mu, diag((lam scale exp(f_sig))^2)),
 * f_sig clamped to [-6, 3]; Metropolis-Hastings adds the correction
 * log q(theta | theta') - log q(theta' | theta), so the chain's target (the
 * posterior of Section "Monte Carlo Markov Chains") is unchanged.
 * Parameters live on the device, FP32, flattened as W1 [hidden][d], b1,
 * W2 [hidden][hidden], b2, W3 [2d][hidden], b3. Created with He-uniform
 * weights (Philox, `seed`), zero biases, a small last layer, mean 0,
 * in_scale 1, scale 1.
 */
int hmm_mlp_create(hmm_mlp **mlp, int32_t d, int32_t hidden, uint64_t seed, void *stream);
int hmm_mlp_destroy(hmm_mlp *mlp);
int64_t hmm_mlp_num_params(const hmm_mlp *mlp);

/* Copy the flattened parameters to (set = 0) or from (set = 1) params_dev. */
int hmm_mlp_params(hmm_mlp *mlp, float *params_dev, int set, void *stream);

/* Input standardisation (device mean[d], in_scale[d]), proposal scale (device
 * scale[d]) and the global step factor lam > 0. */
int hmm_mlp_set_scaling(hmm_mlp *mlp, const float *mean_dev, const float *in_scale_dev, const float *scale_dev,
                        float lam, void *stream);

/* Raw outputs (f_mu, f_sig) for B states: theta [B][d] -> out [B][2d] (device). */
int hmm_mlp_forward(hmm_mlp *mlp, int32_t B, const float *theta, float *out_dev, void *stream);

/*
 * Training loss on B pairs (theta_b, y_b), y being a later state of the same
 * chain: loss = mean_b sum_i ((y - theta)_i / scale_i - f_mu,i)^2 /
 * (2 exp(2 f_sig,i)) + f_sig,i (the negative log density of y under q with
 * lam = 1, without constants). Writes the loss (device double) and keeps the
 * gradient wrt every parameter; grads_dev (device, num_params floats) may be
 * NULL or receives a copy.
 */
int hmm_mlp_loss_grad(hmm_mlp *mlp, int32_t B, const float *theta, const float *y, double *loss_dev,
                      float *grads_dev, void *stream);

/* One Adam step (bias-corrected) with the gradient of the last hmm_mlp_loss_grad. */
int hmm_mlp_adam_step(hmm_mlp *mlp, float lr, float beta1, float beta2, float eps, void *stream);

/*
 * Set the scalings from n training pairs (X[n][d], Y[n][d], device): mean and
 * in_scale = column means and standard deviations of X, scale = column
 * standard deviations of Y - X; and the proposal's step factor lam.
 */
int hmm_mlp_fit_scaling(hmm_mlp *mlp, int32_t n, const float *X, const float *Y, float lam, void *stream);

/* Change the step factor lam > 0 and the drift factor gamma >= 0 (created: 1, 1). */
int hmm_mlp_set_lambda(hmm_mlp *mlp, float lam, float gamma);

/*
 * n_steps Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr),
 * each on `batch` pairs drawn with replacement (Philox, `seed`) from X/Y
 * (device [n][d]). loss_trace (device double [n_steps], may be NULL) gets
 * each step's minibatch loss. Synchronises `stream` before returning.
 */
int hmm_mlp_train(hmm_mlp *mlp, int32_t n, const float *X, const float *Y, int32_t n_steps, int32_t batch,
                  float lr, uint64_t seed, double *loss_trace, void *stream);

/*
 * Switch a sampler's proposal (HMM_PROPOSAL_RW or HMM_PROPOSAL_MLP with an
 * mlp whose d is the sampler's theta dimension; the sampler reads the
 * network at every iteration, so keep it alive and do not train it while the
 * sampler runs). The next hmm_mcmc_step captures a new graph.
 */
int hmm_sampler_set_proposal(hmm_sampler *sampler, int32_t kind, hmm_mlp *mlp);

/* ---- allocation-free variant ---- */
#define HMM_NOALLOC_MAX_K 32             /* largest state count it accepts  */
#define HMM_NOALLOC_MAX_T (1LL << 20)    /* longest sequence it accepts     */

/*
 * hmm_loglik without any device allocation (the paper has no counterpart:
 * this is a library concern).
 *
 * For callers that cannot allocate device memory during the call: code that
 * runs inside a framework owning every allocation, services whose device
 * footprint must stay fixed, or code that must not risk the implicit device
 * synchronisation cudaMalloc/cudaFree can cause. There is no context: the
 * scratch space (about 13 MiB) is one file-scope __device__ array, created
 * when the library is loaded and held by every GPU that loads it until the
 * process exits. The caller passes inputs and output as for hmm_loglik.
 *
 * Computes what hmm_loglik computes with precision HMM_PREC_FP32_SIMT,
 * emit-first convention, chunk_len 1024 and renorm_every 4 (so it agrees
 * with hmm_loglik's default options, whose chunk length is chosen
 * automatically, within the FP32 tolerance, not bit for bit), for
 * 1 <= K <= HMM_NOALLOC_MAX_K and 0 <= T <= HMM_NOALLOC_MAX_T; anything
 * larger is rejected with HMM_EINVAL before any work is queued.
 * out_dev: device pointer to one double. A true zero likelihood gives
 * -INFINITY. There is no context whose status word hmm_status() could
 * read, so the call's last kernel reads the status on `stream` and writes
 * NaN to out_dev when the device found invalid parameter data, a flagged
 * observation with non-finite xy, a value outside the representable range
 * (an emission below 2^-65536 of the step's best state) or an expired wait:
 * a NaN result is this call's device-side error report.
 *
 * The first call on each device looks the scratch address up (with that
 * device current), so make it before any stream capture. Every call reuses
 * the same scratch and leaves its contents behind (the parts that must start
 * at zero are cleared on `stream`). Calls that overlap on the GPU race on
 * the scratch: order them (one stream) or use hmm_loglik with a context.
 * Returns HMM_OK, HMM_EINVAL (bad arguments or sizes) or HMM_ECUDA.
 */
int hmm_loglik_noalloc(const hmm_params *params, const hmm_obs *obs, double *out_dev,
                       void *stream);

/*
 * The t-walk (Christen & Fox, "A general purpose sampling algorithm for
 * continuous distributions (the t-walk)", Bayesian Analysis 2010), the
 * sampler the paper runs (Section "Monte Carlo Markov Chains"). Every chain
 * keeps a second point x'; an iteration moves one of the two (probability
 * 1/2 each) on a random coordinate subset (each coordinate with probability
 * min(D, 4)/D, drawn again while empty) by the traverse (0.4918), walk
 * (0.4918), blow (0.0082) or hop (0.0082) kernel with the other point as
 * reference (a_w = 1.5, a_t = 6), and accepts by the Metropolis-Hastings rule
 * with each kernel's factor. The step sizes of hmm_sampler_create are not
 * used. The chain's reported state, traces and recheck are the first point.
 *
 * hmm_sampler_set_twalk: theta2 = the second points (device [n_chains][D],
 * copied; must differ from the first points in every coordinate for the
 * blow and hop kernels to move); evaluates their log posterior on `stream`
 * (synchronised before returning) and switches the sampler to the t-walk.
 * hmm_sampler_twalk_state: the second points and their log posteriors
 * (device outputs, either may be NULL).
 */
int hmm_sampler_set_twalk(hmm_sampler *sampler, const float *theta2, void *stream);
int hmm_sampler_twalk_state(hmm_sampler *sampler, float *theta2_out, double *logpost2_out, void *stream);

/*
 * Failure-detection check (the paper has no counterpart): runs, on `device`,
 * one bounded wait of the kind every tensor-core kernel uses on its
 * mbarriers, on a barrier phase that nothing completes, with a limit of
 * limit_ms (0 < limit_ms <= 2000) measured in cycles at the rated clock.
 * Returns HMM_ETIMEOUT when the wait gave up, set the status bit and let the
 * kernel finish (the expected outcome), HMM_OK or HMM_EINVAL if it did not,
 * HMM_ECUDA on a runtime error. *waited_ms (host, may be NULL) receives the
 * time waited. Allocates two small buffers; synchronises the device.
 */
int hmm_check_bounded_wait(int device, double limit_ms, double *waited_ms);

/*
 * Measured FP32 FFMA throughput of `device` in TFLOP/s (written to *tflops,
 * a host pointer): the roofline denominator of the FP32-SIMT chunk kernel,
 * from a kernel of independent FFMA chains timed with CUDA events (best of
 * three after a warm-up, about 0.1 s). Allocates a small scratch buffer.
 * A measurement helper; the paper has no counterpart.
 */
int hmm_measure_fp32_peak(int device, double *tflops);

#ifdef __cplusplus
}
#endif

#endif /* HMM_GB300_H */
