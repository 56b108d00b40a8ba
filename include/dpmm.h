/*
 * dpmm.h -- C ABI of the GB300 Para-DPMM sampler (Duan, Pinto & Xie,
 * "Parallel Clustering of Single Cell Transcriptomic Data with Split-Merge
 * Sampling on Dirichlet Process Mixtures", arXiv 1812.10048).
 *
 * One context holds one chain of the sampler for one cells x genes UMI count
 * matrix on one GPU.  All device memory is owned by the library.  Calls that
 * launch work are asynchronous on the context's stream unless stated; calls
 * that return data to the host synchronise that stream.
 *
 * Pointers: every array argument may be a host pointer (pageable or pinned)
 * or a device pointer of the current device; the library copies with
 * cudaMemcpyDefault and keeps no reference to caller memory after the call
 * returns (and, for device pointers, after the stream work it enqueued).
 *
 * Errors: every int-returning call returns DPMM_OK (0) or a negative code;
 * dpmm_last_error() then gives a thread-local message.  No C++ exception
 * crosses this boundary.  After DPMM_ECUDA the context should be freed.
 *
 * Notation follows the paper: x_i^u is the count of gene u in cell i, V (here
 * D) genes, N cells, K clusters, DP concentration alpha, symmetric Dirichlet
 * hyper-parameter lambda (here beta), sub-cluster quantities with a bar.
 */
#ifndef DPMM_H
#define DPMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DPMM_OK 0
#define DPMM_EINVAL -1      /* bad argument or malformed CSR */
#define DPMM_ENOMEM -2      /* device or host allocation failed */
#define DPMM_ECUDA -3       /* a CUDA call failed */
#define DPMM_ECAPACITY -4   /* K would exceed kmax (splits are rejected instead) */
#define DPMM_EOVERFLOW -5   /* a 32-bit gene-count statistic would wrap */
#define DPMM_ETIMEOUT -6    /* a bounded device-side wait gave up */
#define DPMM_ESTATE -7      /* call not valid in the context's current state */

#define DPMM_ENGINE_AUTO 0      /* pick per sweep from K and the count density (measured) */
#define DPMM_ENGINE_CSR_FP32 1  /* warp-per-cell CSR contraction, FP32 */
#define DPMM_ENGINE_TILE_BF16 2 /* dense 128-cell tiles on tcgen05, BF16 hi/lo; needs
                                   the packed entries (D <= 65,536 genes, every count
                                   <= 65,535) and 1 <= K <= 40: a sweep outside that
                                   runs the CSR engine (dpmm_debug_engine tells) */

typedef struct dpmm_ctx dpmm_ctx;

typedef struct dpmm_opts {
    int32_t kmax;      /* cluster capacity, 1..1024 (default 256) */
    int32_t engine;    /* DPMM_ENGINE_* (default AUTO) */
    int32_t split_q;   /* 1 (default): split ratio includes -sum_i log q_i */
    int32_t chain_id;  /* 0 .. 2^24-1, enters every Philox counter */
    uint64_t seed;     /* Philox key (default 42) */
    int32_t hastings;  /* split ratio: 0 (default) theta and pi integrated out (eq. 9,
                          14, 16 in lgamma sums); 1 eq. 18 with theta and pi
                          instantiated from the latest sweep's draws (see
                          dpmm_split_merge); merges use the integrated form */
    int32_t open_new_cluster;  /* 1: every sweep offers the K+1 candidate of
                          eq. 4 (theta, theta-bar from the Dirichlet(beta)
                          prior, weight pi_{K+1}); the cells that choose it
                          form one new cluster.  0 (default): labels range over
                          the K existing clusters (new clusters come from splits) */
    int32_t local_iters;  /* local Gibbs iterations per sweep, 1 (default, the
                          paper's choice) .. 16; 0 reads as 1.  Iterations after
                          the first hold the labels, redraw theta-bar (eq. 19)
                          and then every sub-label (eq. 8); the split proposal
                          term is the last iteration's.  Needs hastings = 0. */
    int32_t reserved[5];
} dpmm_opts;

/* Fill *opts with the defaults above. */
void dpmm_default_opts(dpmm_opts* opts);

/*
 * Create a chain for the N x D count matrix given in CSR form (rows = cells,
 * columns = genes; Section 2.1 stores the same UMI matrix as V x N).
 *   indptr  int32[N+1], non-decreasing, indptr[0] = 0, indptr[N] = nnz
 *   indices int32[nnz], 0 <= indices < D (any order within a row)
 *   data    int32[nnz], counts >= 0
 * alpha > 0 (DP concentration), beta > 0 (eq. 28 lambda).  opts may be NULL.
 * stream: a cudaStream_t to run on, or NULL for a stream owned by the context.
 * The three arrays may be host or device memory: they are copied once on the
 * context's stream (device arrays must be complete before the call), then
 * validated and turned into the packed and blocked copies on the device.
 * The chain starts with K = 1 (all cells in cluster 0) and fair-coin
 * sub-labels.  Errors: DPMM_EINVAL (malformed CSR, D < 1, N < 1, alpha or
 * beta not positive, kmax out of range), DPMM_EOVERFLOW (a gene whose counts
 * sum to 2^32 or more; a blocked copy above 2^31 - 1 entries), DPMM_ENOMEM,
 * DPMM_ECUDA.  Synchronises the stream before returning.
 */
int dpmm_init(dpmm_ctx** out, const int32_t* indptr, const int32_t* indices,
              const int32_t* data, int64_t N, int32_t D, double alpha, double beta,
              const dpmm_opts* opts, void* stream);

/* Release every resource of the context (NULL is ignored). */
void dpmm_free(dpmm_ctx* ctx);

/*
 * A batch of B independent chains (datasets of uneven size sharing D genes),
 * stepped together: every kernel of a dpmm_step / dpmm_sweep /
 * dpmm_split_merge on the batch is ONE launch over all chains (rows, tiles
 * and proposals of all chains dealt to one grid), replayed from one CUDA
 * graph.  Chain b is a full chain (as from dpmm_init) with its own data
 * (indptr[b], indices[b], data[b] of N[b] cells), alpha[b], beta[b], and the
 * random stream of chain_id = opts->chain_id + b; it evolves exactly as that
 * single chain would.  All chains share opts otherwise and the batch's stream
 * (stream, or a new one when NULL).  Paper: the sampler of §2 run for many
 * datasets at once; the batching itself has no counterpart in the paper.
 * Errors as dpmm_init (the first failing chain's).
 */
int dpmm_init_batch(dpmm_ctx** out, int32_t B, const int32_t* const* indptr,
                    const int32_t* const* indices, const int32_t* const* data, const int64_t* N,
                    int32_t D, const double* alpha, const double* beta, const dpmm_opts* opts,
                    void* stream);

/*
 * Chain b of a batch (for a single-chain context: itself, b = 0), for every
 * per-chain call (dpmm_labels, dpmm_get_state, dpmm_set_state, ...; those
 * calls reject a batch context with DPMM_EINVAL).  The handle belongs to the
 * batch: dpmm_free on it does nothing, and it is freed with the batch.
 * dpmm_step / dpmm_sweep / dpmm_split_merge on it step that chain alone.
 */
int dpmm_chain(dpmm_ctx* batch, int32_t b, dpmm_ctx** chain);

/*
 * n_sweeps blocked sweeps of eq. 4 (pi, theta, theta-bar from their Dirichlet
 * posteriors, eq. 19; every label from pi_k p(x_i | theta_k) and every
 * sub-label from eq. 8; Sections 2.1-2.3), each followed by removal of empty
 * clusters.  Asynchronous.
 */
int dpmm_sweep(dpmm_ctx* ctx, int32_t n_sweeps);

/*
 * One move of the split/merge MCMC (Sections 2.3-2.4): mode 1 runs the split
 * chain (every cluster proposes the split given by its sub-labels, accepted
 * by eq. 7 with the lgamma-sum likelihood ratio and q(S*|S) from eq. 8),
 * mode 2 the merge chain (random disjoint pairs, eq. 7 with the eq. 23
 * proposal ratio), mode 0 picks one of the two by a fair coin.  If
 * n_accepted is not NULL the call synchronises and stores the number of
 * accepted moves; otherwise it is asynchronous.
 * With opts.hastings = 1 a split's ratio is eq. 18 (eq. 14 times eq. 16)
 * with theta_{k0,k1} = theta-bar_{k,0/1} and pi_{kr} = pi_k n-bar_r / n_k,
 * taken from the draws of the latest dpmm_sweep / dpmm_step: a cluster is
 * proposed only if that sweep's compaction was the last change of the state
 * and kept its sub-labels; otherwise its log H is NaN and nothing is split.
 * Eq. 18 carries no density for drawing the new theta, so it favours every
 * split by thousands of nats at D ~ 1000 (use the default for sampling).
 */
int dpmm_split_merge(dpmm_ctx* ctx, int32_t mode, int32_t* n_accepted);

/*
 * n_steps iterations of (one sweep + one coin-selected split/merge move),
 * replayed from a CUDA graph captured on first use.  Asynchronous.
 */
int dpmm_step(dpmm_ctx* ctx, int32_t n_steps);

/* Copy the current labels (int32[N], in [0, K)) to out and K to *K_out
 * (either may be NULL).  Synchronises. */
int dpmm_labels(dpmm_ctx* ctx, int32_t* out, int32_t* K_out);

/*
 * Per-phase CUDA-event timing.  With enable = 1, every sweep and move records
 * events on the context stream (also inside the dpmm_step graph, which is
 * re-captured when the setting changes).  dpmm_phase_times()
 * returns the device time of each phase of the last step in ms (n <= 5
 * entries): [0] pi/theta draws (+ the dense-tile B operand), [1] the label
 * kernel (label + sub-label draw: the contraction of eq. 4 third line and
 * eq. 8), [2] statistics (+ the CSR fallback when the dense-tile engine is
 * built), [3] empty-cluster removal, [4] split/merge move.  dpmm_phase_times
 * synchronises.
 */
int dpmm_profile(dpmm_ctx* ctx, int32_t enable);
int dpmm_phase_times(dpmm_ctx* ctx, float* ms, int32_t n);

/*
 * Number of plans applied since dpmm_init: sweep compactions and split/merge
 * moves that changed some label or statistic (the others end right after
 * the plan).  Instrumentation only (the paper has no counterpart).
 * Synchronises.
 */
int dpmm_plans_applied(dpmm_ctx* ctx, int64_t* n);

/*
 * Label engine of the chain's latest sweep: *tile_used = 1 for the dense-tile
 * tensor-core engine, 0 for the FP32 CSR engine.  With DPMM_ENGINE_AUTO the
 * tile engine labels 1 <= K <= 40 clusters, except K <= 2 on count matrices of
 * density 12% or more, where the CSR engine was measured faster.
 * Instrumentation only (the paper has no counterpart).  Synchronises.
 */
int dpmm_debug_engine(dpmm_ctx* ctx, int32_t* tile_used);

/*
 * Launch tuning of a context (a single chain or a batch).  Each field picks how
 * a kernel of the step spreads its work over the GPU; 0 keeps the built-in
 * choice.  None of them changes any result (the same arithmetic in the same
 * order per cell, tile and cluster; integer statistics), so a tuned chain is
 * bit-identical to an untuned one.  The paper has no counterpart: these are
 * properties of this implementation, chosen by measurement (the Python
 * package's autotune module times the candidates and caches the fastest).
 *   stats_blocks_per_sm  statistics kernel blocks per SM: 1, 2, 4 or 8
 *                        (default 4 for one chain, 2 for a batch)
 *   tile_stages          dense-tile label kernel A/B stages: 2, or 4 (four
 *                        when they fit in shared memory, else two); default
 *                        4 for one chain, 2 for a batch
 *   tile_scatter         row entries a producer lane loads per batch: 8, 12 or
 *                        16 (default 12)
 *   draw_blocks_per_sm   parameter-draw kernel blocks per SM: 1 or 2 (default 2)
 *   local_lanes          lanes per cell of the local Gibbs sub-label kernel's
 *                        group form: 4, 8, 16 or 32 (default: the power of
 *                        two nearest below the mean row length / 8, within
 *                        [4, 32])
 *   local_stream         1: that kernel streams the rows through a shared-memory
 *                        ring (bulk copies) wherever the chain has the packed
 *                        rows and its theta-bar table leaves room; 0 (default):
 *                        lane groups read the rows from global memory
 * Other values: DPMM_EINVAL.  dpmm_set_tuning drops the captured step graph
 * (the next dpmm_step captures a new one).  dpmm_get_tuning returns the values
 * in force (defaults resolved).
 */
typedef struct dpmm_tuning {
    int32_t stats_blocks_per_sm;
    int32_t tile_stages;
    int32_t tile_scatter;
    int32_t draw_blocks_per_sm;
    int32_t local_lanes;
    int32_t local_stream;
    int32_t reserved[2];
} dpmm_tuning;

int dpmm_set_tuning(dpmm_ctx* ctx, const dpmm_tuning* tuning);
int dpmm_get_tuning(dpmm_ctx* ctx, dpmm_tuning* tuning);

/* Block until all work enqueued on the context's stream is done. */
int dpmm_sync(dpmm_ctx* ctx);

/* The context's cudaStream_t. */
void* dpmm_stream(dpmm_ctx* ctx);

/* Message of the last failed call on this thread ("" if none). */
const char* dpmm_last_error(void);

/* ---- state hooks (checkpoint / resume, parity tests) -------------------- */

/*
 * Read the chain state: labels int32[N], sub-labels uint8[N] (0/1), K, the
 * sweep counter t and the split/merge call counter m (any output may be
 * NULL).  Synchronises.
 */
int dpmm_get_state(dpmm_ctx* ctx, int32_t* labels, uint8_t* sub, int32_t* K,
                   int64_t* t, int64_t* m);

/*
 * Replace the chain state.  labels in [0, K) with every cluster non-empty,
 * sub-labels 0/1, 1 <= K <= kmax; t, m the counters.  sumlogq (double[K],
 * per-cluster sum of log q_i used by the next split proposal) may be NULL, in
 * which case n_k log(1/2) is used.  Statistics are recomputed on the device.
 * A resumed chain with the same seed continues bit-identically.
 */
int dpmm_set_state(dpmm_ctx* ctx, const int32_t* labels, const uint8_t* sub, int32_t K,
                   int64_t t, int64_t m, const double* sumlogq);

/*
 * Sufficient statistics of the current state: nsub uint32[K][2] (n-bar),
 * Ssub uint32[K][2][D] (gene sums per sub-cluster), sumlogq double[K]
 * (any may be NULL).  Synchronises.
 */
int dpmm_get_stats(dpmm_ctx* ctx, uint32_t* nsub, uint32_t* Ssub, double* sumlogq);

/* ---- phase hooks (the two halves of one sweep) --------------------------- */

/* First half of a sweep: draw log pi (K+1 entries) and log theta for the K
 * clusters and their 2K sub-clusters (eq. 4 first two lines, eq. 19).  With
 * opts.open_new_cluster (and K < kmax) it first appends the K+1 candidate as
 * an empty cluster: K grows by one until dpmm_assign's compaction, the
 * candidate's theta rows are prior draws, log pi_{K-1} is its alpha weight and
 * log pi_K = -inf.  Follow it with dpmm_assign. */
int dpmm_draw_params(dpmm_ctx* ctx);

/* Local Gibbs iteration j (1 <= j < 16) of Section 2.3 on the current state,
 * as a sweep with opts.local_iters > j runs it after its compaction: labels
 * held, theta-bar of every sub-cluster drawn from eq. 19 given the current
 * sub-labels (Philox tag 16 + 2 (j - 1)), then every sub-label from eq. 8
 * (tag 17 + 2 (j - 1)), both with step t - 1 (the sweep just made); n-bar,
 * S-bar and sum log q recounted.  DPMM_EINVAL if j is out of range, t = 0 or
 * the chain was built with opts.local_iters = 1.
 * Asynchronous after the check of t (which synchronises). */
int dpmm_local_gibbs(dpmm_ctx* ctx, int32_t j);

/* Second half: labels and sub-labels from the current parameters (eq. 4 third
 * line, eq. 8), statistics, empty-cluster removal; advances t. */
int dpmm_assign(dpmm_ctx* ctx);

/*
 * Current parameters: logpi float[K+1]; logtheta float[3K][D] with row 3k
 * for cluster k and rows 3k+1, 3k+2 for its sub-clusters 0 and 1.
 * Synchronises.
 */
int dpmm_get_params(dpmm_ctx* ctx, float* logpi, float* logtheta);
int dpmm_set_params(dpmm_ctx* ctx, const float* logpi, const float* logtheta);

/*
 * FP32 log-likelihood scores of selected cells under the current parameters,
 * computed by the same device code as the sweep's contraction:
 * out float[n][3K]: columns 0..K-1 hold log pi_k + sum_u x_i^u log theta_k^u
 * (eq. 4 third line with eq. 26), column K + 2k + r holds
 * sum_u x_i^u log theta-bar_{k,r}^u (the likelihood factor of eq. 8).
 * Synchronises.
 */
int dpmm_debug_scores(dpmm_ctx* ctx, const int32_t* cells, int32_t n, float* out);

/*
 * Dense-tile engine scores of every cell under the current parameters, from
 * the tensor-core contraction without changing the chain: out float[N][3K],
 * column k = sum_u x_i^u (log theta_k^u - m_u) and column K + 2k + r =
 * sum_u x_i^u (log theta-bar_{k,r}^u - m_u), where m_u is the mean of the 3K
 * log theta values of gene u (the centring the engine applies; it shifts a
 * cell's scores by a common constant).  DPMM_ESTATE if the engine is off or
 * K > 40.  Synchronises.
 */
int dpmm_debug_tile_scores(dpmm_ctx* ctx, float* out);

/*
 * The dense-tile engine's blocked copy of the counts, as dpmm_init built it on
 * the device: *T tiles of 128 cells, *C chunks of 64 genes, *n entries.
 * Entries are grouped by segment s = tile * C + chunk and, inside a segment,
 * by quarter q (32-cell row block), in CSR order inside a (segment, quarter)
 * bucket; entry = row-in-tile << 22 | gene-in-chunk << 16 | count; every
 * segment starts on a multiple of 4 entries (padding entries are 0).
 * tile_ptr int32[4 T C + 1]: tile_ptr[4 s + q] = first entry of bucket
 * (s, q), tile_ptr[4 T C] = *n.  With tile_ptr or tile_ent NULL only the sizes
 * are returned.  DPMM_ESTATE if the chain has no blocked copy.  Synchronises.
 */
int dpmm_debug_tile_layout(dpmm_ctx* ctx, int32_t* T, int32_t* C, int64_t* n, int32_t* tile_ptr,
                           uint32_t* tile_ent);

/* Split/merge diagnostics of the last dpmm_split_merge call: chain (1 split,
 * 2 merge), and log H per cluster (split; NaN where no proposal) or per pair
 * (merge, with the pair's cluster indices a < b in pair_ab int32[2][n]).
 * Arrays hold kmax entries.  Synchronises. */
int dpmm_debug_moves(dpmm_ctx* ctx, int32_t* chain, double* log_h, int32_t* pair_ab,
                     int32_t* n_entries);

/* ---- collapsed log marginal likelihood (empirical Bayes) ---------------- */

typedef struct dpmm_logml dpmm_logml;

/*
 * Statistics n_k, S_ku, T_k of fixed labels for the collapsed log marginal
 * likelihood (theta integrated out of eq. 12 against eq. 28 with a gene-wise
 * beta_u, pi out of eq. 10).  CSR as in dpmm_init, labels int32[N] in
 * [0, K); empty clusters are ignored.  stream as in dpmm_init.
 */
int dpmm_logml_create(dpmm_logml** out, const int32_t* indptr, const int32_t* indices,
                      const int32_t* data, int64_t N, int32_t D, const int32_t* labels,
                      int32_t K, void* stream);
void dpmm_logml_free(dpmm_logml* h);

/*
 * LML = K log alpha + lgamma(alpha) - lgamma(alpha+N) + sum_k lgamma(n_k)
 *     + sum_k [lgamma(B) - lgamma(B+T_k) + sum_u (lgamma(beta_u+S_ku) - lgamma(beta_u))]
 * with alpha = exp(log_alpha), beta = exp(log_beta) (float[D]), B = sum beta.
 * Summed in FP64 on the device.  logml is a host double (the call then
 * synchronises) or a device double (asynchronous on the handle's stream).
 */
int dpmm_logml_forward(dpmm_logml* h, double log_alpha, const float* log_beta, double* logml);

/*
 * Gradient of LML: *grad_log_alpha = K + alpha (psi(alpha) - psi(alpha+N)),
 * grad_log_beta[u] = beta_u sum_k [psi(B) - psi(B+T_k) + psi(beta_u+S_ku) - psi(beta_u)]
 * (float[D], FP32 digamma sums).  Each output may be host or device memory;
 * the call is asynchronous on the handle's stream when every output given
 * is device memory, else it synchronises.
 */
int dpmm_logml_backward(dpmm_logml* h, double log_alpha, const float* log_beta,
                        double* grad_log_alpha, float* grad_log_beta);

/*
 * The collapsed log marginal likelihood of dpmm_logml_forward and its
 * gradient (dpmm_logml_backward) for a sampler's data (derived from eq. 10
 * and eq. 12 with gene-wise beta, generalising the symmetric lambda):
 * labels == NULL takes the chain's current partition (its statistics, no
 * pass over the counts); otherwise labels is int32[N] (host or device) in
 * [0, K_labels).  log_beta float[D] (host or device).  Any output may be
 * NULL; logml and grad_log_alpha are host doubles, grad_log_beta float[D]
 * host or device.  Scratch is allocated on the first call and kept with the
 * context.  Synchronises.
 */
int dpmm_logml_grad(dpmm_ctx* ctx, const int32_t* labels, int32_t K_labels, double log_alpha,
                    const float* log_beta, double* logml, double* grad_log_alpha,
                    float* grad_log_beta);

/*
 * Replace the DP concentration alpha and the symmetric Dirichlet parameter
 * beta of a chain (the alpha of eq. 4's pi draw, the lambda of eq. 28) between
 * steps.  The chain's state is kept; the next step draws with the new values.
 * alpha, beta > 0 and finite, else DPMM_EINVAL; a batch or a batch member:
 * DPMM_EINVAL / DPMM_ESTATE.  Synchronises the context's stream.
 */
int dpmm_set_hyper(dpmm_ctx* ctx, double alpha, double beta);

/*
 * One empirical-Bayes step on (log alpha, log beta) for the chain's current
 * partition: gradient ascent on the collapsed log marginal likelihood of
 * dpmm_logml_grad, with beta tied across genes (its gradient is the sum of
 * the gene-wise ones, in FP64):
 *   log alpha += clamp(eta_alpha * dLML/dlog alpha, -max_step, max_step)
 *   log beta  += clamp(eta_beta  * sum_u dLML/dlog beta_u, -max_step, max_step)
 * then dpmm_set_hyper.  Alternating it with dpmm_step gives an empirical-Bayes
 * loop.  Outputs (host, may be NULL): the log ML before the step and the new
 * alpha and beta.  eta finite, max_step >= 0, else DPMM_EINVAL.  Synchronises.
 */
int dpmm_eb_step(dpmm_ctx* ctx, double eta_alpha, double eta_beta, double max_step,
                 double* logml, double* alpha_out, double* beta_out);

/*
 * Allocation-free variant of dpmm_logml_create + dpmm_logml_forward +
 * dpmm_logml_backward, for callers that cannot allocate device memory (for
 * example a framework whose caching allocator owns the GPU's memory, or
 * latency-critical code that must not call cudaMalloc / cudaFree, which
 * synchronise the device).  The paper has no counterpart: it is a property of
 * this library's interface, not of the method.
 *   indptr, indices, data, labels: DEVICE pointers of the current device (CSR
 *     as in dpmm_init, labels int32[N] in [0, K)); host memory or another
 *     GPU's memory returns DPMM_EINVAL; log_beta float[D], logml double,
 *     grad_log_alpha double and grad_log_beta float[D] may be host or device
 *     pointers.
 *   Limits: 1 <= D <= 65536, 1 <= K <= 1024, K * D <= 1048576; larger sizes
 *     return DPMM_EINVAL without touching the GPU.
 * Scratch lives in a static device array of about 4.6 MB that every GPU loading
 * the library holds until exit; no cudaMalloc, cudaFree or other allocating
 * routine is called.  All calls on a device share that array and it keeps the
 * last call's contents (each call clears what must start at zero): calls whose
 * GPU work overlaps race and must be serialised by the caller.  The first call
 * on a device looks up the array's device address (once per device).
 * Malformed CSR rows, columns or labels
 * are skipped on the device and reported as DPMM_EINVAL; a cluster whose
 * count of one gene reaches 2^32 gives DPMM_EOVERFLOW.  Runs on `stream`
 * (NULL: the legacy default stream) and synchronises it before returning.
 */
int dpmm_logml_grad_noalloc(const int32_t* indptr, const int32_t* indices, const int32_t* data,
                            int64_t N, int32_t D, const int32_t* labels, int32_t K,
                            double log_alpha, const float* log_beta, double* logml,
                            double* grad_log_alpha, float* grad_log_beta, void* stream);

/* ---- test hooks ---------------------------------------------------------- */

/* Philox4x32-10 words of the device generator: ctr uint32[n][4] -> out
 * uint32[n][4] with key (seed lo, seed hi).  Synchronises. */
int dpmm_debug_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n);

/* Tensor-core self-test: C[128][N] = A[128][Kd] * B[N][Kd]^T with BF16
 * operands (uint16 bit patterns) and FP32 accumulation, through the same
 * operand layout, descriptors and tensor-memory path as the dense-tile
 * engine.  Kd in {64, 128, 192, 256}, N a multiple of 16 in [16, 256].
 * Host or device pointers.  Synchronises. */
int dpmm_debug_tc_gemm(const uint16_t* A, const uint16_t* B, int32_t Kd, int32_t N, float* C);

/* The first n 4-word outputs of cuRAND's Philox4_32_10 generator after
 * curand_init(seed, 0, 0) (consecutive curand4 calls), out uint32[n][4]:
 * a library reference for the device generator.  Synchronises. */
int dpmm_debug_curand_philox(uint64_t seed, int64_t n, uint32_t* out);

#ifdef __cplusplus
}
#endif

#endif /* DPMM_H */
