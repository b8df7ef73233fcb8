/*
 * phylograd.h -- C ABI of the GB300 library for the phylogenetic log-likelihood and its
 * linear-time branch-length gradient (Ji et al., "Gradients do grow on trees", arXiv 1905.12146).
 *
 * One evaluation runs, on the GPU:
 *   1. P_{i,l} = e^{Q_i b_i r_l} for every branch i and rate category l (Section 2.1
 *      transition matrices; Section 2.5 rate categories): in FP64 for 4 states; for other state
 *      counts by uniformisation, FP64 powers and Poisson weights summed in FP32;
 *   2. the post-order (pruning) pass p_k = (P_i p_i) o (P_j p_j)   (Section 2.3);
 *   3. the site likelihoods L_p = sum_l w_l pi' p_root,l and logL = sum_p wt_p log L_p
 *      (Section 2.3 root inner product, Section 2.5 mixture, sites i.i.d. per Section 2.1);
 *   4. the pre-order pass q_i = P_i' [q_k o (P_j p_j)], q_root = pi   (Section 2.4) fused with
 *      the gradient dlogL/db_i = sum_p wt_p sum_l r_l w_l qt_i,l' Q_i P_{i,l} p_i,l / L_p
 *      (Section 2.5, with qt_i = q_k o (P_j p_j) the pre-order vector at the top of branch i,
 *      which equals the paper's q_i' Q_i p_i because e^{Qb} and Q commute)  and optionally the
 *      diagonal of the Hessian (Section 2.6, applied site by site).
 *
 * Conventions.  A problem has N >= 2 tips and n nodes, n = 2N-1 for a binary tree (fewer with
 * multifurcations, see pg_problem).  Tips are nodes 0..N-1, internal nodes N..n-1 in any order,
 * the root is the one node with parent -1 (the paper numbers tips 1..N and fixes the root at
 * 2N-1, Section 2.1).  A branch is named by its child node, so per-branch arrays have n entries
 * and the root entry is ignored (input) or 0 (output).  Below, "[2N-1]" reads "[n]".
 * All matrices are row-major doubles.  Every call returns a pg_status; no C++ exception crosses
 * this boundary.  The library owns all device memory it allocates; pointers passed in are
 * borrowed for the duration of the call (synchronous calls) or until the stream reaches the
 * enqueued work (asynchronous calls).
 */
#ifndef PHYLOGRAD_H
#define PHYLOGRAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pg_status {
    PG_OK = 0,
    PG_ERR_INVALID = 1,     /* malformed tree, negative/NaN branch length, bad Q row, ... */
    PG_ERR_OOM = 2,         /* device allocation failed or the context's HBM budget is full */
    PG_ERR_CUDA = 3,        /* a CUDA runtime call failed (pg_last_error has the text)    */
    PG_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                         */
    PG_ERR_NUMERIC = 5,     /* a site likelihood was 0, infinite or NaN                   */
    PG_ERR_UNSUPPORTED = 6  /* valid input outside what this build implements              */
} pg_status;

typedef struct pg_ctx pg_ctx;         /* one CUDA device + memory budget                      */
typedef struct pg_handle pg_handle;   /* one device-resident problem (tree, data, model)      */

typedef struct pg_options {
    int32_t device;             /* CUDA device ordinal                                       */
    int32_t patterns_per_tile;  /* site patterns per thread block; multiple of 32, 0=default */
    uint64_t hbm_budget_bytes;  /* cap on device bytes held by this context's handles; 0=none */
    uint32_t flags;             /* PG_FLAG_* below; 0 = defaults                              */
} pg_options;

/* Problems with any state count but 4 (2..64) run their products on the tensor cores (three-pass
 * TF32 with FP32 accumulation) unless this flag selects the CUDA-core (SIMT FP32) kernels. */
#define PG_FLAG_SIMT_MSTATE 1u

/* A 4-state FP64 problem evaluated alone runs its tree pass in a latency kernel that keeps each
 * block's per-pattern vectors in shared memory when they fit (about 200 KB per block at one block
 * per SM); this flag selects the kernel with the partials in device memory instead (comparisons). */
#define PG_FLAG_FP64_DEVICE_PARTIALS 2u

/* Storage and arithmetic of the partial likelihood vectors.  FP32: partials in FP32 with FP64
 * transition matrices split into FP32 hi/lo pairs, an exact-product form of the post-order
 * update and FP64 site likelihoods (the fast path; its error against FP64 is stated per result).
 * FP64: every partial and product in FP64 (for small problems, where latency and not memory
 * traffic bounds the evaluation, and where FP32 rounding noise is a larger share of logL). */
#define PG_PRECISION_FP32 0
#define PG_PRECISION_FP64 1

/*
 * A problem, as in Section 2.1 (all pointers are host pointers, read during pg_upload only).
 *   n_states m: 4 (nucleotides: the CUDA-core path, FP32 or FP64 partials) or any other m in
 *                          2..64 (amino acids, codons, ...: the general path, FP32 partials,
 *                          tensor-core products unless PG_FLAG_SIMT_MSTATE).  m > 64, or FP64
 *                          with m != 4, is rejected with PG_ERR_UNSUPPORTED; m < 2 with
 *                          PG_ERR_INVALID.
 *   n_categories C: 1..4 discrete rate categories (Section 2.5).
 *   n_nodes n              nodes of the tree: 2N-1 for the paper's binary tree (Section 2.1;
 *                          0 also means 2N-1), fewer when internal nodes have more than two
 *                          children (a multifurcation), at least N+1.  Tips are nodes 0..N-1,
 *                          internal nodes N..n-1.  Every per-node array of this problem, of b and
 *                          of the outputs then has n entries.
 *   parent[n]              parent node of each node, -1 for the root; every internal node has at
 *                          least two children.  A node with d > 2 children is evaluated as a
 *                          chain of d-2 added internal nodes joined by branches of length 0
 *                          (P = I, so likelihoods and the derivatives in every original branch
 *                          are those of the multifurcating tree); the added nodes are internal and
 *                          invisible to the caller.
 *   tip_states[N][P]       code of tip t at pattern p, selecting the tip's partial vector
 *                          (Section 2.1): a code y < m is the observed state y (the indicator
 *                          vector); m <= y < m + K selects row y - m of tip_partials (partially
 *                          observed data); a larger code is missing data (the all-ones vector).
 *   n_tip_partials K, tip_partials[K][m]
 *                          partial vectors of partially observed tips, e.g. the sets of an
 *                          ambiguity code or base-call likelihoods: finite and >= 0, each row
 *                          with a positive entry; K >= 0 with m + K <= 256 (K = 0: tip_partials
 *                          unused).  The device holds each row in FP32 scaled exactly by a power
 *                          of two (largest entry in [1, 2)) and adds the scales back to logL.
 *                          A 4-state problem with K > 0 runs on the general path (FP32 only).
 *   pattern_weights[P]     multiplicity of each site pattern, finite and >= 0.
 *   Q[n_models][m][m]      CTMC generators: off-diagonals >= 0, rows summing to 0 (|row sum| <=
 *                          1e-10 * max|Q|); neither reversibility nor stationarity is required.
 *   branch_model[n]        generator used on each branch (NULL: model 0 everywhere).
 *   root_freqs[m]          root state distribution pi (>= 0, sums to 1 within 1e-10), not
 *                          necessarily stationary.
 *   cat_rates[C]           rate multipliers r_l >= 0; cat_weights[C] probabilities (sum 1).
 *   precision              PG_PRECISION_FP32 or PG_PRECISION_FP64 (anything else: invalid).
 */
typedef struct pg_problem {
    int32_t n_tips;
    int32_t n_states;
    int32_t n_patterns;
    int32_t n_categories;
    int32_t n_models;
    int32_t precision;          /* PG_PRECISION_FP32 (0) or PG_PRECISION_FP64 (1), see below */
    const int32_t *parent;
    const uint8_t *tip_states;
    const double *pattern_weights;
    const double *Q;
    const int32_t *branch_model;
    const double *root_freqs;
    const double *cat_rates;
    const double *cat_weights;
    int32_t tip_stride;         /* row pitch of tip_states in bytes (>= n_patterns); 0 = n_patterns */
    int32_t n_tip_partials;     /* K: rows of tip_partials (0 = none)                              */
    const double *tip_partials; /* [K][m]                                                          */
    int32_t n_nodes;            /* n: nodes of the tree, 0 = 2N-1 (binary); fewer: multifurcations */
} pg_problem;

typedef struct pg_handle_info {
    int32_t n_tips, n_nodes, n_states, n_patterns, n_categories;
    int32_t n_levels;            /* tree height = number of level-synchronous steps per pass */
    int32_t n_tiles;             /* thread blocks per pass                                    */
    int32_t patterns_per_tile;
    uint64_t device_bytes;       /* device memory held by this handle                         */
    uint64_t stream_bytes;       /* algorithmic HBM bytes of one evaluation's partial streams */
    uint64_t flops;              /* algorithmic FP32 flops of one evaluation's two passes     */
} pg_handle_info;

/* Create a context on opt->device (NULL opt: device 0, defaults).  The context is not
 * thread-safe; use one per host thread.  Errors: PG_ERR_INVALID (bad options), PG_ERR_CUDA. */
pg_status pg_create(const pg_options *opt, pg_ctx **out);

/* Destroy a context and every handle still attached to it. */
pg_status pg_destroy(pg_ctx *ctx);

/* Validate a problem and copy it to the device (tree levels, tip codes, weights, Q, pi, rates),
 * allocating the partial-likelihood buffers it needs.  Errors: PG_ERR_INVALID (the problem breaks
 * a rule above), PG_ERR_UNSUPPORTED (m > 64, FP64 with m != 4 or with K > 0, C > 4, or more than
 * 2^30 nodes), PG_ERR_OOM (allocation or budget). */
pg_status pg_upload(pg_ctx *ctx, const pg_problem *pr, pg_handle **out);

/* Release a handle's device memory. */
pg_status pg_free(pg_handle *h);

/* Blocking evaluation with HOST pointers: b[2N-1] branch lengths (root entry ignored; each other
 * entry finite and >= 0), outputs logL (scalar), grad[2N-1], hess[2N-1] (diagonal of the Hessian
 * of logL in the branch lengths), site_logL[P]; any output may be NULL.  The first call on a
 * handle allocates a pinned host staging buffer (freed by pg_free); every call copies b in through
 * it with one copy, the requested outputs and the device status back with two, and waits on the
 * stream once.  Errors: PG_ERR_INVALID (bad b), PG_ERR_NUMERIC (a site likelihood 0 or not
 * finite; outputs are still written), PG_ERR_CUDA. */
pg_status pg_eval(pg_handle *h, const double *b, double *logL, double *grad, double *hess,
                  double *site_logL);

/* Asynchronous evaluation with DEVICE pointers on a CUDA stream (cudaStream_t passed as void*,
 * NULL = legacy default stream).  Same arrays as pg_eval.  Nothing is checked on the host after
 * enqueueing: an invalid b or a numeric failure is recorded on the device and reported by
 * pg_eval_status.  One evaluation per handle may be in flight at a time (the handle's partial
 * buffers are reused). */
pg_status pg_eval_async(pg_handle *h, const double *d_b, double *d_logL, double *d_grad,
                        double *d_hess, double *d_site_logL, void *stream);

/* Evaluate k problems in as few launches as possible (problems are grouped by category count;
 * each launch covers every tile of every problem in the group).  d_b[i], d_grad[i], d_hess[i]
 * are per-problem DEVICE pointers (d_grad/d_hess may be NULL, or have NULL entries);
 * d_logL[k] is one DEVICE array.  FP32 problems run every level below the root in level
 * kernels shared by the group (one launch per level index) and the root's level in the fused
 * kernel; FP64 problems run the fused kernel.  Results agree with separate pg_eval_async calls to
 * FP32 rounding order (the same parity bounds hold) and are identical for the same batch.
 * Errors: PG_ERR_INVALID (k < 0, a NULL handle, handles from different contexts). */
pg_status pg_eval_batch_async(pg_handle *const *hs, int32_t k, const double *const *d_b,
                              double *d_logL, double *const *d_grad, double *const *d_hess,
                              void *stream);

/* The two halves of pg_eval_async, for reverse-mode differentiation (a torch.autograd.Function
 * whose forward is the pruning and whose backward is the pre-order pass).
 *
 * pg_forward_async: the P build, the post-order pass (Section 2.3) and the root (Section 2.5
 * mixture): d_logL (DEVICE scalar) and optionally d_site_logL [P].  The post-order partials and
 * the per-pattern root values stay in the handle.
 *
 * pg_backward_async: the pre-order pass (Section 2.4), the branch gradient (Section 2.5) and the
 * Hessian diagonal (Section 2.6) from the partials that the last forward pass (or pg_eval*) on
 * this handle left, for the branch lengths of that pass.  The gradient written to d_grad [2N-1]
 * is multiplied by *d_gscale (DEVICE scalar, e.g. the upstream gradient of logL; NULL = 1);
 * d_hess is not scaled.  The levels near the root, whose partials the forward pass kept on chip
 * only, are recomputed.  Enqueue it on the forward's stream (or order the streams): it reads what
 * the forward wrote.  Any later forward or evaluation on the handle replaces those partials.
 * Errors: PG_ERR_INVALID (NULL handle, no forward pass enqueued on the handle yet). */
pg_status pg_forward_async(pg_handle *h, const double *d_b, double *d_logL, double *d_site_logL, void *stream);
pg_status pg_backward_async(pg_handle *h, const double *d_gscale, double *d_grad, double *d_hess, void *stream);

/* Batched forms of the two halves, grouped and launched as pg_eval_batch_async.  d_gscale is a
 * DEVICE array [k] (entry i scales problem i's gradient) or NULL. */
pg_status pg_forward_batch_async(pg_handle *const *hs, int32_t k, const double *const *d_b, double *d_logL,
                                 void *stream);
pg_status pg_backward_batch_async(pg_handle *const *hs, int32_t k, const double *d_gscale,
                                  double *const *d_grad, double *const *d_hess, void *stream);

/* Random-effects clock (Section 2.1: a branch length is the branch's rate times the time elapsed
 * along it; Section 5.1: the rate is a tree-wise mean mu times a branch effect eps_i):
 *     b_i = mu * eps_i * (t_i - t_parent(i)),   b_root = 0,
 * with node times t in forward time (a child is later than its parent; b_i < 0 is reported by
 * the evaluation as PG_ERR_INVALID).  For each of k problems (handle hs[i] supplies the tree)
 * d_eps[i], d_t[i], d_b[i] are DEVICE arrays [2N-1] (root entries ignored) and d_mu is a DEVICE
 * array [k].  pg_clock_lengths_async writes d_b. */
pg_status pg_clock_lengths_async(pg_handle *const *hs, int32_t k, const double *const *d_eps,
                                 const double *d_mu, const double *const *d_t, double *const *d_b,
                                 void *stream);

/* The chain rule of the branch gradient g = d_grad_b[i] (DEVICE [2N-1], e.g. from
 * pg_backward_async) through the clock above:
 *     d/d eps_i = mu dt_i g_i,   d/d rate_i = dt_i g_i,   d/d mu = sum_i eps_i dt_i g_i,
 *     d/d t_k = rate_k g_k - sum over the children c of k of rate_c g_c,
 * with dt_i = t_i - t_parent(i) and rate_i = mu eps_i; root entries are 0.  Outputs (DEVICE,
 * each may be NULL): d_grad_eps[i], d_grad_t[i], d_grad_rate[i] [2N-1] and d_grad_mu [k].  The
 * sum over branches for mu is taken in a fixed order (the same bits on every call).
 * Errors: PG_ERR_INVALID (NULL handle or input array). */
pg_status pg_clock_grad_async(pg_handle *const *hs, int32_t k, const double *const *d_eps, const double *d_mu,
                              const double *const *d_t, const double *const *d_grad_b,
                              double *const *d_grad_eps, double *d_grad_mu, double *const *d_grad_t,
                              double *const *d_grad_rate, void *stream);

/* ---- serving: continuous batching of requests (no counterpart in the paper; the workload of
 * independent logL + gradient requests that arrive over time) ----------------------------------
 *
 * A server owns one device arena and max_inflight slots (a CUDA stream each).  Requests queue in
 * arrival order; a worker thread admits the oldest while a slot and room in the arena are free,
 * evaluates each on its own slot with the launches of pg_eval_async (so its results are the same
 * bits whether it runs alone or among others) and retires it when its copies complete.  Requests
 * that arrive while others run are admitted as slots and memory free up and overlap with them on
 * the device.  max_inflight = 1 gives the plain path: one request at a time, no overlap. */
typedef struct pg_server pg_server;

typedef struct pg_server_options {
    int32_t max_inflight;   /* requests on the device at once (slots); 0 = 4                    */
    int32_t reserved;
    uint64_t arena_bytes;   /* device bytes for the requests' data; 0 = 60% of the free memory;
                               counted against the context's budget                             */
} pg_server_options;

typedef struct pg_request {
    const pg_problem *problem;   /* host; the struct and its arrays stay valid until completion  */
    const double *b;             /* host [2N-1] branch lengths                                   */
    double *logL;                /* host outputs, written at completion (each may be NULL)       */
    double *grad;                /* [2N-1]                                                       */
    double *hess;                /* [2N-1]                                                       */
} pg_request;

typedef struct pg_request_info {
    int32_t status;              /* the request's pg_status                                      */
    int32_t reserved;
    double submit_s, start_s, done_s;   /* steady-clock seconds since the server was created:
                                           submission, admission to the device, completion      */
} pg_request_info;

/* Errors: PG_ERR_INVALID (NULL ctx/out, max_inflight < 0), PG_ERR_OOM (arena larger than the
 * budget or than the device can give), PG_ERR_CUDA. */
pg_status pg_server_create(pg_ctx *ctx, const pg_server_options *opt, pg_server **out);
/* Queue a request (non-blocking); *ticket identifies it for pg_server_wait. */
pg_status pg_server_submit(pg_server *s, const pg_request *rq, uint64_t *ticket);
/* Block until the request completes, fill *info (may be NULL) and return its status (a problem
 * that cannot be uploaded, e.g. larger than the whole arena, completes with that error).  Each
 * ticket is waited for once. */
pg_status pg_server_wait(pg_server *s, uint64_t ticket, pg_request_info *info);
/* Finish every queued request, then release the arena, streams and threads. */
pg_status pg_server_destroy(pg_server *s);

/* Wait for the handle's last evaluation and return its device-side status (PG_OK,
 * PG_ERR_INVALID for a bad branch length, PG_ERR_NUMERIC for a failed site likelihood,
 * PG_ERR_TIMEOUT for a bounded wait that gave up). */
pg_status pg_eval_status(pg_handle *h);

/* Sizes and algorithmic traffic of a handle (for measurement). */
pg_status pg_get_info(const pg_handle *h, pg_handle_info *out);

/* Fixed device scratch used by pg_eval_noalloc, per GPU that loads this library (64 MiB). */
#define PG_NOALLOC_SCRATCH_BYTES (64u << 20)

/* One blocking evaluation of a small problem that allocates nothing: no cudaMalloc or cudaFree,
 * no allocating library call, no host heap.  The paper has no counterpart; this exists for callers
 * that cannot allocate when they evaluate (for example code that must not trigger an allocation's
 * device-wide synchronisation inside a latency-critical loop, or a plug-in whose host application
 * owns every device allocation).  The problem, b and the outputs are HOST arrays laid out as for
 * pg_upload / pg_eval; there is no handle.  Runs on the calling thread's current device, on
 * `stream` (NULL = legacy default stream), and returns when the results are on the host.
 * Every intermediate array lives in one fixed device array of PG_NOALLOC_SCRATCH_BYTES that each
 * GPU loading the library holds until the process exits; host-side planning uses fixed static
 * buffers (inputs up to 4 MiB and outputs up to 1 MiB go through static host images with one copy
 * each way; larger ones array by array).  FP64 problems with at most 16 patterns per block at one
 * block per SM run the shared-memory latency kernel, as pg_eval does.  The first call on a device
 * looks up that array's device address (set-up), so make it
 * before any stream capture.  All calls share the array and the static buffers: calls that
 * overlap, on the GPU or from several host threads, race and must be serialised by the caller.
 * Errors: PG_ERR_UNSUPPORTED when the problem needs more scratch than PG_NOALLOC_SCRATCH_BYTES, has
 * more than 8192 tips or 64 models, m != 4, C > 4 or tip partial vectors (K > 0); otherwise as
 * pg_upload and pg_eval. */
pg_status pg_eval_noalloc(const pg_problem *pr, const double *b, double *logL, double *grad,
                          double *hess, double *site_logL, void *stream);

/* Device time of one evaluation's phases, summed over every evaluation since timing was enabled.
 * Phases, in launch order: FP64 transition matrices; post-order levels run one launch per level
 * (the wide levels near the tips); the fused kernel (the remaining levels, the root and their
 * pre-order steps); pre-order levels run one launch per level; the per-branch reduction.  The
 * *_bytes fields are the algorithmic HBM bytes of one evaluation's phase (partials, log2 scales and
 * tip codes each read or written once). */
typedef struct pg_phase_times {
    double pmatrix_ms, post_levels_ms, fused_ms, pre_levels_ms, reduce_ms, total_ms;
    int32_t evals;                     /* evaluations summed                                  */
    int32_t launches_per_eval;         /* kernels one evaluation launches                     */
    uint64_t post_levels_bytes, fused_bytes, pre_levels_bytes;
} pg_phase_times;

/* Per-phase timing of this handle's full evaluations: CUDA events recorded on the evaluation's
 * stream (asynchronously, no host synchronisation).  enable: 0 off; 1 at the six phase boundaries
 * (every field of pg_phase_times); 2 around the pre-order levels only (pre_levels_ms and evals; the
 * other times stay 0); 3 as 2 on every 8th full evaluation from the call (evals counts those).  A
 * timed event waits for all earlier work on the stream, so it also ends the programmatic overlap of
 * the kernels on either side and stalls the stream for a few microseconds: mode 1 changes the
 * evaluation's own duration most, mode 3 least.  Setting a mode clears the accumulated times.
 * Errors: PG_ERR_INVALID (NULL handle, enable not 0..3), PG_ERR_UNSUPPORTED (a problem evaluated in
 * pattern chunks). */
pg_status pg_set_phase_timing(pg_handle *h, int enable);

/* Waits for the timed evaluations and returns their summed phase times. */
pg_status pg_get_phase_times(pg_handle *h, pg_phase_times *out);

/* Static text for a status code. */
/* Failure-detection self-test.  Every kernel's device-side waits are bounded.  A wait that gives
 * up records a status bit, lets its own copies land, frees its tensor memory and returns.  The
 * host then reports PG_ERR_TIMEOUT instead of the GPU hanging.  This call runs that bounded wait
 * on the context's device on an mbarrier that nothing arrives at.  limit_cycles is the wait's
 * limit in SM clock cycles, in [1000, 2^32]; the library's own kernels use ~1 s.  Returns
 * PG_ERR_TIMEOUT when the wait gave up as intended, and the context stays usable.  Errors:
 * PG_ERR_INVALID (NULL context, limit out of range), PG_ERR_OOM, PG_ERR_CUDA. */
pg_status pg_selftest_timeout(pg_ctx *ctx, uint64_t limit_cycles);

const char *pg_status_string(pg_status s);

/* Text of the last error raised on the calling thread ("" if none). */
const char *pg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PHYLOGRAD_H */
