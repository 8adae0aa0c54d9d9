/*
 * mcl.h -- C ABI of the GB300 (sm_103a) Markov Cluster expansion library.
 *
 * One MCL iteration (Algorithm 1 of Selvitopi, Hussain, Azad, Buluc,
 * "Optimizing High Performance Markov Clustering for Pre-Exascale
 * Architectures"): expansion B = A A (Alg. 1, expansion, "random walks from
 * all vertices performed as SpGEMM"), Prune (Alg. 1, Prune: drop entries
 * below a threshold and keep the top k of every column; recovery to a mass
 * fraction is this library's reading, below), inflation (Alg. 1, Hadamard
 * power) followed by column renormalisation, and the chaos measure used for
 * the loop's convergence test (Alg. 1, "while change in successive
 * iterations").  Clusters are the connected components of the final
 * matrix (Alg. 1, return).
 *
 * Matrices are square n x n in CSC (Section III-B: CSC is CSR of the
 * transpose, so column-wise products need no conversion):
 *   colptr  int64[n+1], nondecreasing, colptr[0] == 0, colptr[n] == nnz
 *   rowidx  int32[nnz], strictly increasing inside each column, in [0, n)
 *   val     float[nnz], finite and >= 0 (FP32)
 * Every array pointer in mcl_csc is DEVICE memory of the context's device.
 *
 * Prune rule (per column j of B, s = sum_i b_ij, entries ranked by value
 * descending, equal values by row ascending):
 *   t     = #{ i : b_ij >= threshold }
 *   m_rec = smallest m whose top-m mass reaches recover_pct * s
 *   m*    = min(K_rec, max(min(t, select_k), m_rec)),  K_rec = recover_k or select_k
 *   keep the top m* entries.
 * Inflation: a_ij = b_ij^r / sum_i b_ij^r over the kept entries (FP32 power,
 * FP64 column sum).  chaos_j = max(0, max_i a_ij - sum_i a_ij^2) in FP64;
 * chaos = max_j chaos_j.
 *
 * Precision: FP32 values and FP32 accumulation of the products; FP64 only
 * in the column sums and the chaos reduction.
 *
 * Ownership: the caller owns all inputs.  Outputs written into an mcl_csc
 * are allocated by the library with the context's allocator (see
 * mcl_create) and belong to the caller, who releases them with the matching
 * free.  Scratch space is owned by the context and reused across calls.
 *
 * Errors: every call returns an mcl_status; nothing is thrown across the
 * ABI.  After an error the context stays usable and mcl_last_error returns
 * a message.  Streams: every call is ordered on the given cudaStream_t
 * (passed as void*, NULL = legacy default stream).  Calls that must size an
 * output or return a host value synchronise that stream (noted per call).
 * A context must not be used by two host threads at once.
 */
#ifndef MCL_H_
#define MCL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MCL_OK = 0,
    MCL_ERR_INVALID = 1,        /* bad argument or malformed CSC */
    MCL_ERR_OOM = 2,            /* allocator returned NULL */
    MCL_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    MCL_ERR_TIMEOUT = 4,        /* a bounded device wait gave up */
    MCL_ERR_NOT_CONVERGED = 5,  /* mcl_run hit max_iters with chaos >= eps */
    MCL_ERR_INTERNAL = 6        /* a device-side consistency check failed */
} mcl_status;

typedef struct mcl_ctx mcl_ctx;

typedef struct {
    int32_t n;        /* rows == columns, 0 <= n <= 2^31 - 2 */
    int64_t nnz;      /* == colptr[n] */
    int64_t* colptr;  /* device int64[n+1] */
    int32_t* rowidx;  /* device int32[nnz] */
    float* val;       /* device float[nnz] */
} mcl_csc;

typedef struct {
    float threshold;      /* prune threshold theta (b >= theta survives) */
    int32_t select_k;     /* K: top-k kept per column, 1 <= K <= MCL_MAX_SELECT_K */
    float recover_pct;    /* p in [0, 1]: recovery mass fraction */
    int32_t recover_k;    /* K_rec cap on recovery; <= 0 means K */
    float inflation;      /* r > 0 (r = 2 in all of the paper's runs) */
    double chaos_eps;     /* mcl_run stops when chaos < chaos_eps */
    int32_t max_iters;    /* mcl_run iteration cap */
    int32_t use_estimator;/* 0: exact symbolic sizing; 1: learned estimator */
    int32_t batched;      /* mcl_run with comp_offsets: per-component stop */
} mcl_params;

#define MCL_MAX_SELECT_K 4096

/* Device allocator used for outputs and scratch: returns device memory of
 * at least `bytes` (256-byte aligned) or NULL; `stream` is the call's
 * stream.  NULL callbacks mean cudaMallocAsync / cudaFreeAsync. */
typedef void* (*mcl_alloc_fn)(size_t bytes, void* user, void* stream);
typedef void (*mcl_free_fn)(void* ptr, void* user, void* stream);

/* Per-call statistics of the last mcl_expand (or last mcl_run iteration). */
typedef struct {
    int64_t flops;            /* sum_j flops_j (multiply-adds), Section II notation */
    int64_t nnz_in;           /* nnz(A) */
    int64_t nnz_b;            /* nnz(A A) before pruning (exact, counted in the numeric pass) */
    int64_t nnz_out;          /* nnz after prune */
    int64_t estimator_misses; /* columns whose nnz exceeded the size estimate */
    int64_t range_splits;     /* row windows cut because their entries exceeded the capacity */
    double chaos;             /* max_j chaos_j */
    float ms_colstats, ms_estimate, ms_bin, ms_numeric, ms_compact, ms_chaos, ms_total;
    int32_t bins_used;
    int32_t iterations;
    int32_t phases;           /* column batches of the last mcl_expand */
    int32_t graph_replays;    /* iterations of the last batched mcl_run replayed as CUDA graphs */
    int32_t exact_from;       /* mcl_run with use_estimator: first iteration sized exactly because
                                 the learned estimates of an earlier one fell short on more than
                                 1/20 of its columns (0: none) */
    int32_t groups;           /* groups of components of the last mcl_run with comp_offsets
                                 (MCL_OPT_GROUP_BUDGET; 1 when it ran as one group) */
    int64_t flops_run;        /* last mcl_run: multiply-adds over all its iterations */
    int64_t alg_bytes_run;    /* last mcl_run: algorithmic bytes of its iterations, each
                                 8 nnz(A_t) + 8 flops + 8 nnz(A_t+1) + 16 n */
} mcl_stats;

/* Create a context on `device` (made current by every call).  alloc/free
 * may be NULL (see mcl_alloc_fn).  Returns MCL_ERR_INVALID for a bad device. */
mcl_status mcl_create(mcl_ctx** ctx, int device, mcl_alloc_fn alloc, mcl_free_fn release,
                      void* alloc_user);

/* Release the context and its scratch (synchronises the device). */
void mcl_destroy(mcl_ctx* ctx);

/* Message for the last failed call on ctx (static storage inside ctx). */
const char* mcl_last_error(mcl_ctx* ctx);

/* Library version string. */
const char* mcl_version(void);

/* Number of CUDA kernels this library has launched in this process, over
 * all contexts (for accounting; not synchronised with the device). */
int64_t mcl_launch_count(void);

/*
 * One fused MCL iteration: expansion B = A A, prune (threshold / top-k /
 * recovery), inflation and renormalisation, per-column chaos (Alg. 1,
 * expansion + Prune + inflation; the per-column fusion of expansion and
 * pruning follows Section II, "HipMCL fuses expansion and pruning").  The
 * unpruned B is never materialised.  A must be square; it need not be
 * column stochastic (the prune rule uses each column's own sum).
 * out: filled with a new CSC allocated by the context allocator (rows
 * sorted).  chaos: optional host pointer receiving max_j chaos_j.
 * Synchronises `stream` (to size the output).
 */
mcl_status mcl_expand(mcl_ctx* ctx, const mcl_csc* A, const mcl_params* prm, mcl_csc* out,
                      double* chaos, void* stream);

/*
 * The prune rule alone (Alg. 1, Prune, with the recovery reading above) on
 * an already materialised matrix B (square CSC): kept entries keep their B
 * values (no renormalisation).  out allocated as in mcl_expand.
 * Synchronises `stream`.
 */
mcl_status mcl_prune_select_recover(mcl_ctx* ctx, const mcl_csc* B, const mcl_params* prm,
                                    mcl_csc* out, void* stream);

/*
 * Inflation (Alg. 1, Hadamard power r) and column renormalisation, in
 * place on A's values: a_ij <- a_ij^r / sum_i a_ij^r (FP64 sum).  Columns
 * whose powers sum to 0 become 0.  Does not synchronise.
 */
mcl_status mcl_inflate_normalize(mcl_ctx* ctx, mcl_csc* A, float r, void* stream);

/*
 * chaos = max_j max(0, max_i a_ij - sum_i a_ij^2), FP64, written to the
 * host pointer `chaos` (the convergence measure for Alg. 1's loop test).
 * chaos_cols: optional device double[n] receiving chaos_j.
 * Synchronises `stream`.
 */
mcl_status mcl_chaos(mcl_ctx* ctx, const mcl_csc* A, double* chaos, double* chaos_cols,
                     void* stream);

/*
 * Connected components of the undirected pattern of A (Alg. 1, return):
 * labels (device int32[n]) receive the smallest vertex id of each vertex's
 * component.  Does not synchronise.
 */
mcl_status mcl_components(mcl_ctx* ctx, const mcl_csc* A, int32_t* labels, void* stream);

/*
 * Algorithm 1 to convergence: iterate mcl_expand until chaos < chaos_eps
 * or max_iters, then label clusters.  comp_offsets (HOST int32[ncomp+1],
 * or NULL) splits a block-diagonal A into independent components; with
 * prm->batched != 0 each component stops on its own chaos and its columns
 * are carried unchanged afterwards, while all still-active columns of all
 * components are expanded together in one pass per iteration.
 * labels: device int32[n].  iters: host, receives the iteration count (the
 * maximum over components).  chaos_hist: host double[max_iters] or NULL.
 * final_out: optional; receives the final matrix (allocated as in
 * mcl_expand).  Synchronises `stream` every iteration.  Returns
 * MCL_ERR_NOT_CONVERGED (with all outputs valid) when max_iters is reached.
 * Batched runs replay every iteration after the first as one CUDA graph on
 * a stream of the context (MCL_OPT_GRAPH; two replay buffers sized once by
 * sum_c |c| * min(|c|, K_rec)), ordered after `stream` and before the
 * labelling.  With prm->use_estimator, an iteration whose learned estimates
 * fall short on more than 1/20 of its expanded columns hands the rest of the
 * run to the exact symbolic sizing (mcl_stats.exact_from).
 */
mcl_status mcl_run(mcl_ctx* ctx, const mcl_csc* A0, const int32_t* comp_offsets, int32_t ncomp,
                   const mcl_params* prm, int32_t* labels, int32_t* iters, double* chaos_hist,
                   mcl_csc* final_out, void* stream);

/*
 * Exact symbolic expansion: flops_j = sum_{k in inds(A_*j)} nnz(A_*k) and
 * nnz_j = nnz((A A)_*j) for every column (Section II notation; the exact
 * memory estimate of Sections II and V, "symbolic SpGEMM").  flops and nnz_out are
 * device int64[n] (either may be NULL).  Does not synchronise.
 */
mcl_status mcl_symbolic(mcl_ctx* ctx, const mcl_csc* A, int64_t* flops, int64_t* nnz_out,
                        void* stream);

/*
 * Tuning options of a context (not part of the method):
 *   1 MCL_OPT_SIZING     -1 follow prm->use_estimator (default), 0 exact
 *                        symbolic pass, 1 the flops bound min(flops_j, span_j),
 *                        3 Cohen's estimate (mcl_cohen_estimate)
 *   2 MCL_OPT_CONF_MASK  bit mask of numeric-pass configurations (bit 0:
 *                        small CTA and window, bit 1: large; not 0)
 *   3 MCL_OPT_VALIDATE   1 (default) validate inputs
 *   4 MCL_OPT_EST_SCALE  multiply every size estimate by value/1000 (1000 =
 *                        unchanged); a deliberate mis-estimate exercises the
 *                        accumulator overflow path (results stay exact)
 *   5 MCL_OPT_ITERATION  iteration index fed to the estimator's features by
 *                        mcl_expand (default 1; mcl_run sets it itself)
 *   6 MCL_OPT_PHASE_BUDGET  bytes of output staging per column batch; when the
 *                        staging of all columns, sum_j min(K_rec, flops_j,
 *                        span_j) pairs of 8 bytes, exceeds it, mcl_expand runs
 *                        in consecutive column batches that each fit (the
 *                        phased expansion of Section II, one GPU); 0 = off
 *   7 MCL_OPT_COHEN_KEYS keys per vertex of Cohen's estimate (2..16, default 8)
 *   8 MCL_OPT_COHEN_SEED seed of Cohen's keys (default 2002)
 *   9 MCL_OPT_GRAPH      1 (default): a batched mcl_run (comp_offsets given,
 *                        prm->batched, exact or flops-bound sizing) replays
 *                        every iteration after the first as one CUDA graph
 *                        (one host synchronisation per iteration); 0: eager
 *  10 MCL_OPT_GRAPH_CAP  entries of each graph replay buffer; 0 (default):
 *                        sum over components of size * min(size, K_rec), an
 *                        upper bound on any later iteration.  An iteration
 *                        that would exceed it is redone without graphs.
 *  11 MCL_OPT_SMALL_MAX  columns estimated at <= value entries (0..512,
 *                        default 512) use the small numeric configuration
 *  12 MCL_OPT_TABLE      shape of the large numeric configuration (0..2)
 *  13 MCL_OPT_PLAN       entries planned per hashed window (0 = half the
 *                        table, at most 3072)
 *  14 MCL_OPT_GROUP_BUDGET  bytes of device memory one group of components
 *                        may use in an mcl_run with comp_offsets; 0 (default)
 *                        = one group.  Components needing more in total
 *                        (about 32 bytes per entry of size * min(size, K_rec)
 *                        plus 160 bytes per vertex) run in consecutive groups
 *                        of whole components, one group after the other.  A
 *                        batched run gives the same results as one run; a
 *                        run with prm->batched == 0 iterates each group until
 *                        that group's chaos drops below chaos_eps.
 *  15 MCL_OPT_BUCKET_BUDGET  bytes of device memory for the numeric pass's
 *                        per-window product buckets (default 32 GiB); columns
 *                        whose products do not fit a CTA's share walk their
 *                        sources with cursors instead (same results)
 * Returns MCL_ERR_INVALID for an unknown option or value.
 */
#define MCL_OPT_SIZING 1
#define MCL_OPT_CONF_MASK 2
#define MCL_OPT_VALIDATE 3
#define MCL_OPT_EST_SCALE 4
#define MCL_OPT_ITERATION 5
#define MCL_OPT_PHASE_BUDGET 6
#define MCL_OPT_COHEN_KEYS 7
#define MCL_OPT_COHEN_SEED 8
#define MCL_OPT_GRAPH 9
#define MCL_OPT_GRAPH_CAP 10
#define MCL_OPT_SMALL_MAX 11
#define MCL_OPT_TABLE 12
#define MCL_OPT_PLAN 13
#define MCL_OPT_GROUP_BUDGET 14
#define MCL_OPT_BUCKET_BUDGET 15
mcl_status mcl_set_option(mcl_ctx* ctx, int option, int64_t value);

/*
 * Learned output-size estimator (sizing without the symbolic pass).
 *
 * Each column j of A is described by 16 features computed in O(nnz(A_*j))
 * (column and referenced-column sizes, value mass, spans, iteration,
 * previous compression factor); a 16 -> 64 -> 64 -> 2 MLP with ReLU, BF16
 * weights and FP32 accumulation predicts y0 = log(1 + nnz((AA)_*j)) and
 * y1 = log cf_j (cf = flops / nnz, Section II notation).  It replaces the
 * exact symbolic SpGEMM (Sections II and V: the per-iteration memory
 * estimate) when sizing the accumulators; the exact pass remains available
 * (prm->use_estimator = 0, or mcl_symbolic) and judges the estimate.
 * Estimates never change results: an under-estimate narrows the numeric
 * pass's row ranges, an over-estimate widens its tables.
 *
 * Weights: MCL_MLP_NPARAM values laid out W1 [64 x 16] (row = output
 * unit), b1 [64], W2 [64 x 64], b2 [64], W3 [2 x 64], b3 [2], as BF16 bit
 * patterns (uint16).  norm: mu[16] then sigma[16] (FP32); the network sees
 * (x - mu) / sigma.  All pointers below are DEVICE pointers unless marked
 * host.  None of these calls synchronises.
 */
#define MCL_MLP_NPARAM 5378
#define MCL_NFEATURES 16

/* Install estimator weights (host arrays; copied) and the safety factor s
 * (estimate = ceil(expm1(y0) * s), clamped to [1, min(flops_j, span_j)]).
 * The weights come as arrays, not as a file path, so that the library does
 * no file I/O and needs no archive format: a caller reads its weight file
 * (the Python binding reads a .npz) and passes the BF16 bit patterns
 * (5378 values, layout as in the training kernels) and the standardisation
 * (16 means, then 16 standard deviations). */
mcl_status mcl_estimator_load(mcl_ctx* ctx, const uint16_t* w_bf16_host, const float* norm_host,
                              float safety);

/* Features of every column of A into feats (float[n * 16], row-major per
 * column).  iteration >= 1; prev_logcf: float[n] or NULL (feature 13 = 0). */
mcl_status mcl_features(mcl_ctx* ctx, const mcl_csc* A, int32_t iteration,
                        const float* prev_logcf, float* feats, void* stream);

/* MLP forward: out (float[n * 2]) = (y0, y1) for each row of feats. */
mcl_status mcl_mlp_forward(mcl_ctx* ctx, const float* feats, int64_t n, const uint16_t* w_bf16,
                           const float* norm, float* out, void* stream);

/* MLP backward for training: adds d/dw of scale * sum_samples sum_outputs
 * (y - target)^2 into grad (float[MCL_MLP_NPARAM]) and the unscaled sum
 * into *loss (double).  targets: float[n * 2]. */
mcl_status mcl_mlp_backward(mcl_ctx* ctx, const float* feats, const float* targets, int64_t n,
                            const uint16_t* w_bf16, const float* norm, float scale, float* grad,
                            double* loss, void* stream);

/* One Adam step (step >= 1) on FP32 master weights; writes their BF16
 * rounding (nearest even) into w_bf16.  m, v: float[MCL_MLP_NPARAM]. */
mcl_status mcl_adam_step(mcl_ctx* ctx, float* master, float* m, float* v, const float* grad,
                         int64_t step, float lr, float beta1, float beta2, float eps,
                         uint16_t* w_bf16, void* stream);

/* The size estimate the numeric pass would use with the loaded estimator
 * (iteration from MCL_OPT_ITERATION), into est (int64[n]). */
mcl_status mcl_estimate(mcl_ctx* ctx, const mcl_csc* A, int64_t* est, void* stream);

/*
 * Cohen's probabilistic output-size estimate (Section V): each row i of A
 * gets `keys` (r, 2..16) FP32 keys -ln(u) with u from splitmix64 at counter
 * seed + (i*r + l) * 0x9E3779B97F4A7C15 (top 53 bits + 1, over 2^53); the
 * minimum key l over each column's rows, then over each column's sources,
 * gives est_j = (r - 1) / sum_l min_l (0 for an empty column), the
 * estimate of nnz((AA)_*j), in O(r nnz(A)).  est: device float[n].
 * MCL_OPT_SIZING = 3 makes mcl_expand size its windows with it
 * (MCL_OPT_COHEN_KEYS, MCL_OPT_COHEN_SEED).  A is validated first (one
 * synchronisation; MCL_ERR_INVALID for a malformed A or keys outside 2..16).
 */
mcl_status mcl_cohen_estimate(mcl_ctx* ctx, const mcl_csc* A, int32_t keys, uint64_t seed,
                              float* est, void* stream);

/*
 * One MCL iteration with the inner dimension of the expansion split into
 * `nstages` blocks and the partial products combined by the binary merge
 * (Section IV, "Binary merge"; Algorithm 2).  Stage t forms, unpruned and
 * sorted by row, P_t = A(:, K_t) A(K_t, :) for the block K_t of rows
 * [(t-1) n / nstages, t n / nstages) of the right operand; P_t is pushed on
 * a stack, and when t is even the top nmerges + 1 lists are popped and
 * merged (summed) into one (nmerges = the number of times t halves evenly),
 * as in Algorithm 2; lists left on the stack at the end are merged last.
 * The merged B = A A is pruned, inflated and renormalised as mcl_expand does.
 * Partial products carry the exact fixed-point sums of mcl_expand (the same
 * per-column scale), so `out` equals mcl_expand's result bit for bit; the
 * point of the call is the merge schedule and its memory (stats).
 * nstages in [1, 4096].  out allocated as in mcl_expand; chaos: optional
 * host pointer.  stats: optional host pointer.  Synchronises `stream` after
 * every stage and merge (to size their outputs).
 */
typedef struct {
    int32_t stages;
    int32_t merges;                  /* merges of the binary schedule (the final one included) */
    int64_t partial_entries;         /* sum over stages of nnz(P_t): what a multiway merge holds */
    int64_t binary_peak_entries;     /* entries of the largest merge of the binary schedule */
    int64_t live_peak_entries;       /* most entries the binary schedule holds at once (stack,
                                        inputs and output of a merge) */
    int64_t merged_entries;          /* nnz(A A) */
} mcl_merge_stats;
#define MCL_SPLIT_MAX_STAGES 4096
mcl_status mcl_expand_split(mcl_ctx* ctx, const mcl_csc* A, const mcl_params* prm, int32_t nstages,
                            mcl_csc* out, double* chaos, mcl_merge_stats* stats, void* stream);

/* Statistics of the last mcl_expand / mcl_run on ctx. */
mcl_status mcl_get_stats(mcl_ctx* ctx, mcl_stats* stats);

/*
 * Allocation-free exact symbolic pass (the paper has no counterpart; it is
 * an interface for callers that cannot allocate device memory where they
 * need output sizes -- e.g. a service that reserves all of its GPU memory
 * in a pool at start-up and forbids allocation afterwards, because
 * cudaMalloc can synchronise the device and fail under fragmentation).
 *
 * Computes what mcl_symbolic computes -- flops_j and nnz((AA)_*j), device
 * int64[n] outputs supplied by the caller (either may be NULL, not both) --
 * without a context and without allocating: no cudaMalloc / cudaFree and no
 * allocator callback.  Its scratch is one file-scope device array of
 * MCL_NOALLOC_SCRATCH_BYTES (64 MiB), which every GPU that loads this
 * library holds until the process exits.  It needs 24 bytes per column
 * (so n up to about 2.79 million) plus cursor space for the longest
 * column; larger inputs are rejected with MCL_ERR_INVALID and a message in
 * errbuf (caller memory of errlen bytes, may be NULL).
 *
 * The first call on a device looks up the array's device address (with
 * that device current) and caches it; make that first call before any
 * stream capture.  Every call shares the one array, which keeps the last
 * call's contents (the call clears what must start at zero): calls that
 * overlap on the GPU -- on different streams or host threads -- race and
 * must be serialised by the caller.  Synchronises `stream` after the column
 * statistics (to check them and size the cursors) and, when nnz_out is
 * given, once more after the counting pass (to read its error flags).
 */
#define MCL_NOALLOC_SCRATCH_BYTES (64 * 1024 * 1024)
mcl_status mcl_symbolic_noalloc(const mcl_csc* A, int64_t* flops, int64_t* nnz_out, char* errbuf,
                                size_t errlen, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MCL_H_ */
