/*
 * cpapr.h -- C ABI of the GB300 (sm_103a) CP-APR MU library.
 *
 * CP-APR MU (Chi and Kolda's multiplicative-update Poisson CP decomposition,
 * Algorithm 1 of arXiv 2307.03276) factors a sparse count tensor X of size
 * I_1 x ... x I_N into a Kruskal model [lambda; A^(1) .. A^(N)] of rank R.
 * Its hot path is Phi^(n) (Algorithm 2):
 *     Phi^(n) = (X_(n) ./ max(B Pi^(n), eps)) (Pi^(n))^T,
 * evaluated one nonzero at a time (Algorithm 3): for nonzero x at
 * (i_1..i_N), pi = elementwise product of the rows A^(m)[i_m,:] (m != n),
 * v = x / max(<B[i_n,:], pi>, eps), Phi[i_n,:] += v pi.
 *
 * Conventions for every call:
 *  - All indices (modes, coordinates, rows) are 0-based.
 *  - Dense matrices are row-major: factor m is I_m x R, entry (i, r) at
 *    [i * R + r].  Phi and MTTKRP outputs are I_n x R the same way.
 *  - Pointers may be host (pageable or pinned) or device pointers; the
 *    library tells them apart through unified addressing.  Inputs are
 *    copied: the caller keeps ownership of every buffer it passes.
 *  - Outputs are complete when the call returns (the call synchronises its
 *    stream before returning).
 *  - Errors are returned as cpapr_status; no exception crosses the ABI.  A
 *    failed call leaves the context usable, except CPAPR_E_CUDA, which is
 *    sticky: every later call on that context returns CPAPR_E_CUDA.
 *    cpapr_last_error() gives a one-line message.
 *  - A context is not thread-safe: calls on one context must not overlap.
 *    Separate contexts are independent.
 */
#ifndef CPAPR_H
#define CPAPR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPAPR_MAX_MODES 8

typedef struct cpapr_ctx cpapr_ctx;

typedef enum {
    CPAPR_OK = 0,
    CPAPR_E_ARG = 1,     /* bad argument: NULL pointer, mode out of range, rank < 1, ... */
    CPAPR_E_RANGE = 2,   /* a coordinate outside [0, I_m) or a size too large */
    CPAPR_E_VALUE = 3,   /* a tensor value that is negative, NaN or infinite */
    CPAPR_E_NOMEM = 4,   /* a device or host allocation failed */
    CPAPR_E_CUDA = 5,    /* CUDA runtime error (sticky) */
    CPAPR_E_TIMEOUT = 6, /* a bounded device-side wait gave up */
    CPAPR_E_STATE = 7    /* call out of order, e.g. a solve before any model was set */
} cpapr_status;

enum { CPAPR_FP64 = 0, CPAPR_FP32 = 1 };
enum { CPAPR_REDUCE_AUTO = 0, CPAPR_REDUCE_ATOMIC = 1, CPAPR_REDUCE_SEGMENTED = 2 };
enum { CPAPR_PI_AUTO = 0, CPAPR_PI_FUSED = 1, CPAPR_PI_MATERIALISED = 2 };
enum { CPAPR_DOT_AUTO = 0, CPAPR_DOT_FP64 = 1, CPAPR_DOT_FP32_PIPE = 2 };

/*
 * Options.  Fill with cpapr_default_options() and change what you need.
 *  precision  CPAPR_FP64: every step in FP64 (the paper's precision).
 *             CPAPR_FP32: factors, B, Phi, gathers, Khatri-Rao products, dots
 *             and scales in FP32 with compensated (Kahan) row sums; FP64
 *             only for the KKT-violation maximum, the log-likelihood sum and
 *             the lambda / column normalisation.  Results are returned as FP64.
 *  reduction  how rows of Phi that span several tiles of nonzeros are summed:
 *             SEGMENTED writes per-tile partials and adds them in a fixed
 *             order (bit-reproducible); ATOMIC adds them with atomics.
 *  eps        minimum divisor of Algorithm 2 (default 1e-10).
 *  kappa, kappa_tol  inadmissible-zero shift S of Algorithm 1: S(i,r) = kappa
 *             when the outer iteration is not the first, A(i,r) < kappa_tol and
 *             the previous Phi(i,r) > 1 (defaults 0.01, 1e-10).
 *  seed       reserved for callers; cpapr_init_random takes its own seed.
 *  stream     a cudaStream_t to run on, or NULL for a stream the context owns.
 *  tile_nnz   nonzeros per tile (one thread block); 0 = automatic.  A
 *             multiple of 4 in [64, 2^20] whose staged index and value
 *             streams fit in shared memory (about 220 KB per block, e.g. at
 *             most 8192 for a 3-way FP64 tensor); E_ARG otherwise.
 *  rank_lanes lanes that share one nonzero (1..32, power of two); 0 = automatic.
 *  use_graph  1 = run each mode's inner loop as a CUDA graph with a device-side
 *             early exit (default), 0 = plain stream launches.
 *  autotune   1 = time candidate (tile_nnz, rank_lanes, reduction, pi_mode)
 *             choices on the tensor when it is created and keep the fastest
 *             per mode; 0 = use the built-in heuristic (default).  Each
 *             candidate is timed as a Phi of the MU inner loop runs (with
 *             its KKT reduction, and for atomic adds the zeroing and the
 *             separate KKT pass they need).  Timing replaces the model; set
 *             one after cpapr_create.
 *  fp64_dot   how the FP64 form's Phi evaluates the divisor's dot product
 *             <B[i_n], pi>.  CPAPR_DOT_FP64: FP64 FMAs.  CPAPR_DOT_FP32_PIPE:
 *             on the FP32 pipe (64 times the FP64 FMA rate on GB300) with
 *             error-free transformations of 48-bit hi/lo cuts of the FP64
 *             operands; its error stays below 6e-13 relative to
 *             max(s, eps), inside the FP64 form's 1e-12 bound (it applies to
 *             lanes of 8 or fewer ranks and eps >= 2^-43; operands >= 2^31 take
 *             the FP64 dot for their batch).  CPAPR_DOT_AUTO (default): the FP32
 *             pipe where a launch has at least 608 tiles (4 per SM), the FP64
 *             dot below that, where one tile's latency bounds the launch.  The
 *             batched solver always takes the FP64 dot.  Ignored in FP32.
 *  tune_cache NULL (default) or the path of a text file of tuned choices,
 *             one line per shape class: precision, number of modes, padded
 *             rank, and power-of-two buckets of the nonzeros, of the mode's
 *             rows and of the nonzeros per non-empty row.  At create each
 *             mode whose class is in the file takes the cached choice (no
 *             timing); with autotune = 1 the other modes are timed and their
 *             choices appended to the file, with autotune = 0 they keep the
 *             heuristic.  Lines that do not parse, or choices that do not
 *             fit this tensor, are ignored.  cpapr_batch_mu_solve keeps each
 *             context's tile size and Pi form (its lanes and reduction are
 *             fixed by the batched kernel).
 *  profile    1 = record CUDA events around every Phi launch so that
 *             cpapr_kernel_stats() can report per-kernel device time.
 *  pi_mode    the Khatri-Rao rows Pi of Algorithm 3.  CPAPR_PI_FUSED: formed
 *             per nonzero inside every Phi evaluation from the factor rows.
 *             CPAPR_PI_MATERIALISED: built once per mode and outer iteration
 *             (the factors of the other modes do not change within a mode's
 *             inner loop) into a buffer of nnz x R values of the working
 *             precision, which every Phi of the inner loop streams; results
 *             are identical to the fused form.  CPAPR_PI_AUTO (default):
 *             materialised in FP64 with three or more modes and in FP32 with
 *             four or more, when the buffer takes at most half of the free
 *             device memory; else fused.
 *             MTTKRP, the log-likelihood and the batched solver always form
 *             the rows in place.
 *  l2_persist 1 = mark the factor matrices (held in one allocation) as
 *             persisting in L2 for the kernels that gather factor rows (Phi,
 *             MTTKRP, log-likelihood, the Khatri-Rao build): an access-policy
 *             window over them on each such launch, with the process's
 *             persisting-L2 set-aside raised to cover it (up to the device
 *             maximum; never lowered; persisting lines are returned to normal
 *             when the context is destroyed).  0 = off (default).  Ignored
 *             on devices without persisting L2 or that refuse the set-aside
 *             (cpapr_get_info then reports l2_window_bytes = 0).
 */
typedef struct {
    int32_t precision;
    int32_t reduction;
    double eps;
    double kappa;
    double kappa_tol;
    uint64_t seed;
    void *stream;
    int32_t tile_nnz;
    int32_t rank_lanes;
    int32_t use_graph;
    int32_t autotune;
    int32_t profile;
    int32_t pi_mode;
    int32_t l2_persist;
    int32_t fp64_dot;
    const char *tune_cache;
} cpapr_options;

void cpapr_default_options(cpapr_options *opt);

/*
 * Builds a context for one sparse tensor (Algorithm 1's input X).
 *  nmodes  N, 2..CPAPR_MAX_MODES.   dims  N sizes, each 1..2^31-1.
 *  nnz     number of stored entries, 0..2^31-1.
 *  idx     N pointers, idx[m][j] = mode-m coordinate of entry j (int64).
 *  vals    nnz counts (>= 0, finite).  Repeated coordinates are allowed;
 *          they act as one entry holding their sum, because Phi, MTTKRP and
 *          the log-likelihood are linear in x.
 *  rank    R >= 1.   opt  NULL for defaults.   out  receives the context.
 * The tensor is copied to the device and sorted once per mode (the per-mode
 * ordering of the paper's Section "CP-APR MU Implementation and
 * Parallelization": sorting each mode once at the start).  idx and vals may
 * be host memory (pageable or pinned: copied by the copy engines, pinned
 * being faster) or device memory (read in place); the call returns after the
 * inputs are no longer used.
 * Errors: E_ARG, E_RANGE (coordinate out of range), E_VALUE, E_NOMEM, E_CUDA.
 * On error *out is NULL and the message is available from
 * cpapr_last_error(NULL) on the calling thread.
 */
cpapr_status cpapr_create(int32_t nmodes, const int64_t *dims, int64_t nnz, const int64_t *const *idx,
                          const double *vals, int32_t rank, const cpapr_options *opt, cpapr_ctx **out);

/* Frees the context and all its device memory.  NULL is a no-op. */
void cpapr_destroy(cpapr_ctx *ctx);

/*
 * Sets the model [lambda; A^(1) .. A^(N)] (Algorithm 1's initial guess):
 * lambda is R doubles, factors[m] is I_m x R row-major doubles.  Resets the
 * outer-iteration counter and the stored Phi used by S.  The values are used
 * as given (no normalisation).  Errors: E_ARG, E_VALUE (negative or
 * non-finite entry), E_CUDA.
 */
cpapr_status cpapr_set_model(cpapr_ctx *ctx, const double *lambda, const double *const *factors);

/*
 * Random initial model: factor entries U(0,1) from a SplitMix64 stream
 * (Steele, Lea, Flood 2014; entry e of factor m is draw e of the sub-stream
 * whose base is draw 200+m of a generator seeded with `seed`), each column
 * scaled to sum to 1, lambda_r = product over modes of the column sums.
 * Resets the outer-iteration counter like cpapr_set_model.
 */
cpapr_status cpapr_init_random(cpapr_ctx *ctx, uint64_t seed);

/* Copies the current model out (lambda: R doubles; factors[m]: I_m x R). */
cpapr_status cpapr_get_model(cpapr_ctx *ctx, double *lambda, double *const *factors);

/*
 * Checkpoint / resume.  The state the MU loop of Algorithm 1 carries from one
 * outer iteration to the next: the model (lambda, factors), the Phi^(m) of
 * each mode's last inner iteration (I_m x R doubles each; the shift S of the
 * next iteration reads it) and the number of outer iterations run since the
 * model was set.  Restoring a state into a context built from the same
 * tensor with the same options continues the solve exactly as if it had not
 * stopped (bit for bit).  phi_prev may be NULL in cpapr_get_state to skip it;
 * in cpapr_set_state NULL means zeros (no shift).
 */
cpapr_status cpapr_get_state(cpapr_ctx *ctx, double *lambda, double *const *factors, double *const *phi_prev,
                             int64_t *outer_done);
cpapr_status cpapr_set_state(cpapr_ctx *ctx, const double *lambda, const double *const *factors,
                             const double *const *phi_prev, int64_t outer_done);

/*
 * Phi^(mode) of Algorithm 2 for the current factors.  B is I_mode x R; pass
 * NULL to use B = A^(mode) diag(lambda) (Algorithm 1 without S).  out
 * receives I_mode x R doubles.  Errors: E_ARG, E_STATE (no model), E_CUDA.
 */
cpapr_status cpapr_phi(cpapr_ctx *ctx, int32_t mode, const double *B, double *out);

/* Size of the fixed device scratch used by cpapr_phi_noalloc (8 MiB). */
#define CPAPR_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * Phi^(mode) like cpapr_phi, for callers that cannot have the library
 * allocate device memory during the call: for example code whose device
 * memory is held by another allocator (a framework's caching allocator that
 * has reserved the GPU, a fixed memory budget) or a loop that must not block
 * on cudaMalloc/cudaFree.  The paper has no counterpart.
 *  B    NULL (B = A^(mode) diag(lambda)) or a DEVICE pointer, I_mode x R doubles.
 *  out  DEVICE pointer receiving I_mode x R doubles.
 * The kernel's scratch (per-tile partial rows, 2 x tiles x padded rank
 * elements) comes from a fixed array of CPAPR_NOALLOC_SCRATCH_BYTES in device
 * memory that every GPU loading the library holds until the process exits;
 * the call performs no cudaMalloc, cudaFree or other allocating call.  It
 * runs on the context's device (made current for the call; the caller's
 * current device is restored before it returns) and synchronises the
 * context's stream before returning.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress).
 * All calls share the one array and it keeps the last call's contents
 * (nothing in it needs to start at zero): calls that overlap on the GPU --
 * on other streams, contexts or host threads -- race and must be serialised
 * by the caller.
 * Errors: E_RANGE when the mode needs more scratch than the array holds
 * (raise tile_nnz or use cpapr_phi), E_ARG for host pointers or a bad mode,
 * E_STATE without a model, E_TIMEOUT when a bounded device-side wait gave up
 * (out is then incomplete; the context stays usable), E_CUDA.
 */
cpapr_status cpapr_phi_noalloc(cpapr_ctx *ctx, int32_t mode, const double *B, double *out);

/*
 * MTTKRP of the paper's Experiment 8: M[i_n,:] = sum over entries in slice
 * i_n of x * (elementwise product of A^(m)[i_m,:], m != n), i.e.
 * X_(n) (A^(N) (.) ... (.) A^(n+1) (.) A^(n-1) (.) ... (.) A^(1)).
 * out receives I_mode x R doubles.
 */
cpapr_status cpapr_mttkrp(cpapr_ctx *ctx, int32_t mode, double *out);

/*
 * Poisson log-likelihood of the current model without the constant
 * sum log(x!):  sum_nz x log(m) - sum over all entries of the model, with
 * m = sum_r lambda_r prod_m A^(m)[i_m, r].  -inf when some m is 0 at a
 * nonzero.  (Not in the paper; it is the quantity CP-APR maximises.)
 */
cpapr_status cpapr_loglik(cpapr_ctx *ctx, double *out);

typedef struct {
    int32_t outer_iters;  /* outer iterations run by this call */
    int32_t total_inner;  /* inner iterations summed over modes and outer iterations */
    int32_t converged;    /* 1 if in the last outer iteration every mode passed its KKT check at once */
    int32_t reserved;
    double loglik;        /* log-likelihood of the final model */
    double kkt_viol;      /* largest last-checked violation over modes, last outer iteration */
} cpapr_result;

/*
 * Algorithm 1: for each outer iteration and each mode n,
 *   B <- (A^(n) + S) Lambda;  repeat up to max_inner times:
 *   Phi <- Algorithm 2; stop when max|min(B, 1 - Phi)| < tol; B <- B * Phi;
 *   then lambda <- column sums of B, A^(n) <- B Lambda^-1.
 * Stops after max_outer outer iterations or when every mode passed its KKT
 * check at the first inner iteration.  The outer-iteration counter carries
 * over between calls, so two calls with max_outer = 1 equal one call with
 * max_outer = 2 (S is applied from the second outer iteration on).
 * inner_trace (NULL or max_outer * N int32) receives the inner iterations
 * of each (outer, mode); ll_trace (NULL or max_outer doubles) receives the
 * log-likelihood after each outer iteration (costs one pass per iteration);
 * kkt_trace (NULL or max_outer doubles) receives, per outer iteration, the
 * largest last-checked violation max|min(B, 1 - Phi)| over the modes (free:
 * the host reads the inner-loop states once per outer iteration anyway).
 * Errors: E_ARG, E_STATE (no model), E_CUDA.
 */
cpapr_status cpapr_mu_solve(cpapr_ctx *ctx, double tol, int32_t max_outer, int32_t max_inner, cpapr_result *res,
                            int32_t *inner_trace, double *ll_trace, double *kkt_trace);

/*
 * Solves `count` independent contexts (each with its own tensor, rank and
 * model) together: for every outer iteration, the Phi work of all tensors
 * for mode n runs in one persistent launch that pulls tiles from a shared
 * work list.  Each context ends exactly as cpapr_mu_solve would leave it.
 * The contexts must live on the same device and use the same precision.
 * results receives `count` entries.
 */
cpapr_status cpapr_batch_mu_solve(cpapr_ctx *const *ctxs, int32_t count, double tol, int32_t max_outer,
                                  int32_t max_inner, cpapr_result *results);

typedef struct {
    int32_t nmodes;
    int32_t rank;
    int32_t rank_padded;   /* R rounded up for 16-byte vector rows */
    int32_t precision;
    int64_t nnz;
    int64_t dims[CPAPR_MAX_MODES];
    int32_t tile_nnz[CPAPR_MAX_MODES];    /* chosen per mode */
    int32_t rank_lanes[CPAPR_MAX_MODES];  /* chosen per mode */
    int32_t reduction[CPAPR_MAX_MODES];   /* chosen per mode */
    int32_t ntiles[CPAPR_MAX_MODES];
    int32_t nsplit[CPAPR_MAX_MODES];      /* rows that span more than one tile */
    int32_t pi_mode[CPAPR_MAX_MODES];     /* CPAPR_PI_FUSED or CPAPR_PI_MATERIALISED, per mode */
    int64_t device_bytes;  /* device memory held by the context */
    int64_t kernel_launches; /* kernels this context has launched (graph replays counted per kernel) */
    int64_t l2_window_bytes; /* bytes of the persisting-L2 window over the factors (0: none) */
} cpapr_info;

cpapr_status cpapr_get_info(const cpapr_ctx *ctx, cpapr_info *info);

/*
 * Per-kernel device time recorded while opt.profile = 1 (CUDA events on the
 * context's stream).  kind 0 = Phi tile kernel (rows that span tiles are
 * finished inside it), 1 = materialised Khatri-Rao rows, 2 = MU update, 3 = normalisation, 4 = S and B, 5 = log-likelihood,
 * 6 = MTTKRP.  Returns the launch count and the summed milliseconds since
 * the last reset; reset = 1 clears the counters after reading.
 */
cpapr_status cpapr_kernel_stats(cpapr_ctx *ctx, int32_t kind, int64_t *launches, double *total_ms, int32_t reset);

/* One-line description of the last error on ctx, or of the last failed
 * cpapr_create on this thread when ctx is NULL.  Never NULL. */
const char *cpapr_last_error(const cpapr_ctx *ctx);

/* Library version string. */
const char *cpapr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CPAPR_H */
