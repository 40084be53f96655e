// Internal declarations of the CP-APR MU CUDA library (sm_103a).
//
// Device layout of one context (all allocations owned by the context):
//   per mode n (sorted by i_n once, at create):
//     seg[n]      int32 [I_n + 1]    first sorted position of each row
//     rstart[n]   uint32 bits        bit p set where a row starts at sorted position p
//     nzrow[n]    int32 [K_n]        the rows holding nonzeros, increasing (K_n of them)
//     idx[n][k]   int32 [nnz_pad]    coordinate of the k-th other mode (k = 0..N-2,
//                                    increasing mode number), in mode-n order
//     val[n]      T     [nnz_pad]    counts in mode-n order (T = double or float)
//     tile table  row_first[t], krow[t] (index in nzrow of the row holding
//                 the tile's first nonzero), the rows that span tiles, each
//                 tile's split of its head and tail partial, per-split counters
//   model:  A[m] T [I_m x Rp], lambda double [Rp], B T [Imax x Rp],
//           Phi[m] T [I_m x Rp] (kept for the shift S of the next iteration);
//           FP32 form: also FP64 masters A64[m] [I_m x Rp] and B64 [Imax x Rp]
//           that the MU update and the normalisation keep (A and B are then
//           their FP32 copies, which the Phi family reads)
//   scratch: carry T [2 x ntiles x Rp] (per-tile partial rows), reductions.
// Rp is R rounded up so that one factor row is a whole number of 16-byte
// vectors; the padding columns are zero everywhere and never leave the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cpapr.h"

namespace cpapr {

constexpr int kMaxModes = CPAPR_MAX_MODES;

enum KernelKind { K_PHI = 0, K_PI = 1, K_UPDATE = 2, K_NORM = 3, K_SB = 4, K_LL = 5, K_MTTKRP = 6, K_NKINDS = 7 };

// Device-side state of one mode's inner loop (written by the kernels only).
struct InnerState {
    int32_t l;          // inner iteration about to run (0-based)
    int32_t done;       // KKT check passed: skip the rest of the inner loop
    int32_t used;       // inner iterations run
    int32_t passed;     // 1 if the check passed (at iteration used)
    uint32_t counter;   // last-block election counter
    int32_t pad[3];
    unsigned long long kkt[2];  // max violation of iteration l, as ordered bits of a double >= 0
    double viol;        // last checked violation
};

struct ModeLayout {
    int32_t In = 0;
    int32_t *seg = nullptr;
    uint32_t *rstart = nullptr;    // row-start bits of the sorted positions (a word per 32 nonzeros)
    int32_t *nzrow = nullptr;      // [K] rows with nonzeros, increasing
    int32_t K = 0;
    int32_t *idx[kMaxModes - 1] = {};
    void *val = nullptr;
    // tiles
    int32_t tile_nnz = 0, ntiles = 0, lanes = 1, reduction = CPAPR_REDUCE_SEGMENTED, threads = 256;
    int32_t *row_first = nullptr;  // [ntiles] row holding the tile's first nonzero
    int32_t *krow = nullptr;       // [ntiles + 1] index in nzrow of that row; krow[ntiles] = K - 1
    int32_t nsplit = 0;
    int32_t *split = nullptr;      // [3 * nsplit] (row, first tile, last tile)
    int32_t *tsplit = nullptr;     // [2 * ntiles] split of each tile's head / tail partial, or -1
    int32_t *splitcnt = nullptr;   // [nsplit] partial counters of the tile kernel (zero between launches)
    int32_t pi = 0;                // 1: Phi streams the materialised Khatri-Rao rows (built per outer iteration)
    int32_t nempty = 0;
    int32_t *erows = nullptr;      // [nempty] rows without nonzeros, increasing
};

struct cpapr_ctx_impl;

}  // namespace cpapr

struct cpapr_ctx {
    int N = 0;
    int64_t dims[CPAPR_MAX_MODES] = {};
    int64_t nnz = 0;
    int64_t nnz_pad = 0;
    int R = 0, Rp = 0;
    int Imax = 0;
    cpapr_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    size_t esize = 8;  // bytes per element of the working precision
    cpapr::ModeLayout mode[CPAPR_MAX_MODES];
    // model
    double *lambda = nullptr;
    void *A[CPAPR_MAX_MODES] = {};   // views into factor_block
    void *factor_block = nullptr;    // all factor matrices, one allocation
    size_t factor_bytes = 0;
    cudaAccessPolicyWindow l2win{};  // persisting-L2 window over factor_block (num_bytes 0: none)
    void *B = nullptr;
    // FP32 form: FP64 masters of the factors and of B.  The multiplicative
    // update, the shift S and the normalisation run on them in FP64 and
    // refresh the FP32 copies A[m] and B that Phi gathers, so an entry that
    // decays below the FP32 range keeps its FP64 value instead of becoming a
    // zero that MU could never move again.  Null in the FP64 form.
    double *A64[CPAPR_MAX_MODES] = {};
    double *B64 = nullptr;
    void *outbuf = nullptr;  // Phi / MTTKRP output of the one-off calls (Imax x Rp)
    void *Phi[CPAPR_MAX_MODES] = {};
    double *stage = nullptr;  // FP64 staging for I/O (Imax x Rp)
    void *carry = nullptr;
    int64_t carry_elems = 0;
    void *pibuf = nullptr;  // materialised Khatri-Rao rows of the current mode [nnz_pad x Rp]
    int pi_mode_built = -1;  // mode whose rows pibuf holds, built from the current other factors (-1: none)
    int64_t llpart_n = 0;    // capacity of llpart (tiles)
    double *colpart = nullptr;   // column-sum partials [N x kColParts x Rp]
    unsigned int *llcount = nullptr;  // last-block counters (zero between launches): [0] log-likelihood total, [1] normalisation column sums
    double *colsum = nullptr;    // per-mode column sums [N x Rp]
    double *llpart = nullptr;    // per-tile log-likelihood partials
    cpapr::InnerState *inner = nullptr;  // [N]
    double *scalars = nullptr;   // misc device scalars
    int32_t *errflag = nullptr;  // device error flags
    bool model_set = false;
    int64_t k_total = 0;
    bool sticky = false;
    std::string err;
    int64_t device_bytes = 0;
    int64_t launches = 0;         // kernels launched (see count_launch)
    int graph_body_kernels[CPAPR_MAX_MODES] = {};
    int graph_capture_kernels = 0;  // kernels recorded by the capture in progress
    std::vector<void *> allocs;
    // profiling
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    int64_t prof_launches[cpapr::K_NKINDS] = {};
    double prof_ms[cpapr::K_NKINDS] = {};
    // graphs (one per mode and inner-loop bound)
    cudaGraphExec_t graph_exec[CPAPR_MAX_MODES] = {};
    int graph_max_inner[CPAPR_MAX_MODES] = {};
    double graph_tol[CPAPR_MAX_MODES] = {};
};

namespace cpapr {

constexpr int kColParts = 256;
// tiles from which an FP64 Phi launch takes the kernel with its dot on the FP32 pipe
constexpr int kDfMinTiles = 152 * 4;

// ---- error plumbing ------------------------------------------------------
cpapr_status fail(cpapr_ctx *ctx, cpapr_status st, const std::string &msg);
cpapr_status cuda_fail(cpapr_ctx *ctx, cudaError_t e, const char *what);

#define CPAPR_CUDA(ctx, call)                                  \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return cpapr::cuda_fail((ctx), _e, #call); \
    } while (0)

#define CPAPR_TRY(expr)                       \
    do {                                      \
        cpapr_status _s = (expr);             \
        if (_s != CPAPR_OK) return _s;        \
    } while (0)

cpapr_status dev_alloc(cpapr_ctx *ctx, void **p, size_t bytes);
// persisting-L2 access-policy window over the factor matrices (l2_persist)
cpapr_status configure_l2_window(cpapr_ctx *ctx);
// the window for launches that gather factor rows, or null
inline const cudaAccessPolicyWindow *l2_window(const cpapr_ctx *ctx) {
    return ctx->l2win.num_bytes ? &ctx->l2win : nullptr;
}
// stream-ordered allocation from the library's memory pool of the current device
cudaError_t lib_malloc_raw(void **p, size_t bytes, cudaStream_t s);
template <typename T> inline cudaError_t lib_malloc(T **p, size_t bytes, cudaStream_t s) {
    return lib_malloc_raw(reinterpret_cast<void **>(p), bytes, s);
}

// Counts kernel launches; launches recorded while a stream capture is active
// are not counted here (graph replays are counted from the iterations run).
void count_launch(cpapr_ctx *ctx, int k = 1);

// ---- profiling ------------------------------------------------------------
struct ProfScope {
    cpapr_ctx *ctx;
    int kind;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(cpapr_ctx *c, int k);
    ~ProfScope();
};
void prof_collect(cpapr_ctx *ctx);

// ---- index build (index.cu) ------------------------------------------------
cpapr_status build_layouts(cpapr_ctx *ctx, const int64_t *const *idx_in, const double *vals_in);
cpapr_status build_tiles(cpapr_ctx *ctx, int n, int tile_nnz);

// ---- Phi family (phi.cu) -----------------------------------------------------
enum PhiOp { OP_PHI = 0, OP_MTTKRP = 1, OP_LL = 2 };
// Launches the tile kernel for mode n writing `out` (I_n x Rp).
// B: I_n x Rp of the working type (ignored for MTTKRP).  inner: state whose
// done flag / kkt slot the kernels use (may be null for a one-off Phi).
cpapr_status launch_phi(cpapr_ctx *ctx, int n, PhiOp op, const void *B, void *out, InnerState *inner);
// builds the materialised Khatri-Rao rows of mode n (a no-op unless the mode uses them)
cpapr_status launch_pi_build(cpapr_ctx *ctx, int n);
// selects the materialised (on = 1) or fused (0) Khatri-Rao rows for mode n
cpapr_status configure_pi(cpapr_ctx *ctx, int n, int on);
int pi_auto(const cpapr_ctx *ctx);
int pi_fits(const cpapr_ctx *ctx);
// bytes the staging barrier of the tile kernels expects beyond its copies (failure injection; 0 normally)
uint32_t injected_stage_shortfall();
// Sum of x log(m) over nonzeros, into llpart then *dst (device double).
// log-likelihood sum of the current model (without the model total) into *dst (device)
cpapr_status launch_loglik(cpapr_ctx *ctx, double *dst);
// Rows of mode n without nonzeros: zero them in `out`; add their KKT term
// (first inner iteration) after the S/B kernel.
cpapr_status launch_zero_empty(cpapr_ctx *ctx, int n, void *out);
cpapr_status launch_empty_kkt(cpapr_ctx *ctx, int n, const void *B, InnerState *inner);
bool phi_config_supported(int esize, int nm1, int rp, int lanes);
// shared memory of a tile kernel launch, and the most a launch may use
size_t phi_smem_for(int esize, int nm1, int tile, int rp, int lanes);
constexpr size_t kMaxPhiSmem = 220 * 1024;

// ---- MU kernels (mu.cu) -------------------------------------------------------
cpapr_status launch_sb(cpapr_ctx *ctx, int n, bool shift, InnerState *inner);
cpapr_status launch_update(cpapr_ctx *ctx, int n, double tol, int max_inner, InnerState *inner,
                           unsigned long long cond_handle, int use_cond);
cpapr_status launch_normalise(cpapr_ctx *ctx, int n);
cpapr_status launch_scale_b(cpapr_ctx *ctx, int n, void *dstB);     // B = A^(n) diag(lambda)
// dst = sum of llpart[0..nll) - sum_r lambda_r prod_m colsum_m(r), one launch
cpapr_status launch_ll_total(cpapr_ctx *ctx, const double *llpart, int nll, double *dst);
cpapr_status launch_init_random(cpapr_ctx *ctx, uint64_t seed);
cpapr_status upload_matrix(cpapr_ctx *ctx, const double *src, int64_t rows, void *dst);   // R cols -> Rp cols, to T
// factor m from the caller's rows x R doubles (and its FP64 master in the FP32 form)
cpapr_status upload_factor(cpapr_ctx *ctx, int m, const double *src);
cpapr_status download_matrix(cpapr_ctx *ctx, const void *src, int64_t rows, double *dst); // Rp cols T -> R cols
cpapr_status launch_kkt_rows(cpapr_ctx *ctx, int n, const void *B, const void *Phi, InnerState *inner);

// ---- small utilities (index.cu) ---------------------------------------------
cpapr_status exclusive_scan_u32(cpapr_ctx *ctx, uint32_t *data, int64_t n, uint32_t *total_out_dev);

// ---- solver (solver.cu) -------------------------------------------------------
cpapr_status mu_solve(cpapr_ctx *ctx, double tol, int max_outer, int max_inner, cpapr_result *res,
                      int32_t *inner_trace, double *ll_trace, double *kkt_trace);
cpapr_status batch_mu_solve(cpapr_ctx *const *ctxs, int count, double tol, int max_outer, int max_inner,
                            cpapr_result *results);

// ---- device helpers -------------------------------------------------------------
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

// elementwise product of two 16-byte vectors
__device__ __forceinline__ float4 vmul(float4 a, float4 b) {
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }

// FP32 form of B <- B * Phi on the FP64 master, for the pair of entries
// (2e, 2e + 1): the master pair times the FP32 Phi pair, and its FP32 copy
// (a warp reads and writes 512 contiguous bytes of the master, 256 of Phi and B)
__device__ __forceinline__ void master_mul(double2 *__restrict__ Bm, float2 *__restrict__ B,
                                           const float2 *__restrict__ P, int64_t e) {
    const float2 p = P[e];
    double2 b = Bm[e];
    b.x *= (double)p.x;
    b.y *= (double)p.y;
    Bm[e] = b;
    B[e] = make_float2((float)b.x, (float)b.y);
}

__device__ __forceinline__ unsigned long long ordered_bits(double v) {
    // v >= 0: IEEE bit patterns of non-negative doubles order like the values
    return (unsigned long long)__double_as_longlong(v);
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// FP64 factor m: the master in the FP32 form, the factor itself in FP64
inline const double *factor64(const cpapr_ctx *ctx, int m) {
    return ctx->A64[m] ? ctx->A64[m] : reinterpret_cast<const double *>(ctx->esize == 8 ? ctx->A[m] : nullptr);
}

}  // namespace cpapr
