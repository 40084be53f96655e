// C ABI of the CP-APR MU library: argument checks, context lifecycle, model
// I/O and the one-off Phi / MTTKRP / log-likelihood calls.  The MU loop
// itself lives in solver.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace {
thread_local std::string g_create_error = "no error";
}

namespace cpapr {

cpapr_status fail(cpapr_ctx *ctx, cpapr_status st, const std::string &msg) {
    if (ctx)
        ctx->err = msg;
    else
        g_create_error = msg;
    return st;
}

cpapr_status cuda_fail(cpapr_ctx *ctx, cudaError_t e, const char *what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, CPAPR_E_NOMEM, msg);
    }
    if (ctx) ctx->sticky = true;
    return fail(ctx, CPAPR_E_CUDA, msg);
}

// Host-side fault injection for testing error paths: when the environment
// variable CPAPR_FAULT_ALLOC_AT holds k > 0, the k-th context allocation
// counted from the moment that value was first seen reports CPAPR_E_NOMEM
// (no device call fails; nothing is done to the GPU).
static bool injected_alloc_failure() {
    static std::mutex mu;
    static std::string seen;
    static long long calls = 0;
    const char *s = std::getenv("CPAPR_FAULT_ALLOC_AT");
    std::lock_guard<std::mutex> lock(mu);
    const std::string v = s ? s : "";
    if (v != seen) {
        seen = v;
        calls = 0;
    }
    if (v.empty()) return false;
    const long long k = std::atoll(v.c_str());
    return k > 0 && ++calls == k;
}

// Device memory of every context comes from one stream-ordered pool per
// device owned by the library.  The pool keeps up to a quarter of the
// device's memory cached after frees, so contexts created and destroyed in a
// loop (a new tensor per request) do not pay for cudaMalloc / cudaFree each
// time; memory above that is returned to the driver at synchronisation.
static cudaMemPool_t device_pool(int dev) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        size_t freeb = 0, totalb = 0;
        cudaMemGetInfo(&freeb, &totalb);
        uint64_t keep = (uint64_t)totalb / 4;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaGetLastError();
        pools[dev] = pool;
    }
    return pools[dev];
}

cudaError_t lib_malloc_raw(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return cudaMallocAsync(p, std::max<size_t>(bytes, 16), s);
    return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, s);
}

cpapr_status dev_alloc(cpapr_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (injected_alloc_failure()) return fail(ctx, CPAPR_E_NOMEM, "injected allocation failure (CPAPR_FAULT_ALLOC_AT)");
    cudaError_t e = lib_malloc(p, bytes, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device allocation");
    ctx->allocs.push_back(*p);
    ctx->device_bytes += (int64_t)bytes;
    return CPAPR_OK;
}

void count_launch(cpapr_ctx *ctx, int k) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        ctx->graph_capture_kernels += k;
        return;
    }
    ctx->launches += k;
}

ProfScope::ProfScope(cpapr_ctx *c, int k) : ctx(c), kind(k) {
    if (!ctx->opt.profile) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (ctx->ev_pool.size() < 2 && !ctx->ev_pending.empty()) {
        // recycle the pairs that have completed, oldest first, without waiting
        size_t k = 0;
        for (; k < ctx->ev_pending.size(); ++k) {
            auto &p = ctx->ev_pending[k];
            if (cudaEventQuery(p.second.second) != cudaSuccess) break;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
                ctx->prof_launches[p.first] += 1;
                ctx->prof_ms[p.first] += ms;
            }
            ctx->ev_pool.push_back(p.second.first);
            ctx->ev_pool.push_back(p.second.second);
        }
        cudaGetLastError();
        ctx->ev_pending.erase(ctx->ev_pending.begin(), ctx->ev_pending.begin() + k);
    }
    auto take = [&]() {
        cudaEvent_t e = nullptr;
        if (!ctx->ev_pool.empty()) {
            e = ctx->ev_pool.back();
            ctx->ev_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
        }
        return e;
    };
    a = take();
    b = take();
    if (a && b) cudaEventRecord(a, ctx->stream);
}

ProfScope::~ProfScope() {
    if (!a || !b) {
        if (a) ctx->ev_pool.push_back(a);
        if (b) ctx->ev_pool.push_back(b);
        return;
    }
    cudaEventRecord(b, ctx->stream);
    ctx->ev_pending.push_back({kind, {a, b}});
}

void prof_collect(cpapr_ctx *ctx) {
    for (auto &p : ctx->ev_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.second.second) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
            ctx->prof_launches[p.first] += 1;
            ctx->prof_ms[p.first] += ms;
        }
        ctx->ev_pool.push_back(p.second.first);
        ctx->ev_pool.push_back(p.second.second);
    }
    ctx->ev_pending.clear();
}

static int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Built-in choice of lanes per nonzero and nonzeros per tile (from sweeps on
// GB300 over the 1e7-nonzero 3-way and 5e7-nonzero 4-way workloads).  FP64:
// 8 ranks per lane (one lane up to 8 ranks) with batches of up to four
// nonzeros; FP32: 16-byte vectors of 4 ranks per lane up to 32 ranks, 8 ranks
// per lane above, and the largest tile whose shared-memory stage leaves room
// for the blocks per SM the tile kernel is built for (four with one float4 per
// lane, else three).  With materialised Khatri-Rao rows the stage holds only
// row ids and values, so the same room takes larger tiles.
static void heuristic_config(const cpapr_ctx *ctx, int n, int pi, int *lanes, int *tile, int *reduction) {
    const int Rp = ctx->Rp;
    int g;
    if (ctx->esize == 8)
        g = std::max(1, Rp / 8);
    else
        g = Rp <= 32 ? std::max(1, Rp / 4) : Rp / 8;
    *lanes = g;
    if (ctx->esize == 8) {
        *tile = Rp <= 16 ? 2048 : 1024;
    } else {
        const int nm1 = pi ? 0 : ctx->N - 1;
        const size_t per_block = (Rp / g <= 4 ? 227 / 4 : 227 / 3) * 1024 - 1024;
        *tile = 1024;
        for (int t : {4096, 2048})
            if (phi_smem_for(4, nm1, t, Rp, g) <= per_block) {
                *tile = t;
                break;
            }
    }
    *reduction = CPAPR_REDUCE_SEGMENTED;
    (void)n;
}

void batch_forget(cpapr_ctx *ctx);

cpapr_status configure_mode(cpapr_ctx *ctx, int n, int lanes, int tile, int reduction) {
    batch_forget(ctx);
    if (!phi_config_supported((int)ctx->esize, ctx->N - 1, ctx->Rp, lanes))
        return fail(ctx, CPAPR_E_ARG, "rank_lanes not supported for this rank and precision");
    if (tile < 64 || tile > (1 << 20) || tile % 4)
        return fail(ctx, CPAPR_E_ARG, "tile_nnz must be a multiple of 4 in [64, 2^20]");
    if (phi_smem_for((int)ctx->esize, ctx->N - 1, tile, ctx->Rp, lanes) > kMaxPhiSmem)
        return fail(ctx, CPAPR_E_ARG, "tile_nnz too large: its staged streams and partial rows exceed shared memory");
    ModeLayout &L = ctx->mode[n];
    L.lanes = lanes;
    L.reduction = reduction == CPAPR_REDUCE_ATOMIC ? CPAPR_REDUCE_ATOMIC : CPAPR_REDUCE_SEGMENTED;
    if (L.tile_nnz != tile || !L.row_first) CPAPR_TRY(build_tiles(ctx, n, tile));
    // per-tile log-likelihood partials (the sum runs along mode 0 or N-1)
    if (L.ntiles > ctx->llpart_n || !ctx->llpart) {
        if (ctx->llpart) cudaFreeAsync(ctx->llpart, ctx->stream);
        ctx->llpart = nullptr;
        ctx->llpart_n = 0;
        CPAPR_CUDA(ctx, lib_malloc((void **)&ctx->llpart, (size_t)std::max(L.ntiles, 1) * 8, ctx->stream));
        ctx->llpart_n = std::max(L.ntiles, 1);
    }
    if (ctx->graph_exec[n]) {
        cudaGraphExecDestroy(ctx->graph_exec[n]);
        ctx->graph_exec[n] = nullptr;
    }
    return CPAPR_OK;
}

// Materialised Khatri-Rao rows: one buffer of nnz_pad x Rp elements shared by
// the modes (a mode's rows are rebuilt at the start of its inner loop).
cpapr_status configure_pi(cpapr_ctx *ctx, int n, int on) {
    ModeLayout &L = ctx->mode[n];
    if (on && ctx->N >= 2 && ctx->nnz > 0 && !ctx->pibuf) {
        void *p = nullptr;
        CPAPR_TRY(dev_alloc(ctx, &p, (size_t)ctx->nnz_pad * ctx->Rp * ctx->esize));
        ctx->pibuf = p;
    }
    L.pi = on && ctx->pibuf ? 1 : 0;
    if (ctx->graph_exec[n]) {
        cudaGraphExecDestroy(ctx->graph_exec[n]);
        ctx->graph_exec[n] = nullptr;
    }
    return CPAPR_OK;
}

// The materialised rows are worth a buffer when there are Khatri-Rao
// products to save (three or more modes) and it takes at most half of the
// free device memory (or is already there).
int pi_fits(const cpapr_ctx *ctx) {
    if (ctx->N < 3 || ctx->nnz == 0) return 0;
    if (ctx->pibuf) return 1;
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (double)ctx->nnz_pad * ctx->Rp * ctx->esize <= 0.5 * (double)freeb ? 1 : 0;
}

// Automatic choice (from GB300 sweeps): materialise in FP64, where the
// products cost time on the narrow FP64 pipe, and in FP32 from four modes on,
// where streaming one row beats gathering three or more; a 3-way FP32 Phi
// gathers and multiplies in place.
int pi_auto(const cpapr_ctx *ctx) { return (ctx->esize == 8 || ctx->N >= 4) ? pi_fits(ctx) : 0; }

cpapr_status autotune(cpapr_ctx *ctx);

// Access-policy window over the factor block: hits persist in the set-aside
// part of L2, raised (never lowered) to cover the window where the device
// allows; the hit ratio scales the window down to the set-aside.
cpapr_status configure_l2_window(cpapr_ctx *ctx) {
    int max_persist = 0, max_window = 0;
    CPAPR_CUDA(ctx, cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, ctx->device));
    CPAPR_CUDA(ctx, cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device));
    if (max_persist <= 0 || max_window <= 0 || ctx->factor_bytes == 0) return CPAPR_OK;
    const size_t window = std::min(ctx->factor_bytes, (size_t)max_window);
    // a device or mode that refuses the set-aside leaves the option without effect
    size_t setaside = 0;
    if (cudaDeviceGetLimit(&setaside, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
        cudaGetLastError();
        return CPAPR_OK;
    }
    const size_t want = std::min(window, (size_t)max_persist);
    if (setaside < want) {
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess ||
            cudaDeviceGetLimit(&setaside, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
            cudaGetLastError();
            return CPAPR_OK;
        }
    }
    if (setaside == 0) return CPAPR_OK;
    ctx->l2win.base_ptr = ctx->factor_block;
    ctx->l2win.num_bytes = window;
    ctx->l2win.hitRatio = (float)std::min(1.0, (double)setaside / (double)window);
    ctx->l2win.hitProp = cudaAccessPropertyPersisting;
    ctx->l2win.missProp = cudaAccessPropertyStreaming;
    return CPAPR_OK;
}

}  // namespace cpapr

using namespace cpapr;

extern "C" {

void cpapr_default_options(cpapr_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = CPAPR_FP64;
    opt->reduction = CPAPR_REDUCE_AUTO;
    opt->eps = 1e-10;
    opt->kappa = 0.01;
    opt->kappa_tol = 1e-10;
    opt->seed = 0;
    opt->stream = nullptr;
    opt->tile_nnz = 0;
    opt->rank_lanes = 0;
    opt->use_graph = 1;
    opt->autotune = 0;
    opt->profile = 0;
}

const char *cpapr_version(void) { return "cpapr-gb300 0.1 (sm_103a)"; }

const char *cpapr_last_error(const cpapr_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.empty() ? "no error" : ctx->err.c_str();
}


void cpapr_destroy(cpapr_ctx *ctx) {
    if (!ctx) return;
    batch_forget(ctx);
    cudaStreamSynchronize(ctx->stream);
    for (int n = 0; n < ctx->N; ++n) {
        ModeLayout &L = ctx->mode[n];
        if (L.row_first) cudaFreeAsync(L.row_first, ctx->stream);
        if (L.krow) cudaFreeAsync(L.krow, ctx->stream);
        if (L.split) cudaFreeAsync(L.split, ctx->stream);
        if (L.tsplit) cudaFreeAsync(L.tsplit, ctx->stream);
        if (L.splitcnt) cudaFreeAsync(L.splitcnt, ctx->stream);
        if (ctx->graph_exec[n]) cudaGraphExecDestroy(ctx->graph_exec[n]);
    }
    if (ctx->carry) cudaFreeAsync(ctx->carry, ctx->stream);
    if (ctx->llpart) cudaFreeAsync(ctx->llpart, ctx->stream);
    for (void *p : ctx->allocs) cudaFreeAsync(p, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    // lines this context marked persisting go back to normal priority
    if (ctx->l2win.num_bytes) cudaCtxResetPersistingL2Cache();
    for (auto &p : ctx->ev_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

cpapr_status cpapr_create(int32_t nmodes, const int64_t *dims, int64_t nnz, const int64_t *const *idx,
                          const double *vals, int32_t rank, const cpapr_options *opt, cpapr_ctx **out) {
    if (!out) return fail(nullptr, CPAPR_E_ARG, "out is NULL");
    *out = nullptr;
    if (nmodes < 2 || nmodes > CPAPR_MAX_MODES) return fail(nullptr, CPAPR_E_ARG, "nmodes must lie in [2, 8]");
    if (!dims) return fail(nullptr, CPAPR_E_ARG, "dims is NULL");
    for (int m = 0; m < nmodes; ++m)
        if (dims[m] < 1 || dims[m] > INT32_MAX - 1) return fail(nullptr, CPAPR_E_RANGE, "each dim must lie in [1, 2^31-2]");
    if (nnz < 0 || nnz > INT32_MAX - 4096) return fail(nullptr, CPAPR_E_RANGE, "nnz must lie in [0, 2^31 - 4096]");
    if (nnz > 0 && (!idx || !vals)) return fail(nullptr, CPAPR_E_ARG, "idx or vals is NULL");
    if (nnz > 0)
        for (int m = 0; m < nmodes; ++m)
            if (!idx[m]) return fail(nullptr, CPAPR_E_ARG, "idx[m] is NULL");
    if (rank < 1 || rank > 128) return fail(nullptr, CPAPR_E_ARG, "rank must lie in [1, 128]");
    cpapr_options o;
    cpapr_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != CPAPR_FP64 && o.precision != CPAPR_FP32) return fail(nullptr, CPAPR_E_ARG, "bad precision");
    if (o.reduction < 0 || o.reduction > 2) return fail(nullptr, CPAPR_E_ARG, "bad reduction");
    if (!(o.eps > 0.0) || !(o.kappa >= 0.0) || !(o.kappa_tol >= 0.0)) return fail(nullptr, CPAPR_E_ARG, "bad eps/kappa");
    if (o.rank_lanes < 0 || o.rank_lanes > 32 || (o.rank_lanes & (o.rank_lanes - 1)))
        return fail(nullptr, CPAPR_E_ARG, "rank_lanes must be 0 or a power of two <= 32");
    if (o.tile_nnz != 0 && (o.tile_nnz < 64 || o.tile_nnz > (1 << 20) || o.tile_nnz % 4))
        return fail(nullptr, CPAPR_E_ARG, "tile_nnz must be 0 or a multiple of 4 in [64, 2^20]");
    if (o.l2_persist != 0 && o.l2_persist != 1) return fail(nullptr, CPAPR_E_ARG, "l2_persist must be 0 or 1");
    if (o.fp64_dot < CPAPR_DOT_AUTO || o.fp64_dot > CPAPR_DOT_FP32_PIPE)
        return fail(nullptr, CPAPR_E_ARG, "fp64_dot must be CPAPR_DOT_AUTO, CPAPR_DOT_FP64 or CPAPR_DOT_FP32_PIPE");

    cpapr_ctx *ctx = new (std::nothrow) cpapr_ctx();
    if (!ctx) return fail(nullptr, CPAPR_E_NOMEM, "host allocation failed");
    auto bail = [&](cpapr_status st) {
        g_create_error = ctx->err;
        cpapr_destroy(ctx);
        return st;
    };
    ctx->N = nmodes;
    ctx->nnz = nnz;
    ctx->R = rank;
    ctx->opt = o;
    ctx->esize = o.precision == CPAPR_FP64 ? 8 : 4;
    ctx->Rp = std::max(ctx->esize == 8 ? 2 : 4, next_pow2(rank));
    for (int m = 0; m < nmodes; ++m) {
        ctx->dims[m] = dims[m];
        ctx->Imax = (int)std::max<int64_t>(ctx->Imax, dims[m]);
    }
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaGetDevice"));
    if (o.stream) {
        ctx->stream = (cudaStream_t)o.stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaStreamCreate"));
        ctx->own_stream = true;
    }
    const int Rp = ctx->Rp;
    void *p = nullptr;
    cpapr_status st;
#define CR_TRY(expr)                     \
    do {                                 \
        st = (expr);                     \
        if (st != CPAPR_OK) return bail(st); \
    } while (0)
    CR_TRY(dev_alloc(ctx, &p, 64));
    ctx->errflag = (int32_t *)p;
    CR_TRY(dev_alloc(ctx, &p, sizeof(InnerState) * nmodes));
    ctx->inner = (InnerState *)p;
    CR_TRY(dev_alloc(ctx, &p, (size_t)Rp * 8));
    ctx->lambda = (double *)p;
    CR_TRY(dev_alloc(ctx, &p, (size_t)nmodes * kColParts * Rp * 8));
    ctx->colpart = (double *)p;
    CR_TRY(dev_alloc(ctx, &p, 16));
    ctx->llcount = (unsigned int *)p;
    if (cudaMemsetAsync(ctx->llcount, 0, 16, ctx->stream) != cudaSuccess)
        return bail(fail(ctx, CPAPR_E_CUDA, "memset"));
    CR_TRY(dev_alloc(ctx, &p, (size_t)nmodes * Rp * 8));
    ctx->colsum = (double *)p;
    CR_TRY(dev_alloc(ctx, &p, 64 * 8));
    ctx->scalars = (double *)p;
    if (cudaMemsetAsync(ctx->inner, 0, sizeof(InnerState) * nmodes, ctx->stream) != cudaSuccess)
        return bail(fail(ctx, CPAPR_E_CUDA, "memset"));

    CR_TRY(build_layouts(ctx, idx, vals));

    // the factor matrices share one allocation (each start 256-byte aligned)
    // so that one access-policy window can cover all of them
    size_t fofs[CPAPR_MAX_MODES + 1] = {};
    for (int m = 0; m < nmodes; ++m)
        fofs[m + 1] = fofs[m] + (((size_t)dims[m] * Rp * ctx->esize + 255) & ~(size_t)255);
    CR_TRY(dev_alloc(ctx, &ctx->factor_block, fofs[nmodes]));
    ctx->factor_bytes = fofs[nmodes];
    for (int m = 0; m < nmodes; ++m) {
        ctx->A[m] = (char *)ctx->factor_block + fofs[m];
        CR_TRY(dev_alloc(ctx, &p, (size_t)dims[m] * Rp * ctx->esize));
        ctx->Phi[m] = p;
        if (cudaMemsetAsync(ctx->A[m], 0, (size_t)dims[m] * Rp * ctx->esize, ctx->stream) != cudaSuccess ||
            cudaMemsetAsync(ctx->Phi[m], 0, (size_t)dims[m] * Rp * ctx->esize, ctx->stream) != cudaSuccess)
            return bail(fail(ctx, CPAPR_E_CUDA, "memset"));
    }
    if (ctx->esize == 4) {
        // FP64 masters of the factors and of B (see cpapr_ctx::A64)
        size_t mofs[CPAPR_MAX_MODES + 1] = {};
        for (int m = 0; m < nmodes; ++m) mofs[m + 1] = mofs[m] + (((size_t)dims[m] * Rp * 8 + 255) & ~(size_t)255);
        CR_TRY(dev_alloc(ctx, &p, mofs[nmodes]));
        if (cudaMemsetAsync(p, 0, mofs[nmodes], ctx->stream) != cudaSuccess)
            return bail(fail(ctx, CPAPR_E_CUDA, "memset"));
        for (int m = 0; m < nmodes; ++m) ctx->A64[m] = (double *)((char *)p + mofs[m]);
        CR_TRY(dev_alloc(ctx, &p, (size_t)ctx->Imax * Rp * 8));
        ctx->B64 = (double *)p;
    }
    CR_TRY(dev_alloc(ctx, &p, (size_t)ctx->Imax * Rp * ctx->esize));
    ctx->B = p;
    CR_TRY(dev_alloc(ctx, &p, (size_t)ctx->Imax * Rp * ctx->esize));
    ctx->outbuf = p;
    CR_TRY(dev_alloc(ctx, &p, (size_t)ctx->Imax * Rp * 8));
    ctx->stage = (double *)p;

    if (o.l2_persist) CR_TRY(configure_l2_window(ctx));

    for (int n = 0; n < nmodes; ++n) {
        int lanes, tile, red;
        const int pi = o.pi_mode == CPAPR_PI_MATERIALISED ? 1 : o.pi_mode == CPAPR_PI_FUSED ? 0 : pi_auto(ctx);
        heuristic_config(ctx, n, pi, &lanes, &tile, &red);
        if (o.rank_lanes) lanes = o.rank_lanes;
        if (o.tile_nnz) tile = o.tile_nnz;
        if (o.reduction) red = o.reduction;
        CR_TRY(configure_mode(ctx, n, lanes, tile, red));
        CR_TRY(configure_pi(ctx, n, pi));
    }
    if (o.autotune || o.tune_cache) CR_TRY(autotune(ctx));
    ctx->opt.tune_cache = nullptr;  // the caller's string is not kept
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "build"));
#undef CR_TRY
    *out = ctx;
    return CPAPR_OK;
}

#define API_ENTER(ctx)                                                             \
    do {                                                                           \
        if (!(ctx)) return fail(nullptr, CPAPR_E_ARG, "ctx is NULL");             \
        if ((ctx)->sticky) return CPAPR_E_CUDA;                                    \
    } while (0)

cpapr_status cpapr_set_model(cpapr_ctx *ctx, const double *lambda, const double *const *factors) {
    API_ENTER(ctx);
    if (!lambda || !factors) return fail(ctx, CPAPR_E_ARG, "lambda or factors is NULL");
    for (int m = 0; m < ctx->N; ++m)
        if (!factors[m]) return fail(ctx, CPAPR_E_ARG, "factors[m] is NULL");
    std::vector<double> hl(ctx->Rp, 0.0);
    CPAPR_CUDA(ctx, cudaMemcpy(hl.data(), lambda, (size_t)ctx->R * 8, cudaMemcpyDefault));
    for (int r = 0; r < ctx->R; ++r)
        if (!(hl[r] >= 0.0) || std::isinf(hl[r])) return fail(ctx, CPAPR_E_VALUE, "lambda must be finite and >= 0");
    CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, 16, ctx->stream));
    CPAPR_CUDA(ctx, cudaMemcpyAsync(ctx->lambda, hl.data(), (size_t)ctx->Rp * 8, cudaMemcpyHostToDevice, ctx->stream));
    for (int m = 0; m < ctx->N; ++m) {
        CPAPR_TRY(upload_factor(ctx, m, factors[m]));
        CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->Phi[m], 0, (size_t)ctx->dims[m] * ctx->Rp * ctx->esize, ctx->stream));
    }
    int32_t flags[4] = {0, 0, 0, 0};
    CPAPR_CUDA(ctx, cudaMemcpyAsync(flags, ctx->errflag, 16, cudaMemcpyDeviceToHost, ctx->stream));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->k_total = 0;
    ctx->pi_mode_built = -1;
    if (flags[2]) {
        ctx->model_set = false;
        return fail(ctx, CPAPR_E_VALUE, "factor entries must be finite and >= 0");
    }
    ctx->model_set = true;
    return CPAPR_OK;
}

cpapr_status cpapr_init_random(cpapr_ctx *ctx, uint64_t seed) {
    API_ENTER(ctx);
    CPAPR_TRY(launch_init_random(ctx, seed));
    for (int m = 0; m < ctx->N; ++m)
        CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->Phi[m], 0, (size_t)ctx->dims[m] * ctx->Rp * ctx->esize, ctx->stream));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->k_total = 0;
    ctx->pi_mode_built = -1;
    ctx->model_set = true;
    return CPAPR_OK;
}

cpapr_status cpapr_get_model(cpapr_ctx *ctx, double *lambda, double *const *factors) {
    API_ENTER(ctx);
    if (!ctx->model_set) return fail(ctx, CPAPR_E_STATE, "no model set");
    if (lambda) CPAPR_CUDA(ctx, cudaMemcpyAsync(lambda, ctx->lambda, (size_t)ctx->R * 8, cudaMemcpyDefault, ctx->stream));
    if (factors)
        for (int m = 0; m < ctx->N; ++m) {
            if (!factors[m]) continue;
            // the FP32 form returns the FP64 masters (what the MU loop keeps)
            if (ctx->A64[m])
                CPAPR_CUDA(ctx, cudaMemcpy2DAsync(factors[m], (size_t)ctx->R * 8, ctx->A64[m], (size_t)ctx->Rp * 8,
                                                  (size_t)ctx->R * 8, (size_t)ctx->dims[m], cudaMemcpyDefault,
                                                  ctx->stream));
            else
                CPAPR_TRY(download_matrix(ctx, ctx->A[m], ctx->dims[m], factors[m]));
            // download_matrix stages FP32 through ctx->stage: finish before reuse
            CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        }
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CPAPR_OK;
}

cpapr_status cpapr_get_state(cpapr_ctx *ctx, double *lambda, double *const *factors, double *const *phi_prev,
                             int64_t *outer_done) {
    API_ENTER(ctx);
    CPAPR_TRY(cpapr_get_model(ctx, lambda, factors));
    if (phi_prev)
        for (int m = 0; m < ctx->N; ++m) {
            if (!phi_prev[m]) continue;
            CPAPR_TRY(download_matrix(ctx, ctx->Phi[m], ctx->dims[m], phi_prev[m]));
            CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        }
    if (outer_done) *outer_done = ctx->k_total;
    return CPAPR_OK;
}

cpapr_status cpapr_set_state(cpapr_ctx *ctx, const double *lambda, const double *const *factors,
                             const double *const *phi_prev, int64_t outer_done) {
    API_ENTER(ctx);
    if (outer_done < 0) return fail(ctx, CPAPR_E_ARG, "outer_done must be >= 0");
    CPAPR_TRY(cpapr_set_model(ctx, lambda, factors));
    if (phi_prev) {
        CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, 16, ctx->stream));
        for (int m = 0; m < ctx->N; ++m)
            if (phi_prev[m]) {
                CPAPR_TRY(upload_matrix(ctx, phi_prev[m], ctx->dims[m], ctx->Phi[m]));
                // Phi rows of empty slices are zero by definition (and the
                // kernels rely on it)
                CPAPR_TRY(launch_zero_empty(ctx, m, ctx->Phi[m]));
            }
        int32_t flags[4] = {0, 0, 0, 0};
        CPAPR_CUDA(ctx, cudaMemcpyAsync(flags, ctx->errflag, 16, cudaMemcpyDeviceToHost, ctx->stream));
        CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (flags[2]) {
            ctx->model_set = false;
            return fail(ctx, CPAPR_E_VALUE, "phi_prev entries must be finite and >= 0");
        }
    }
    ctx->k_total = outer_done;
    return CPAPR_OK;
}

// After a call's last synchronisation: did a bounded device-side wait give
// up?  (errflag[3]; a call without one, such as cpapr_phi_noalloc, leaves it
// for the next call that checks.)
static cpapr_status check_waits(cpapr_ctx *ctx) {
    int32_t f = 0;
    CPAPR_CUDA(ctx, cudaMemcpyAsync(&f, ctx->errflag + 3, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!f) return CPAPR_OK;
    CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->errflag + 3, 0, 4, ctx->stream));
    // tiles that gave up never counted their partials: clear the counters
    for (int n = 0; n < ctx->N; ++n)
        if (ctx->mode[n].splitcnt)
            CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->mode[n].splitcnt, 0,
                                            (size_t)std::max(ctx->mode[n].nsplit, 1) * 4, ctx->stream));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return fail(ctx, CPAPR_E_TIMEOUT, "a device-side staging wait gave up; the results of this call are incomplete");
}

static cpapr_status check_mode(cpapr_ctx *ctx, int32_t mode) {
    if (mode < 0 || mode >= ctx->N) return fail(ctx, CPAPR_E_ARG, "mode out of range");
    if (!ctx->model_set) return fail(ctx, CPAPR_E_STATE, "no model set");
    return CPAPR_OK;
}

cpapr_status cpapr_phi(cpapr_ctx *ctx, int32_t mode, const double *B, double *out) {
    API_ENTER(ctx);
    CPAPR_TRY(check_mode(ctx, mode));
    if (!out) return fail(ctx, CPAPR_E_ARG, "out is NULL");
    if (B) {
        CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, 16, ctx->stream));
        CPAPR_TRY(upload_matrix(ctx, B, ctx->dims[mode], ctx->B));
    } else {
        CPAPR_TRY(launch_scale_b(ctx, mode, ctx->B));
    }
    // Phi[mode] holds the previous iteration's Phi that S reads: compute into
    // the separate output buffer instead.
    CPAPR_TRY(launch_pi_build(ctx, mode));
    CPAPR_TRY(launch_phi(ctx, mode, OP_PHI, ctx->B, ctx->outbuf, nullptr));
    CPAPR_TRY(download_matrix(ctx, ctx->outbuf, ctx->dims[mode], out));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_waits(ctx);
}

cpapr_status cpapr_mttkrp(cpapr_ctx *ctx, int32_t mode, double *out) {
    API_ENTER(ctx);
    CPAPR_TRY(check_mode(ctx, mode));
    if (!out) return fail(ctx, CPAPR_E_ARG, "out is NULL");
    CPAPR_TRY(launch_phi(ctx, mode, OP_MTTKRP, nullptr, ctx->outbuf, nullptr));
    CPAPR_TRY(download_matrix(ctx, ctx->outbuf, ctx->dims[mode], out));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_waits(ctx);
}

cpapr_status cpapr_loglik(cpapr_ctx *ctx, double *out) {
    API_ENTER(ctx);
    if (!out) return fail(ctx, CPAPR_E_ARG, "out is NULL");
    if (!ctx->model_set) return fail(ctx, CPAPR_E_STATE, "no model set");
    CPAPR_TRY(launch_loglik(ctx, ctx->scalars));
    CPAPR_CUDA(ctx, cudaMemcpyAsync(out, ctx->scalars, 8, cudaMemcpyDefault, ctx->stream));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_waits(ctx);
}

cpapr_status cpapr_mu_solve(cpapr_ctx *ctx, double tol, int32_t max_outer, int32_t max_inner, cpapr_result *res,
                            int32_t *inner_trace, double *ll_trace, double *kkt_trace) {
    API_ENTER(ctx);
    if (!res) return fail(ctx, CPAPR_E_ARG, "res is NULL");
    if (max_outer < 0 || max_inner < 1 || !(tol >= 0.0)) return fail(ctx, CPAPR_E_ARG, "bad tol / iteration bounds");
    if (!ctx->model_set) return fail(ctx, CPAPR_E_STATE, "no model set");
    CPAPR_TRY(mu_solve(ctx, tol, max_outer, max_inner, res, inner_trace, ll_trace, kkt_trace));
    return check_waits(ctx);
}

cpapr_status cpapr_batch_mu_solve(cpapr_ctx *const *ctxs, int32_t count, double tol, int32_t max_outer,
                                  int32_t max_inner, cpapr_result *results) {
    if (!ctxs || !results || count < 0) return fail(nullptr, CPAPR_E_ARG, "bad batch arguments");
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i]) return fail(nullptr, CPAPR_E_ARG, "ctxs[i] is NULL");
        if (ctxs[i]->sticky) return CPAPR_E_CUDA;
        if (!ctxs[i]->model_set) return fail(ctxs[i], CPAPR_E_STATE, "no model set");
        if (ctxs[i]->esize != ctxs[0]->esize) return fail(nullptr, CPAPR_E_ARG, "mixed precisions in a batch");
    }
    if (max_outer < 0 || max_inner < 1 || !(tol >= 0.0)) return fail(nullptr, CPAPR_E_ARG, "bad tol / iteration bounds");
    const cpapr_status st = batch_mu_solve(ctxs, count, tol, max_outer, max_inner, results);
    if (st != CPAPR_OK) return st;
    for (int i = 0; i < count; ++i) CPAPR_TRY(check_waits(ctxs[i]));
    return CPAPR_OK;
}

cpapr_status cpapr_get_info(const cpapr_ctx *ctx, cpapr_info *info) {
    if (!ctx || !info) return CPAPR_E_ARG;
    std::memset(info, 0, sizeof(*info));
    info->nmodes = ctx->N;
    info->rank = ctx->R;
    info->rank_padded = ctx->Rp;
    info->precision = ctx->opt.precision;
    info->nnz = ctx->nnz;
    for (int m = 0; m < ctx->N; ++m) {
        info->dims[m] = ctx->dims[m];
        info->tile_nnz[m] = ctx->mode[m].tile_nnz;
        info->rank_lanes[m] = ctx->mode[m].lanes;
        info->reduction[m] = ctx->mode[m].reduction;
        info->ntiles[m] = ctx->mode[m].ntiles;
        info->nsplit[m] = ctx->mode[m].nsplit;
        info->pi_mode[m] = ctx->mode[m].pi ? CPAPR_PI_MATERIALISED : CPAPR_PI_FUSED;
    }
    info->device_bytes = ctx->device_bytes;
    info->kernel_launches = ctx->launches;
    info->l2_window_bytes = (int64_t)ctx->l2win.num_bytes;
    return CPAPR_OK;
}

cpapr_status cpapr_kernel_stats(cpapr_ctx *ctx, int32_t kind, int64_t *launches, double *total_ms, int32_t reset) {
    API_ENTER(ctx);
    if (kind < 0 || kind >= K_NKINDS) return fail(ctx, CPAPR_E_ARG, "bad kernel kind");
    prof_collect(ctx);
    if (launches) *launches = ctx->prof_launches[kind];
    if (total_ms) *total_ms = ctx->prof_ms[kind];
    if (reset) {
        ctx->prof_launches[kind] = 0;
        ctx->prof_ms[kind] = 0.0;
    }
    return CPAPR_OK;
}

}  // extern "C"
