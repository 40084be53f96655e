// Index builder: COO -> one mode-sorted layout per mode.
//
// The paper's Section "CP-APR MU Implementation and Parallelization" sorts
// the nonzeros once per mode at the start so that entries updating the same
// row of Phi^(n) are contiguous, and keeps N permutation arrays.  Here the
// permutation is applied once: each mode gets its own physically permuted
// copy of the other modes' coordinates and of the values, so the hot loop
// streams them contiguously instead of reading through a permutation array
// (the paper notes that indirect access through the permutation is slow).
//
// Steps (all on the device; the copies of step 1 run on a second stream and
// overlap the sorts of the modes already copied):
//   1. copy the int64 COO in, check 0 <= i_m < I_m and x finite and >= 0,
//      narrow coordinates to int32;
//   2. per mode n: stable LSD radix sort of (i_n, position) with 8-bit digits
//      (per-tile digit histograms, an exclusive scan, and a stable scatter
//      that ranks equal digits with warp match/ballot);
//   3. seg[i] = first sorted position of row i (I_n + 1 offsets) and the
//      sorted row ids themselves (the tile kernels stage them with the tile);
//   4. gather the other modes' coordinates and the values in sorted order;
//   5. tile tables: tiles of tile_nnz consecutive sorted nonzeros, the row
//      holding each tile's first nonzero, the rows that span more than one
//      tile with, per tile, the split its head and tail partials belong to,
//      and one counter per split.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace cpapr {

// ---------------------------------------------------------------------------
// exclusive scan of uint32 (in place), three kernels + recursion on block sums
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total, uint32_t *sm_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? sm_warp[lane] : 0u;
        uint32_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sm_warp[lane] = s - w;
        if (lane == nw - 1) sm_warp[32] = s;
    }
    __syncthreads();
    uint32_t r = sm_warp[warp] + x - v;
    *total = sm_warp[32];
    __syncthreads();
    return r;
}

__global__ void scan_reduce_kernel(const uint32_t *__restrict__ d, int64_t n, uint32_t *__restrict__ bsum) {
    __shared__ uint32_t smw[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += d[base + k];
    uint32_t tot;
    block_exclusive_scan(s, &tot, smw);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void scan_apply_kernel(uint32_t *__restrict__ d, int64_t n, const uint32_t *__restrict__ boff,
                                  uint32_t *__restrict__ total_out) {
    __shared__ uint32_t smw[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? d[base + k] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(s, &tot, smw) + (boff ? boff[blockIdx.x] : 0u);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) d[base + k] = pre;
        pre += v[k];
    }
    if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *total_out = pre;
}

cpapr_status exclusive_scan_u32(cpapr_ctx *ctx, uint32_t *data, int64_t n, uint32_t *total_out_dev) {
    if (n <= 0) {
        if (total_out_dev) CPAPR_CUDA(ctx, cudaMemsetAsync(total_out_dev, 0, 4, ctx->stream));
        return CPAPR_OK;
    }
    int64_t nb = ceil_div(n, kScanTile);
    uint32_t *bs = nullptr;
    if (nb > 1) {
        CPAPR_CUDA(ctx, lib_malloc((void **)&bs, nb * 4, ctx->stream));
        scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(data, n, bs);
        count_launch(ctx);
        CPAPR_CUDA(ctx, cudaGetLastError());
        cpapr_status st = exclusive_scan_u32(ctx, bs, nb, nullptr);
        if (st != CPAPR_OK) return st;
    }
    scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(data, n, bs, total_out_dev);
    count_launch(ctx);
    CPAPR_CUDA(ctx, cudaGetLastError());
    if (bs) CPAPR_CUDA(ctx, cudaFreeAsync(bs, ctx->stream));
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// input conversion and validation
// ---------------------------------------------------------------------------
__global__ void narrow_check_kernel(const int64_t *__restrict__ src, int64_t nnz, int64_t dim,
                                    int32_t *__restrict__ dst, int32_t *__restrict__ errflag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = src[j];
        if (v < 0 || v >= dim) {
            atomicOr(&errflag[0], 1);
            v = 0;
        }
        dst[j] = (int32_t)v;
    }
}

// copies the values (read in place from device memory) and checks them
__global__ void copy_check_values_kernel(const double *__restrict__ src, int64_t nnz, double *__restrict__ dst,
                                         int32_t *__restrict__ errflag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x) {
        double x = src[j];
        if (!(x >= 0.0) || isinf(x)) atomicOr(&errflag[1], 1);
        dst[j] = x;
    }
}

__global__ void check_values_kernel(const double *__restrict__ v, int64_t nnz, int32_t *__restrict__ errflag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x) {
        double x = v[j];
        if (!(x >= 0.0) || isinf(x)) atomicOr(&errflag[1], 1);
    }
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint32 key, uint32 value)
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsThreads * kRsRounds;

__global__ void iota_kernel(uint32_t *__restrict__ v, int64_t n) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        v[j] = (uint32_t)j;
}

__global__ void rs_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ counts,
                               int ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int k = threadIdx.x; k < kRsTile; k += kRsThreads) {
        int64_t p = base + k;
        if (p < n) atomicAdd(&h[(keys[p] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: elements of a tile are visited in position order, 256 at a
// time; inside a round, equal digits are ranked by lane (match_any) and by
// warp (per-warp counts turned into offsets), so the output keeps the input
// order among equal digits.
__global__ void rs_scatter_kernel(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                  uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                                  const uint32_t *__restrict__ offsets, int ntiles) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kRsThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = offsets[(int64_t)tid * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int q = 0; q < kRsRounds; ++q) {
#pragma unroll
        for (int w = 0; w < kRsThreads / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        int64_t p = base + (int64_t)q * kRsThreads + tid;
        bool valid = p < n;
        uint32_t key = valid ? kin[p] : 0u;
        uint32_t val = valid ? vin[p] : 0u;
        uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t r = run[tid];
#pragma unroll
            for (int w = 0; w < kRsThreads / 32; ++w) {
                uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = r;
                r += c;
            }
            run[tid] = r;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wcnt[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

// Sorts keys/vals (n entries) by the low `bits` bits of the key, stably.
// tmp buffers must hold n entries each.  Result ends in keys/vals.
static cpapr_status radix_sort(cpapr_ctx *ctx, uint32_t *keys, uint32_t *vals, uint32_t *tk, uint32_t *tv,
                               int64_t n, int bits) {
    if (n <= 1 || bits <= 0) return CPAPR_OK;
    int ntiles = (int)ceil_div(n, kRsTile);
    uint32_t *counts = nullptr;
    CPAPR_CUDA(ctx, lib_malloc((void **)&counts, (size_t)256 * ntiles * 4, ctx->stream));
    uint32_t *ka = keys, *va = vals, *kb = tk, *vb = tv;
    int passes = (bits + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        int shift = ps * 8;
        rs_hist_kernel<<<ntiles, kRsThreads, 0, ctx->stream>>>(ka, n, shift, counts, ntiles);
        CPAPR_CUDA(ctx, cudaGetLastError());
        CPAPR_TRY(exclusive_scan_u32(ctx, counts, (int64_t)256 * ntiles, nullptr));
        rs_scatter_kernel<<<ntiles, kRsThreads, 0, ctx->stream>>>(ka, va, kb, vb, n, shift, counts, ntiles);
        count_launch(ctx, 2);
        CPAPR_CUDA(ctx, cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        CPAPR_CUDA(ctx, cudaMemcpyAsync(keys, ka, n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        CPAPR_CUDA(ctx, cudaMemcpyAsync(vals, va, n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    CPAPR_CUDA(ctx, cudaFreeAsync(counts, ctx->stream));
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// segment offsets and permuted copies
// ---------------------------------------------------------------------------
__global__ void seg_kernel(const uint32_t *__restrict__ skeys, int64_t nnz, int32_t In, int32_t *__restrict__ seg) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t key = (int32_t)skeys[k];
        int32_t prev = k > 0 ? (int32_t)skeys[k - 1] : -1;
        for (int32_t r = prev + 1; r <= key; ++r) seg[r] = (int32_t)k;
        if (k == nnz - 1)
            for (int32_t r = key + 1; r <= In; ++r) seg[r] = (int32_t)nnz;
    }
}

__global__ void empty_flags_kernel(const int32_t *__restrict__ seg, int32_t In, uint32_t *__restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < In; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = seg[i] == seg[i + 1] ? 1u : 0u;
}

__global__ void empty_write_kernel(const int32_t *__restrict__ seg, int32_t In, const uint32_t *__restrict__ pos,
                                   int32_t *__restrict__ erows) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < In; i += (int64_t)gridDim.x * blockDim.x)
        if (seg[i] == seg[i + 1]) erows[pos[i]] = (int32_t)i;
}

// nzrow[k] = the k-th row holding nonzeros (pos: exclusive scan of the
// empty-row flags, so row i is preceded by pos[i] empty rows)
__global__ void nzrow_kernel(const int32_t *__restrict__ seg, int32_t In, const uint32_t *__restrict__ pos,
                             int32_t *__restrict__ nzrow) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < In; i += (int64_t)gridDim.x * blockDim.x)
        if (seg[i] != seg[i + 1]) nzrow[i - pos[i]] = (int32_t)i;
}

// Row-start bits of the sorted positions: bit p of word p / 32 is set where
// a row begins (p = 0 or keys[p] != keys[p - 1]); one warp per word.
__global__ void rstart_kernel(const uint32_t *__restrict__ keys, int64_t nnz, uint32_t *__restrict__ bits) {
    const int64_t nwords = (nnz + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nwords;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t p = w * 32 + lane;
        const bool start = p < nnz && (p == 0 || keys[p] != keys[p - 1]);
        const uint32_t b = __ballot_sync(0xffffffffu, start);
        if (lane == 0) bits[w] = b;
    }
}

__global__ void gather_i32_kernel(const int32_t *__restrict__ src, const uint32_t *__restrict__ perm, int64_t n,
                                  int32_t *__restrict__ dst) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[perm[k]];
}

template <typename T>
__global__ void gather_val_kernel(const double *__restrict__ src, const uint32_t *__restrict__ perm, int64_t n,
                                  T *__restrict__ dst) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = (T)src[perm[k]];
}

static unsigned grid_for(int64_t n, int threads = 256) {
    int64_t g = ceil_div(n, threads);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// A pointer kernels read in place: device or managed memory.  Host memory,
// pinned or not, goes through a staging copy: on GB300 the copy engines
// move pinned host memory faster (207 GB/s measured) than kernels reading
// it in place over the host link (create 2.94 -> 4.35 ms when tried).
static const void *device_view(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.devicePointer;
    return nullptr;
}

cpapr_status build_layouts(cpapr_ctx *ctx, const int64_t *const *idx_in, const double *vals_in) {
    const int N = ctx->N;
    const int64_t nnz = ctx->nnz;
    cudaStream_t s = ctx->stream;
    // padded length so vector and bulk loads past the end stay inside the buffer
    ctx->nnz_pad = ceil_div(std::max<int64_t>(nnz, 1), 256) * 256 + 256;
    const int64_t np = ctx->nnz_pad;

    // The input crosses to the device on a second stream, one array at a
    // time, while the main stream narrows and sorts the modes that have
    // arrived (mode n's sort needs only its own coordinates); the gathers,
    // which need every array, follow.  Invalid input is flagged by the
    // device (and clamped, so every later index stays in bounds) and
    // reported once everything has run.
    int32_t *idx32[kMaxModes] = {};
    int64_t *stage[kMaxModes] = {};
    uint32_t *perm[kMaxModes] = {};
    uint32_t *flags[kMaxModes] = {};
    double *vals = nullptr;
    uint32_t *keys = nullptr, *tk = nullptr, *tv = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[kMaxModes + 2] = {};
    auto cleanup = [&]() {
        // the copies finish before their buffers go back to the pool
        if (cs) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e, cs);
                cudaStreamWaitEvent(s, e, 0);
                cudaEventDestroy(e);
            }
        }
        for (int m = 0; m < N; ++m) {
            if (idx32[m]) cudaFreeAsync(idx32[m], s);
            if (stage[m]) cudaFreeAsync(stage[m], s);
            if (perm[m]) cudaFreeAsync(perm[m], s);
            if (flags[m]) cudaFreeAsync(flags[m], s);
        }
        if (vals) cudaFreeAsync(vals, s);
        if (keys) cudaFreeAsync(keys, s);
        if (tk) cudaFreeAsync(tk, s);
        if (tv) cudaFreeAsync(tv, s);
        cudaStreamSynchronize(s);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
    };
#define BL_CUDA(call)                                      \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) {                           \
            cleanup();                                     \
            return cuda_fail(ctx, _e, #call);              \
        }                                                  \
    } while (0)
#define BL_TRY(expr)                   \
    do {                               \
        cpapr_status _st = (expr);     \
        if (_st != CPAPR_OK) {         \
            cleanup();                 \
            return _st;                \
        }                              \
    } while (0)

    const int64_t nb = std::max<int64_t>(nnz, 1);
    BL_CUDA(cudaMemsetAsync(ctx->errflag, 0, 16, s));
    // the layouts themselves (owned by the context); only the padding past
    // nnz needs a value before the streams are written
    for (int n = 0; n < N; ++n) {
        ModeLayout &L = ctx->mode[n];
        L.In = (int32_t)ctx->dims[n];
        void *p = nullptr;
        BL_TRY(dev_alloc(ctx, &p, (size_t)(L.In + 1) * 4));
        L.seg = (int32_t *)p;
        // row-start bits: a word per 32 sorted positions, zero past nnz, with
        // whole 16-byte groups to spare for the tile kernels' bulk copies
        const size_t words = ((size_t)(np + 31) / 32 + 8 + 3) & ~(size_t)3;
        BL_TRY(dev_alloc(ctx, &p, words * 4));
        L.rstart = (uint32_t *)p;
        BL_CUDA(cudaMemsetAsync(L.rstart, 0, words * 4, s));
        for (int k = 0; k < N - 1; ++k) {
            BL_TRY(dev_alloc(ctx, &p, (size_t)np * 4));
            L.idx[k] = (int32_t *)p;
            BL_CUDA(cudaMemsetAsync(L.idx[k] + nnz, 0, (size_t)(np - nnz) * 4, s));
        }
        BL_TRY(dev_alloc(ctx, &p, (size_t)np * ctx->esize));
        L.val = p;
        BL_CUDA(cudaMemsetAsync((char *)p + (size_t)nnz * ctx->esize, 0, (size_t)(np - nnz) * ctx->esize, s));
        if (nnz == 0) BL_CUDA(cudaMemsetAsync(L.seg, 0, (size_t)(L.In + 1) * 4, s));
    }
    if (nnz > 0) {
        const int64_t *src[kMaxModes] = {};
        for (int m = 0; m < N; ++m) src[m] = static_cast<const int64_t *>(device_view(idx_in[m]));
        const double *vsrc = static_cast<const double *>(device_view(vals_in));
        for (int m = 0; m < N; ++m) {
            if (!src[m]) BL_CUDA(lib_malloc((void **)&stage[m], nb * 8, s));
            BL_CUDA(lib_malloc((void **)&idx32[m], nb * 4, s));
            BL_CUDA(lib_malloc((void **)&perm[m], nb * 4, s));
        }
        BL_CUDA(lib_malloc((void **)&vals, nb * 8, s));
        BL_CUDA(lib_malloc((void **)&keys, nb * 4, s));
        BL_CUDA(lib_malloc((void **)&tk, nb * 4, s));
        BL_CUDA(lib_malloc((void **)&tv, nb * 4, s));
        BL_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        for (int k = 0; k <= N + 1; ++k) BL_CUDA(cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming));
        // the copy stream starts after the allocations above
        BL_CUDA(cudaEventRecord(ev[N + 1], s));
        BL_CUDA(cudaStreamWaitEvent(cs, ev[N + 1], 0));
        for (int n = 0; n < N; ++n) {
            if (src[n]) {
                // device input: read in place by the narrowing kernel, on the copy stream
                narrow_check_kernel<<<grid_for(nnz), 256, 0, cs>>>(src[n], nnz, ctx->dims[n], idx32[n], ctx->errflag);
                BL_CUDA(cudaGetLastError());
                BL_CUDA(cudaEventRecord(ev[n], cs));
                BL_CUDA(cudaStreamWaitEvent(s, ev[n], 0));
            } else {
                BL_CUDA(cudaMemcpyAsync(stage[n], idx_in[n], nnz * 8, cudaMemcpyDefault, cs));
                BL_CUDA(cudaEventRecord(ev[n], cs));
                BL_CUDA(cudaStreamWaitEvent(s, ev[n], 0));
                narrow_check_kernel<<<grid_for(nnz), 256, 0, s>>>(stage[n], nnz, ctx->dims[n], idx32[n], ctx->errflag);
                BL_CUDA(cudaGetLastError());
                BL_CUDA(cudaFreeAsync(stage[n], s));
                stage[n] = nullptr;
            }
            // sort mode n by its row: row offsets (seg), row-start bits, the permutation
            ModeLayout &L = ctx->mode[n];
            BL_CUDA(cudaMemcpyAsync(keys, idx32[n], nnz * 4, cudaMemcpyDeviceToDevice, s));
            iota_kernel<<<grid_for(nnz), 256, 0, s>>>(perm[n], nnz);
            BL_CUDA(cudaGetLastError());
            int bits = 0;
            while (bits < 31 && ((int64_t)1 << bits) < (int64_t)L.In) ++bits;
            BL_TRY(radix_sort(ctx, keys, perm[n], tk, tv, nnz, bits));
            seg_kernel<<<grid_for(nnz), 256, 0, s>>>(keys, nnz, L.In, L.seg);
            BL_CUDA(cudaGetLastError());
            rstart_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(keys, nnz, L.rstart);
            BL_CUDA(cudaGetLastError());
            count_launch(ctx, 4);  // narrow, iota, seg, row-start bits
        }
        if (vsrc) {
            copy_check_values_kernel<<<grid_for(nnz), 256, 0, cs>>>(vsrc, nnz, vals, ctx->errflag);
            BL_CUDA(cudaGetLastError());
            BL_CUDA(cudaEventRecord(ev[N], cs));
            BL_CUDA(cudaStreamWaitEvent(s, ev[N], 0));
        } else {
            BL_CUDA(cudaMemcpyAsync(vals, vals_in, nnz * 8, cudaMemcpyDefault, cs));
            BL_CUDA(cudaEventRecord(ev[N], cs));
            BL_CUDA(cudaStreamWaitEvent(s, ev[N], 0));
            check_values_kernel<<<grid_for(nnz), 256, 0, s>>>(vals, nnz, ctx->errflag);
            BL_CUDA(cudaGetLastError());
        }
        count_launch(ctx);
        // every mode's other coordinates and values in its sorted order
        for (int n = 0; n < N; ++n) {
            ModeLayout &L = ctx->mode[n];
            int k = 0;
            for (int m = 0; m < N; ++m) {
                if (m == n) continue;
                gather_i32_kernel<<<grid_for(nnz), 256, 0, s>>>(idx32[m], perm[n], nnz, L.idx[k]);
                BL_CUDA(cudaGetLastError());
                ++k;
            }
            if (ctx->esize == 8)
                gather_val_kernel<double><<<grid_for(nnz), 256, 0, s>>>(vals, perm[n], nnz, (double *)L.val);
            else
                gather_val_kernel<float><<<grid_for(nnz), 256, 0, s>>>(vals, perm[n], nnz, (float *)L.val);
            BL_CUDA(cudaGetLastError());
            count_launch(ctx, N);
        }
    }
    // per mode: the rows without nonzeros (their Phi row is zero); the counts
    // of all modes come back in one synchronisation, with the input flags
    for (int n = 0; n < N; ++n) {
        ModeLayout &L = ctx->mode[n];
        BL_CUDA(lib_malloc((void **)&flags[n], (size_t)(L.In + 1) * 4, s));
        empty_flags_kernel<<<grid_for(L.In), 256, 0, s>>>(L.seg, L.In, flags[n]);
        BL_CUDA(cudaGetLastError());
        BL_TRY(exclusive_scan_u32(ctx, flags[n], L.In, flags[n] + L.In));
        count_launch(ctx);
    }
    uint32_t totals[kMaxModes] = {};
    int32_t hflag[4] = {0, 0, 0, 0};
    for (int n = 0; n < N; ++n)
        BL_CUDA(cudaMemcpyAsync(&totals[n], flags[n] + ctx->mode[n].In, 4, cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaMemcpyAsync(hflag, ctx->errflag, 16, cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaStreamSynchronize(s));
    if (hflag[0]) {
        cleanup();
        return fail(ctx, CPAPR_E_RANGE, "a coordinate lies outside [0, I_m)");
    }
    if (hflag[1]) {
        cleanup();
        return fail(ctx, CPAPR_E_VALUE, "a tensor value is negative, NaN or infinite");
    }
    for (int n = 0; n < N; ++n) {
        ModeLayout &L = ctx->mode[n];
        L.nempty = (int32_t)totals[n];
        void *p = nullptr;
        BL_TRY(dev_alloc(ctx, &p, (size_t)std::max<int32_t>(L.nempty, 1) * 4));
        L.erows = (int32_t *)p;
        empty_write_kernel<<<grid_for(L.In), 256, 0, s>>>(L.seg, L.In, flags[n], L.erows);
        BL_CUDA(cudaGetLastError());
        // the rows with nonzeros, increasing (+ 16-byte groups to spare for bulk copies)
        L.K = L.In - L.nempty;
        BL_TRY(dev_alloc(ctx, &p, (size_t)(L.K + 8) * 4));
        L.nzrow = (int32_t *)p;
        BL_CUDA(cudaMemsetAsync(L.nzrow, 0, (size_t)(L.K + 8) * 4, s));
        nzrow_kernel<<<grid_for(L.In), 256, 0, s>>>(L.seg, L.In, flags[n], L.nzrow);
        BL_CUDA(cudaGetLastError());
        count_launch(ctx, 2);
    }
    cleanup();
    BL_CUDA(cudaStreamSynchronize(s));
#undef BL_CUDA
#undef BL_TRY
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// tile tables
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t upper_bound_seg(const int32_t *seg, int32_t lo, int32_t hi, int64_t p) {
    // first i in [lo, hi) with seg[i] > p (hi if none)
    while (lo < hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)seg[mid] > p)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

__global__ void tile_rows_kernel(const int32_t *__restrict__ seg, int32_t In, int32_t T, int32_t ntiles,
                                 int32_t *__restrict__ row_first) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    row_first[t] = upper_bound_seg(seg, 0, In, (int64_t)t * T) - 1;
}

// krow[t] = index in nzrow of row_first[t] (nzrow is increasing and holds it);
// krow[ntiles] = K - 1, the last row
__global__ void tile_krow_kernel(const int32_t *__restrict__ nzrow, int32_t K, const int32_t *__restrict__ row_first,
                                 int32_t ntiles, int32_t *__restrict__ krow) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    if (t == ntiles) {
        krow[t] = K - 1;
        return;
    }
    const int32_t r = row_first[t];
    int32_t lo = 0, hi = K;  // first k with nzrow[k] >= r
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (nzrow[mid] < r)
            lo = mid + 1;
        else
            hi = mid;
    }
    krow[t] = lo;
}

__global__ void split_flags_kernel(const int32_t *__restrict__ seg, const int32_t *__restrict__ row_first, int32_t T,
                                   int32_t ntiles, uint32_t *__restrict__ flag) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    uint32_t f = 0;
    if (t >= 1) {
        int32_t r = row_first[t];
        bool cut = (int64_t)seg[r] < (int64_t)t * T;
        bool prev_cut = t >= 2 && row_first[t - 1] == r && (int64_t)seg[r] < (int64_t)(t - 1) * T;
        f = (cut && !prev_cut) ? 1u : 0u;
    }
    flag[t] = f;
}

__global__ void split_write_kernel(const int32_t *__restrict__ seg, const int32_t *__restrict__ row_first, int32_t T,
                                   int32_t ntiles, const uint32_t *__restrict__ pos, int32_t *__restrict__ split) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 1 || t >= ntiles) return;
    int32_t r = row_first[t];
    bool cut = (int64_t)seg[r] < (int64_t)t * T;
    bool prev_cut = t >= 2 && row_first[t - 1] == r && (int64_t)seg[r] < (int64_t)(t - 1) * T;
    if (cut && !prev_cut) {
        uint32_t k = pos[t];
        split[3 * k + 0] = r;
        split[3 * k + 1] = t - 1;
        split[3 * k + 2] = (int32_t)(((int64_t)seg[r + 1] - 1) / T);
    }
}

// tsplit[2t] = split whose row holds tile t's head partial (the row began in
// an earlier tile), tsplit[2t+1] = split whose first tile is t (tile t's tail
// partial); -1 where there is none.  pos = exclusive scan of the split-start
// flags, total = their sum: the splits started at or before tile u number
// incl(u) = pos[u + 1] (total for the last tile).
__global__ void tile_split_kernel(const int32_t *__restrict__ seg, const int32_t *__restrict__ row_first, int32_t T,
                                  int32_t ntiles, const uint32_t *__restrict__ pos, const uint32_t *__restrict__ total,
                                  int32_t *__restrict__ tsplit) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    auto incl = [&](int u) -> int32_t { return (int32_t)(u + 1 < ntiles ? pos[u + 1] : *total); };
    int32_t head = -1, tail = -1;
    if (t >= 1 && (int64_t)seg[row_first[t]] < (int64_t)t * T) head = incl(t) - 1;
    if (t + 1 < ntiles && incl(t + 1) - (int32_t)pos[t + 1] == 1) tail = (int32_t)pos[t + 1];
    tsplit[2 * t] = head;
    tsplit[2 * t + 1] = tail;
}

cpapr_status build_tiles(cpapr_ctx *ctx, int n, int tile_nnz) {
    ModeLayout &L = ctx->mode[n];
    cudaStream_t s = ctx->stream;
    if (L.row_first) cudaFreeAsync(L.row_first, s);
    if (L.krow) cudaFreeAsync(L.krow, s);
    if (L.split) cudaFreeAsync(L.split, s);
    if (L.tsplit) cudaFreeAsync(L.tsplit, s);
    if (L.splitcnt) cudaFreeAsync(L.splitcnt, s);
    L.row_first = L.krow = L.split = L.tsplit = L.splitcnt = nullptr;
    L.tile_nnz = tile_nnz;
    L.ntiles = (int32_t)ceil_div(ctx->nnz, tile_nnz);
    L.nsplit = 0;
    const int nt = L.ntiles;
    CPAPR_CUDA(ctx, lib_malloc((void **)&L.row_first, (size_t)std::max(nt, 1) * 4, s));
    count_launch(ctx, nt >= 2 ? 3 : 1);
    tile_rows_kernel<<<(unsigned)ceil_div(std::max(nt, 1), 256), 256, 0, s>>>(L.seg, L.In, tile_nnz, nt, L.row_first);
    CPAPR_CUDA(ctx, cudaGetLastError());
    CPAPR_CUDA(ctx, lib_malloc((void **)&L.krow, (size_t)(nt + 1) * 4, s));
    if (ctx->nnz > 0) {
        tile_krow_kernel<<<(unsigned)ceil_div(nt + 1, 256), 256, 0, s>>>(L.nzrow, L.K, L.row_first, nt, L.krow);
        CPAPR_CUDA(ctx, cudaGetLastError());
        count_launch(ctx);
    }
    if (nt >= 2) {
        uint32_t *flag = nullptr, *dtot = nullptr;
        CPAPR_CUDA(ctx, lib_malloc((void **)&flag, (size_t)nt * 4 + 4, s));
        dtot = flag + nt;
        split_flags_kernel<<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(L.seg, L.row_first, tile_nnz, nt, flag);
        CPAPR_CUDA(ctx, cudaGetLastError());
        CPAPR_TRY(exclusive_scan_u32(ctx, flag, nt, dtot));
        uint32_t total = 0;
        CPAPR_CUDA(ctx, cudaMemcpyAsync(&total, dtot, 4, cudaMemcpyDeviceToHost, s));
        CPAPR_CUDA(ctx, cudaStreamSynchronize(s));
        L.nsplit = (int32_t)total;
        CPAPR_CUDA(ctx, lib_malloc((void **)&L.split, (size_t)std::max<int>(L.nsplit, 1) * 12, s));
        split_write_kernel<<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(L.seg, L.row_first, tile_nnz, nt, flag, L.split);
        CPAPR_CUDA(ctx, cudaGetLastError());
        CPAPR_CUDA(ctx, lib_malloc((void **)&L.tsplit, (size_t)nt * 8, s));
        tile_split_kernel<<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(L.seg, L.row_first, tile_nnz, nt, flag, dtot,
                                                                      L.tsplit);
        count_launch(ctx);
        CPAPR_CUDA(ctx, cudaGetLastError());
        CPAPR_CUDA(ctx, cudaFreeAsync(flag, s));
    } else {
        CPAPR_CUDA(ctx, lib_malloc((void **)&L.split, 12, s));
        CPAPR_CUDA(ctx, lib_malloc((void **)&L.tsplit, (size_t)std::max(nt, 1) * 8, s));
        CPAPR_CUDA(ctx, cudaMemsetAsync(L.tsplit, 0xff, (size_t)std::max(nt, 1) * 8, s));
    }
    CPAPR_CUDA(ctx, lib_malloc((void **)&L.splitcnt, (size_t)std::max(L.nsplit, 1) * 4, s));
    CPAPR_CUDA(ctx, cudaMemsetAsync(L.splitcnt, 0, (size_t)std::max(L.nsplit, 1) * 4, s));
    // the carry buffer holds two partial rows per tile
    int64_t need = (int64_t)2 * std::max(nt, 1) * ctx->Rp;
    if (need > ctx->carry_elems) {
        if (ctx->carry) cudaFreeAsync(ctx->carry, s);
        ctx->carry = nullptr;
        CPAPR_CUDA(ctx, lib_malloc(&ctx->carry, (size_t)need * ctx->esize, s));
        ctx->carry_elems = need;
    }
    CPAPR_CUDA(ctx, cudaStreamSynchronize(s));
    return CPAPR_OK;
}

}  // namespace cpapr
