// Batched CP-APR MU: many tensors (uneven nonzero counts and ranks) solved
// together.  For every mode index n, each step of Algorithm 1 is one launch
// over all tensors:
//   batch_sb_kernel      B_t <- (A_t^(n) + S) Lambda_t           (row chunks)
//   batch_phi_kernel     Phi_t for every tile of every tensor    (persistent,
//                        blocks pull (tensor, tile) items from a counter;
//                        each item runs the tile body instantiated for its
//                        tensor's rank class)
//   batch_update_kernel  B_t <- B_t * Phi_t unless tensor t passed its KKT
//                        check; per-tensor bookkeeping by the last block of
//                        the tensor, loop condition by the last block overall
//   batch_colsum/scale   lambda_t <- e^T B_t, A_t <- B_t Lambda_t^-1
//   at the end           every tensor's log-likelihood: batch_scale_b_kernel,
//                        batch_phi_kernel<..., OP_LL> over mode 0's tiles,
//                        batch_ll_total_kernel
// The inner loop is one CUDA graph with a conditional WHILE node whose body
// is {phi, update}; it runs while any tensor still iterates.  Tensors
// that converged are masked on the device (their kernels return at once).
// Every reduction keeps a fixed order (results are reproducible run to run);
// a tensor's result equals solving it alone up to the order of the column
// sums (64-row chunks here, row-strided blocks in the single-tensor path).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ll_total.cuh"
#include "phi_kernels.cuh"

namespace cpapr {

cpapr_status configure_mode(cpapr_ctx *ctx, int n, int lanes, int tile, int reduction);

namespace {

constexpr int kChunkRows = 64;

struct BatchTensor {
    PhiArgs a;           // Phi arguments of this tensor for mode n
    int32_t cfg;         // index into the rank-class case list
    int32_t rp;
    int64_t rows;        // I_n
    void *A;             // A^(n)
    double *Am;          // FP32 form: FP64 masters of A^(n) and of B (else null)
    double *Bm;
    double *lambda;
    double *colpart;     // [nchunks][rp] column-sum partials
    int32_t chunk0, nchunks;
    double kappa, kappa_tol;
    const int32_t *erows;  // rows of mode n without nonzeros
    int64_t nempty;
};

constexpr int kEmptyChunk = 8192;  // (row, rank) elements per empty-row work item

struct BatchCtl {
    unsigned int tile_next, tile_exit, upd_blocks, active;
};

// rank classes of the batched Phi kernel: (ranks per lane, lanes), ranks up
// to 32.  All classes are inlined into one kernel, so its registers are the
// largest class's: FP32 keeps one float4 per lane; FP64 one lane up to 8
// ranks and lanes of 8 ranks above (the single-tensor heuristic's choices).
template <typename T> struct Classes;
template <> struct Classes<float> {
    static constexpr int n = 4;
    static constexpr int rpl[n] = {4, 4, 4, 4};
    static constexpr int g[n] = {1, 2, 4, 8};
};
template <> struct Classes<double> {
    static constexpr int n = 5;
    static constexpr int rpl[n] = {2, 4, 8, 8, 8};
    static constexpr int g[n] = {1, 1, 1, 2, 4};
};

template <typename T>
int class_for(int rp) {
    for (int k = 0; k < Classes<T>::n; ++k)
        if (Classes<T>::rpl[k] * Classes<T>::g[k] == rp) return k;
    return -1;
}

template <typename T, int RPL, int G>
__host__ __device__ constexpr int batch_unroll() {
    return (sizeof(T) == 8 && G == 1) ? 1 : 2;
}

template <typename T> __host__ __device__ constexpr int batch_threads() { return sizeof(T) == 8 ? 128 : 256; }
// resident blocks per SM the registers are held to (measured on GB300): the
// FP32 classes all keep one float4 per lane, like the single-tensor kernel's
// four-block case; every FP64 class fits three blocks (168 registers)
template <typename T> __host__ __device__ constexpr int batch_min_blocks() { return sizeof(T) == 8 ? 3 : 4; }

template <typename T, int NM1, int K, int OP, bool PI = false>
__device__ __forceinline__ bool run_class(const PhiArgs &a, int tile, unsigned char *smem, double *red, uint64_t *bar,
                                          uint32_t &phase) {
    constexpr int RPL = Classes<T>::rpl[K];
    constexpr int G = Classes<T>::g[K];
    return phi_tile_body<T, NM1, RPL, G, OP, batch_threads<T>(), batch_unroll<T, RPL, G>(), PI>(a, tile, smem, red,
                                                                                               bar, phase);
}

// One item's tile with the tensor's rank class; FP64 tensors with
// materialised Khatri-Rao rows (a.pi set) stream them.
template <typename T, int NM1, int OP, bool PI>
__device__ __forceinline__ bool run_item(const PhiArgs &a, int cfg, int tile, unsigned char *smem, double *red,
                                         uint64_t *bar, uint32_t &phase) {
    switch (cfg) {
        case 0: return run_class<T, NM1, 0, OP, PI>(a, tile, smem, red, bar, phase);
        case 1: return run_class<T, NM1, 1, OP, PI>(a, tile, smem, red, bar, phase);
        case 2: return run_class<T, NM1, 2, OP, PI>(a, tile, smem, red, bar, phase);
        case 3: return run_class<T, NM1, 3, OP, PI>(a, tile, smem, red, bar, phase);
        default:
            if constexpr (Classes<T>::n > 4)
                return run_class<T, NM1, (Classes<T>::n > 4 ? 4 : 0), OP, PI>(a, tile, smem, red, bar, phase);
            return true;
    }
}

// OP_PHI: Phi of every listed tile; OP_LL: the tile sums of x log m (the
// descriptors then carry the scaled mode-0 B and no inner-loop state).
template <typename T, int NM1, int OP = OP_PHI>
__global__ void __launch_bounds__(batch_threads<T>(), batch_min_blocks<T>()) batch_phi_kernel(const BatchTensor *__restrict__ desc,
                                                                       const int2 *__restrict__ items, int nitems,
                                                                       BatchCtl *ctl) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[batch_threads<T>() / 32];
    __shared__ int s_item;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) stage_barrier_init(&bar);
    __syncthreads();
    uint32_t phase = 0;
    bool ok = true;
    while (ok) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&ctl->tile_next, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const int2 w = items[it];
        const PhiArgs a = desc[w.x].a;
        if constexpr (sizeof(T) == 8 && OP == OP_PHI) {
            if (a.pi) {
                ok = run_item<T, NM1, OP, true>(a, desc[w.x].cfg, w.y, smem_raw, red, &bar, phase);
                continue;
            }
        }
        ok = run_item<T, NM1, OP, false>(a, desc[w.x].cfg, w.y, smem_raw, red, &bar, phase);
    }
    // the last block out resets the work counter for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned e = atomicAdd(&ctl->tile_exit, 1u);
        if (e == gridDim.x - 1) {
            ctl->tile_next = 0;
            ctl->tile_exit = 0;
            __threadfence();
        }
    }
}

constexpr int64_t kPiChunk = 1 << 16;  // 16-byte vectors of Khatri-Rao rows per build item

// Materialised Khatri-Rao rows of every tensor that streams them, for mode n:
// one block per (tensor, chunk of kPiChunk vectors) item; skipped tensors
// (converged or finished) keep their rows.
template <typename T, int NM1>
__global__ void __launch_bounds__(256) batch_pi_build_kernel(const BatchTensor *__restrict__ desc,
                                                             const int2 *__restrict__ items,
                                                             const int32_t *__restrict__ flags) {
    const int2 w = items[blockIdx.x];
    if (flags[2 * w.x]) return;
    const PhiArgs &a = desc[w.x].a;
    const int64_t total = a.nnz * (a.Rp / Vec16<T>::n);
    const int64_t e0 = (int64_t)w.y * kPiChunk;
    pi_build_range<T, NM1>(a, reinterpret_cast<T *>(const_cast<void *>(a.pi)), e0 + threadIdx.x,
                           min(e0 + kPiChunk, total), (int64_t)blockDim.x);
}

// flags[2t] = skip (converged or finished), flags[2t+1] = apply the shift S
template <typename T>
__global__ void __launch_bounds__(256) batch_sb_kernel(const BatchTensor *__restrict__ desc,
                                                       const int2 *__restrict__ chunks, const int32_t *__restrict__ flags) {
    const int2 w = chunks[blockIdx.x];
    const BatchTensor &d = desc[w.x];
    InnerState *inner = d.a.inner;
    const bool skip = flags[2 * w.x] != 0;
    if (w.y == 0 && threadIdx.x == 0) {
        inner->l = 0;
        inner->done = skip ? 1 : 0;
        inner->used = 0;
        inner->passed = 0;
        inner->counter = 0;
        inner->kkt[0] = 0ull;
        inner->kkt[1] = 0ull;
        inner->viol = 0.0;
    }
    if (skip) return;
    const int shift = flags[2 * w.x + 1];
    const int Rp = d.rp;
    const int64_t r0 = (int64_t)w.y * kChunkRows;
    const int64_t r1 = min(r0 + kChunkRows, d.rows);
    const T *A = reinterpret_cast<const T *>(d.A);
    const T *P = reinterpret_cast<const T *>(d.a.out);
    T *B = reinterpret_cast<T *>(const_cast<void *>(d.a.B));
    for (int64_t e = r0 * Rp + threadIdx.x; e < r1 * Rp; e += blockDim.x) {
        const double a = d.Am ? d.Am[e] : (double)A[e];
        const double s = (shift && a < d.kappa_tol && (double)P[e] > 1.0) ? d.kappa : 0.0;
        const double b = (a + s) * d.lambda[e & (Rp - 1)];  // Rp is a power of two
        if (d.Bm) d.Bm[e] = b;
        B[e] = (T)b;
    }
}

// KKT term of the empty rows for the first inner iteration (see empty_kkt_kernel).
template <typename T>
__global__ void __launch_bounds__(256) batch_empty_kkt_kernel(const BatchTensor *__restrict__ desc,
                                                              const int2 *__restrict__ items,
                                                              const int32_t *__restrict__ flags) {
    __shared__ double red[8];
    const int2 w = items[blockIdx.x];
    const BatchTensor &d = desc[w.x];
    if (flags[2 * w.x]) return;
    const int Rp = d.rp;
    const int lg = 31 - __clz(Rp);  // Rp is a power of two
    const int64_t q0 = (int64_t)w.y * kEmptyChunk;
    const int64_t q1 = min(q0 + kEmptyChunk, d.nempty * Rp);
    const T *B = reinterpret_cast<const T *>(d.a.B);
    T v = T(0);
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x)
        v = tmax(v, viol_t(B[(int64_t)d.erows[q >> lg] * Rp + (q & (Rp - 1))], T(0)));
    publish_kkt<256>((double)v, d.a.inner, red);
}

template <typename T>
__global__ void __launch_bounds__(256) batch_update_kernel(const BatchTensor *__restrict__ desc,
                                                           const int2 *__restrict__ chunks, unsigned int *chunk_count,
                                                           BatchCtl *ctl, double tol, int max_inner,
                                                           cudaGraphConditionalHandle cond, int use_cond) {
    __shared__ int s_l, s_done;
    __shared__ double s_viol;
    const int2 w = chunks[blockIdx.x];
    const BatchTensor &d = desc[w.x];
    InnerState *inner = d.a.inner;
    if (threadIdx.x == 0) {
        s_l = *((volatile int32_t *)&inner->l);
        s_done = *((volatile int32_t *)&inner->done);
        s_viol = __longlong_as_double((long long)inner->kkt[s_l & 1]);
    }
    __syncthreads();
    const int l = s_l, done = s_done;
    const double viol = s_viol;
    if (!done && !(viol < tol)) {
        const int Rp = d.rp;
        const int64_t r0 = (int64_t)w.y * kChunkRows;
        const int64_t r1 = min(r0 + kChunkRows, d.rows);
        if constexpr (sizeof(T) == 4) {
            // FP32 form: on the FP64 master, in pairs (a row is a whole number of them)
            for (int64_t e = r0 * Rp / 2 + threadIdx.x; e < r1 * Rp / 2; e += blockDim.x)
                master_mul(reinterpret_cast<double2 *>(d.Bm), reinterpret_cast<float2 *>(const_cast<void *>(d.a.B)),
                           reinterpret_cast<const float2 *>(d.a.out), e);
        } else {
            // 16-byte vectors (a row is a whole number of them)
            using V = typename Vec16<T>::type;
            constexpr int W = Vec16<T>::n;
            V *B = reinterpret_cast<V *>(const_cast<void *>(d.a.B));
            const V *P = reinterpret_cast<const V *>(d.a.out);
            for (int64_t e = r0 * Rp / W + threadIdx.x; e < r1 * Rp / W; e += blockDim.x) B[e] = vmul(B[e], P[e]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&chunk_count[w.x], 1u);
        if (prev == (unsigned)d.nchunks - 1) {  // last chunk of this tensor: its bookkeeping
            chunk_count[w.x] = 0;
            int now_done = done;
            if (!done) {
                inner->viol = viol;
                inner->used = l + 1;
                if (viol < tol) {
                    inner->done = 1;
                    inner->passed = 1;
                    now_done = 1;
                }
            }
            inner->l = l + 1;
            inner->kkt[(l + 1) & 1] = 0ull;
            if (!now_done && l + 1 < max_inner) atomicAdd(&ctl->active, 1u);
            __threadfence();
        }
        const unsigned g = atomicAdd(&ctl->upd_blocks, 1u);
        if (g == gridDim.x - 1) {  // last block overall: the loop condition
            __threadfence();
            const unsigned act = atomicAdd(&ctl->active, 0u);
            ctl->active = 0;
            ctl->upd_blocks = 0;
            __threadfence();
            if (use_cond) cudaGraphSetConditional(cond, act > 0 ? 1u : 0u);
        }
    }
}

// Column partials per chunk; the last chunk of each tensor to finish (an
// atomic count per tensor, no waiting) adds them in chunk order into lambda.
template <typename T>
__global__ void __launch_bounds__(256) batch_colsum_kernel(const BatchTensor *__restrict__ desc,
                                                           const int2 *__restrict__ chunks,
                                                           const int32_t *__restrict__ flags,
                                                           unsigned int *__restrict__ chunk_count) {
    __shared__ double sm[256];
    __shared__ bool last;
    const int2 w = chunks[blockIdx.x];
    const BatchTensor &d = desc[w.x];
    if (flags[2 * w.x]) return;
    const int Rp = d.rp;
    const int c = threadIdx.x % Rp, rl = threadIdx.x / Rp, nrl = blockDim.x / Rp;
    const int64_t r0 = (int64_t)w.y * kChunkRows;
    const int64_t r1 = min(r0 + kChunkRows, d.rows);
    const T *B = reinterpret_cast<const T *>(d.a.B);
    double s = 0.0;
    if (rl < nrl)
        for (int64_t i = r0 + rl; i < r1; i += nrl) s += d.Bm ? d.Bm[i * Rp + c] : (double)B[i * Rp + c];
    sm[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < Rp) {
        double t = 0.0;
        for (int k = 0; k < nrl; ++k) t += sm[k * Rp + threadIdx.x];
        d.colpart[(int64_t)w.y * Rp + threadIdx.x] = t;
    }
    __threadfence();  // every writer's partial is visible device-wide before the count
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&chunk_count[w.x], 1u) == (unsigned)d.nchunks - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int c2 = threadIdx.x; c2 < Rp; c2 += blockDim.x) {
        double t = 0.0;
        for (int p = 0; p < d.nchunks; ++p) t += __ldcg(d.colpart + (int64_t)p * Rp + c2);
        d.lambda[c2] = t;
    }
    if (threadIdx.x == 0) chunk_count[w.x] = 0;
}

template <typename T>
__global__ void __launch_bounds__(256) batch_scale_kernel(const BatchTensor *__restrict__ desc,
                                                          const int2 *__restrict__ chunks,
                                                          const int32_t *__restrict__ flags) {
    __shared__ double lam[256], inv[256];
    const int2 w = chunks[blockIdx.x];
    const BatchTensor &d = desc[w.x];
    if (flags[2 * w.x]) return;
    const int Rp = d.rp;
    // one reciprocal per column (no overflow: lambda >= 2^-1000, else a plain
    // division); lambda = 0 marks an all-zero column, whose A stays
    for (int c = threadIdx.x; c < Rp; c += blockDim.x) {
        const double l = d.lambda[c];
        lam[c] = l;
        inv[c] = l >= 0x1p-1000 ? 1.0 / l : 0.0;
    }
    __syncthreads();
    const int64_t r0 = (int64_t)w.y * kChunkRows;
    const int64_t r1 = min(r0 + kChunkRows, d.rows);
    const T *B = reinterpret_cast<const T *>(d.a.B);
    T *A = reinterpret_cast<T *>(d.A);
    for (int64_t e = r0 * Rp + threadIdx.x; e < r1 * Rp; e += blockDim.x) {
        const int c = (int)(e & (Rp - 1));  // Rp is a power of two
        const double l = lam[c];
        if (l > 0.0) {
            const double b = d.Bm ? d.Bm[e] : (double)B[e];
            const double v = inv[c] != 0.0 ? b * inv[c] : b / l;
            if (d.Am) d.Am[e] = v;
            A[e] = (T)v;
        }
    }
}

// B_t = A_t^(0) Lambda_t for every tensor (the log-likelihood's scaled rows;
// the same arithmetic as the single-tensor scale_b_kernel)
template <typename T>
__global__ void __launch_bounds__(256) batch_scale_b_kernel(const BatchTensor *__restrict__ desc,
                                                            const int2 *__restrict__ chunks) {
    const int2 w = chunks[blockIdx.x];
    const BatchTensor &d = desc[w.x];
    const int Rp = d.rp;
    const int64_t r0 = (int64_t)w.y * kChunkRows;
    const int64_t r1 = min(r0 + kChunkRows, d.rows);
    const T *A = reinterpret_cast<const T *>(d.A);
    T *B = reinterpret_cast<T *>(const_cast<void *>(d.a.B));
    for (int64_t e = r0 * Rp + threadIdx.x; e < r1 * Rp; e += blockDim.x) {
        const double b = (d.Am ? d.Am[e] : (double)A[e]) * d.lambda[e & (Rp - 1)];
        if (d.Bm) d.Bm[e] = b;
        B[e] = (T)b;
    }
}

// Every tensor's log-likelihood total: item (t, b) is block b of tensor t's
// total (the single-tensor launch's blocks, so the sums are the same).
template <typename T>
__global__ void __launch_bounds__(256) batch_ll_total_kernel(const LLTotalArgs *__restrict__ args,
                                                             const int2 *__restrict__ items) {
    const int2 w = items[blockIdx.x];
    ll_total_body<T>(args[w.x], w.y);
}

__global__ void gather_states_kernel(InnerState *const *src, int n, InnerState *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = *src[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct ModePlan {
    BatchTensor *desc = nullptr;
    int2 *tiles = nullptr, *chunks = nullptr, *echunks = nullptr;
    int ntiles = 0, nchunks = 0, nechunks = 0;
    cudaGraphExec_t exec = nullptr;
    int body_kernels = 0;
    size_t smem = 0;  // dynamic shared memory of the Phi launch (largest tile of the batch)
    int2 *pitems = nullptr;  // (tensor, chunk) items of the batched Khatri-Rao row build
    int npitems = 0;
};

struct Plan {
    std::vector<ModePlan> modes;
    BatchCtl *ctl = nullptr;
    unsigned int *chunk_count = nullptr;  // per tensor: chunks of the update done (zero between launches)
    unsigned int *col_count = nullptr;    // per tensor: chunks of the column sums done (zero between launches)
    double *colpart = nullptr;
    int32_t *flags = nullptr;
    InnerState **state_ptrs = nullptr;
    InnerState *states = nullptr;
    double *ll = nullptr;  // [count] final log-likelihoods
    // the final log-likelihood: mode-0 descriptors without inner-loop state or
    // materialised rows, each tensor's total arguments, and (tensor, block) items
    BatchTensor *lldesc = nullptr;
    LLTotalArgs *llargs = nullptr;
    int2 *llitems = nullptr;
    int nllitems = 0;
    std::vector<void *> owned;
    // what the plan was built for (it is reused while these match)
    std::vector<cpapr_ctx *> key;
    double tol = 0.0;
    int max_inner = 0, graph = 0, esize = 0, grid = 0;
};

// The last plan is kept: building it (work lists, descriptors, three graph
// instantiations) costs milliseconds, a step of a small batch about as much.
std::mutex g_cache_mu;
Plan *g_cache = nullptr;

template <typename T>
cudaError_t launch_phi_batch(const ModePlan &mp, int nm1, int grid, BatchCtl *ctl, cudaStream_t s) {
    const size_t smem = mp.smem;
    auto go = [&](auto kern) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, batch_threads<T>(), smem, s>>>(mp.desc, mp.tiles, mp.ntiles, ctl);
        return cudaGetLastError();
    };
    switch (nm1) {
        case 2: return go(batch_phi_kernel<T, 2>);
        case 3: return go(batch_phi_kernel<T, 3>);
        case 4: return go(batch_phi_kernel<T, 4>);
        default: return go(batch_phi_kernel<T, 0>);
    }
}

template <typename T>
cudaError_t launch_ll_batch(const Plan &P, int nm1, int grid, cudaStream_t s) {
    const ModePlan &m0 = P.modes[0];
    auto go = [&](auto kern) {
        if (m0.smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m0.smem);
        kern<<<grid, batch_threads<T>(), m0.smem, s>>>(P.lldesc, m0.tiles, m0.ntiles, P.ctl);
        return cudaGetLastError();
    };
    switch (nm1) {
        case 2: return go(batch_phi_kernel<T, 2, OP_LL>);
        case 3: return go(batch_phi_kernel<T, 3, OP_LL>);
        case 4: return go(batch_phi_kernel<T, 4, OP_LL>);
        default: return go(batch_phi_kernel<T, 0, OP_LL>);
    }
}

template <typename T>
cudaError_t launch_pi_batch(const ModePlan &mp, int nm1, const int32_t *flags, cudaStream_t s) {
    switch (nm1) {
        case 2: batch_pi_build_kernel<T, 2><<<mp.npitems, 256, 0, s>>>(mp.desc, mp.pitems, flags); break;
        case 3: batch_pi_build_kernel<T, 3><<<mp.npitems, 256, 0, s>>>(mp.desc, mp.pitems, flags); break;
        case 4: batch_pi_build_kernel<T, 4><<<mp.npitems, 256, 0, s>>>(mp.desc, mp.pitems, flags); break;
        default: batch_pi_build_kernel<T, 0><<<mp.npitems, 256, 0, s>>>(mp.desc, mp.pitems, flags); break;
    }
    return cudaGetLastError();
}

template <typename T>
int persistent_grid(int nm1, size_t smem) {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *k = nm1 == 2 ? (const void *)batch_phi_kernel<T, 2>
                             : nm1 == 3 ? (const void *)batch_phi_kernel<T, 3>
                                        : nm1 == 4 ? (const void *)batch_phi_kernel<T, 4> : (const void *)batch_phi_kernel<T, 0>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, batch_threads<T>(), smem) != cudaSuccess || per < 1)
        per = 1;
    cudaGetLastError();
    return sms * per;
}

template <typename T>
cpapr_status enqueue_inner_body(cpapr_ctx *c0, Plan &P, int n, double tol, int max_inner, cudaGraphConditionalHandle h,
                                int use_cond, int grid) {
    ModePlan &mp = P.modes[n];
    cudaStream_t s = c0->stream;
    if (mp.ntiles > 0) CPAPR_CUDA(c0, launch_phi_batch<T>(mp, c0->N - 1, grid, P.ctl, s));
    batch_update_kernel<T><<<mp.nchunks, 256, 0, s>>>(mp.desc, mp.chunks, P.chunk_count, P.ctl, tol, max_inner, h,
                                                      use_cond);
    CPAPR_CUDA(c0, cudaGetLastError());
    return CPAPR_OK;
}

template <typename T>
cpapr_status build_graph(cpapr_ctx *c0, Plan &P, int n, double tol, int max_inner, int grid) {
    ModePlan &mp = P.modes[n];
    cudaGraph_t g = nullptr;
    CPAPR_CUDA(c0, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c0, e, "cudaGraphConditionalHandleCreate");
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(c0->stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c0, e, "batch graph");
    }
    cpapr_status st = enqueue_inner_body<T>(c0, P, n, tol, max_inner, h, 1, grid);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(c0->stream, &captured);
    if (st != CPAPR_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        return st != CPAPR_OK ? st : cuda_fail(c0, e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&mp.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c0, e, "cudaGraphInstantiate(batch)");
    mp.body_kernels = 2;
    return CPAPR_OK;
}

void free_plan(Plan &P) {
    for (auto &mp : P.modes)
        if (mp.exec) cudaGraphExecDestroy(mp.exec);
    for (void *p : P.owned) cudaFree(p);
    P.owned.clear();
}

void drop_cache_locked() {
    if (g_cache) {
        free_plan(*g_cache);
        delete g_cache;
        g_cache = nullptr;
    }
}

template <typename T>
cpapr_status batch_solve_t(cpapr_ctx *const *ctxs, int count, double tol, int max_outer, int max_inner,
                           cpapr_result *results) {
    cpapr_ctx *c0 = ctxs[0];
    const int N = c0->N;
    cudaStream_t s = c0->stream;
    for (int i = 0; i < count; ++i) {
        CPAPR_CUDA(ctxs[i], cudaStreamSynchronize(ctxs[i]->stream));
        ctxs[i]->pi_mode_built = -1;  // the batched solve changes every factor
    }
    // every tensor needs a rank class of the batched kernel and the segmented
    // reduction; it keeps its own tile size (tuned or heuristic) as long as
    // the stage leaves the batched kernel its resident blocks per SM (the
    // whole launch runs at the largest tile's shared memory), else the tile
    // is halved until it does
    int maxrpl = 0;
    for (int k = 0; k < Classes<T>::n; ++k) maxrpl = std::max(maxrpl, Classes<T>::rpl[k]);
    const size_t budget = (size_t)227 * 1024 / batch_min_blocks<T>() - 1024;
    for (int i = 0; i < count; ++i) {
        const int k = class_for<T>(ctxs[i]->Rp);
        if (k < 0) return fail(ctxs[i], CPAPR_E_ARG, "rank not supported by the batched solver");
        const int lanes = Classes<T>::g[k];
        for (int n = 0; n < N; ++n) {
            ModeLayout &L = ctxs[i]->mode[n];
            int tile = L.tile_nnz;
            while (tile > 256 && phi_smem_bytes(tile, N - 1, (int)sizeof(T), batch_threads<T>(), maxrpl) > budget)
                tile /= 2;
            if (L.lanes != lanes || L.reduction != CPAPR_REDUCE_SEGMENTED || tile != L.tile_nnz)
                CPAPR_TRY(configure_mode(ctxs[i], n, lanes, tile, CPAPR_REDUCE_SEGMENTED));
        }
        CPAPR_CUDA(ctxs[i], cudaStreamSynchronize(ctxs[i]->stream));
    }
    std::lock_guard<std::mutex> cache_lock(g_cache_mu);
    const int graph_flag = c0->opt.use_graph != 0 ? 1 : 0;
    const std::vector<cpapr_ctx *> key(ctxs, ctxs + count);
    const bool hit = g_cache && g_cache->key == key && g_cache->tol == tol && g_cache->max_inner == max_inner &&
                     g_cache->graph == graph_flag && g_cache->esize == (int)sizeof(T);
    if (!hit) {
        drop_cache_locked();
        g_cache = new Plan();
    }
    Plan &P = *g_cache;
    auto dalloc = [&](void **p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) P.owned.push_back(*p);
        return e;
    };
#define BT_CUDA(call)                               \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess) {                    \
            drop_cache_locked();                    \
            return cuda_fail(c0, _e, #call);        \
        }                                           \
    } while (0)
    if (!hit) {
    P.modes.resize(N);
    P.key = key;
    P.tol = tol;
    P.max_inner = max_inner;
    P.graph = graph_flag;
    P.esize = (int)sizeof(T);
    // per-tensor column partial areas (sized for the longest mode)
    std::vector<int64_t> colpart_off(count);
    int64_t colpart_total = 0;
    for (int i = 0; i < count; ++i) {
        int64_t mx = 0;
        for (int n = 0; n < N; ++n) mx = std::max<int64_t>(mx, ceil_div(ctxs[i]->dims[n], kChunkRows));
        colpart_off[i] = colpart_total;
        colpart_total += mx * ctxs[i]->Rp;
    }
    BT_CUDA(dalloc((void **)&P.colpart, (size_t)colpart_total * 8));
    BT_CUDA(dalloc((void **)&P.ctl, sizeof(BatchCtl)));
    BT_CUDA(dalloc((void **)&P.chunk_count, (size_t)count * 4));
    BT_CUDA(dalloc((void **)&P.col_count, (size_t)count * 4));
    BT_CUDA(dalloc((void **)&P.flags, (size_t)count * 8));
    BT_CUDA(dalloc((void **)&P.state_ptrs, (size_t)count * N * sizeof(InnerState *)));
    BT_CUDA(dalloc((void **)&P.states, (size_t)count * N * sizeof(InnerState)));
    BT_CUDA(dalloc((void **)&P.ll, (size_t)count * sizeof(double)));
    BT_CUDA(cudaMemsetAsync(P.ctl, 0, sizeof(BatchCtl), s));
    BT_CUDA(cudaMemsetAsync(P.chunk_count, 0, (size_t)count * 4, s));
    BT_CUDA(cudaMemsetAsync(P.col_count, 0, (size_t)count * 4, s));
    {
        std::vector<InnerState *> sp((size_t)count * N);
        for (int i = 0; i < count; ++i)
            for (int n = 0; n < N; ++n) sp[(size_t)i * N + n] = ctxs[i]->inner + n;
        BT_CUDA(cudaMemcpy(P.state_ptrs, sp.data(), sp.size() * sizeof(InnerState *), cudaMemcpyHostToDevice));
    }
    size_t smem_max = 0;
    std::vector<BatchTensor> desc0;
    for (int n = 0; n < N; ++n) {
        ModePlan &mp = P.modes[n];
        std::vector<BatchTensor> desc(count);
        std::vector<int2> tiles, chunks, echunks, pitems;
        for (int i = 0; i < count; ++i) {
            cpapr_ctx *c = ctxs[i];
            const ModeLayout &L = c->mode[n];
            BatchTensor &d = desc[i];
            std::memset(&d, 0, sizeof(d));
            PhiArgs &a = d.a;
            a.nnz = c->nnz;
            a.T = L.tile_nnz;
            a.ntiles = L.ntiles;
            a.Rp = c->Rp;
            a.In = L.In;
            a.nm1 = c->N - 1;
            a.atomic = 0;
            a.rstart = L.rstart;
            a.nzrow = L.nzrow;
            a.krow = L.krow;
            int k = 0;
            for (int m = 0; m < N; ++m) {
                if (m == n) continue;
                a.idx[k] = L.idx[k];
                a.A[k] = c->A[m];
                a.Am[k] = c->A64[m];
                ++k;
            }
            a.Bm = c->B64;
            a.val = L.val;
            a.B = c->B;
            a.out = c->Phi[n];
            a.carry = c->carry;
            a.split = L.split;
            a.tsplit = L.tsplit;
            a.splitcnt = L.splitcnt;
            a.nsplit = L.nsplit;
            a.eps = c->opt.eps;
            a.inner = c->inner + n;
            a.llpart = c->llpart;
            a.err = c->errflag + 3;
            a.stage_extra = injected_stage_shortfall();
            a.dfdot = 0;  // the batched kernel keeps the FP64 dot (measured faster on the 64-tensor batch)
            // FP64 tensors whose mode n materialises its Khatri-Rao rows stream them here too
            if (sizeof(T) == 8 && L.pi && c->pibuf && c->nnz > 0) {
                a.pi = c->pibuf;
                const int64_t vecs = c->nnz * (c->Rp / Vec16<T>::n);
                for (int64_t q = 0; q < ceil_div(vecs, kPiChunk); ++q) pitems.push_back(make_int2(i, (int)q));
            }
            d.cfg = class_for<T>(c->Rp);
            d.rp = c->Rp;
            d.rows = c->dims[n];
            d.A = c->A[n];
            d.Am = c->A64[n];
            d.Bm = c->B64;
            d.lambda = c->lambda;
            d.colpart = P.colpart + colpart_off[i];
            d.nchunks = (int32_t)ceil_div(c->dims[n], kChunkRows);
            d.chunk0 = (int32_t)chunks.size();
            d.kappa = c->opt.kappa;
            d.kappa_tol = c->opt.kappa_tol;
            d.erows = L.erows;
            d.nempty = c->nnz > 0 ? L.nempty : 0;
            for (int t = 0; t < (c->nnz > 0 ? L.ntiles : 0); ++t) tiles.push_back(make_int2(i, t));
            for (int t = 0; t < d.nchunks; ++t) chunks.push_back(make_int2(i, t));
            for (int t = 0; t < (int)ceil_div(d.nempty * c->Rp, kEmptyChunk); ++t) echunks.push_back(make_int2(i, t));
        }
        // larger tensors' tiles first: the persistent blocks finish together
        std::stable_sort(tiles.begin(), tiles.end(), [&](const int2 &x, const int2 &y) {
            return ctxs[x.x]->nnz > ctxs[y.x]->nnz;
        });
        mp.ntiles = (int)tiles.size();
        {
            int maxtile = 4;
            for (int i = 0; i < count; ++i) maxtile = std::max(maxtile, ctxs[i]->mode[n].tile_nnz);
            mp.smem = phi_smem_bytes(maxtile, N - 1, (int)sizeof(T), batch_threads<T>(), maxrpl);
            smem_max = std::max(smem_max, mp.smem);
        }
        mp.nchunks = (int)chunks.size();
        mp.nechunks = (int)echunks.size();
        BT_CUDA(dalloc((void **)&mp.desc, desc.size() * sizeof(BatchTensor)));
        BT_CUDA(dalloc((void **)&mp.tiles, tiles.size() * sizeof(int2)));
        BT_CUDA(dalloc((void **)&mp.chunks, chunks.size() * sizeof(int2)));
        BT_CUDA(dalloc((void **)&mp.echunks, echunks.size() * sizeof(int2)));
        if (!echunks.empty())
            BT_CUDA(cudaMemcpy(mp.echunks, echunks.data(), echunks.size() * sizeof(int2), cudaMemcpyHostToDevice));
        mp.npitems = (int)pitems.size();
        BT_CUDA(dalloc((void **)&mp.pitems, pitems.size() * sizeof(int2)));
        if (!pitems.empty())
            BT_CUDA(cudaMemcpy(mp.pitems, pitems.data(), pitems.size() * sizeof(int2), cudaMemcpyHostToDevice));
        BT_CUDA(cudaMemcpy(mp.desc, desc.data(), desc.size() * sizeof(BatchTensor), cudaMemcpyHostToDevice));
        if (!tiles.empty())
            BT_CUDA(cudaMemcpy(mp.tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice));
        BT_CUDA(cudaMemcpy(mp.chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice));
        if (n == 0) desc0 = desc;
    }
    {
        std::vector<LLTotalArgs> args(count);
        std::vector<int2> items;
        for (int i = 0; i < count; ++i) {
            desc0[i].a.inner = nullptr;
            desc0[i].a.pi = nullptr;
            const int nll = ctxs[i]->nnz > 0 ? ctxs[i]->mode[0].ntiles : 0;
            args[i] = ll_total_args(ctxs[i], ctxs[i]->llpart, nll, P.ll + i);
            for (int b = 0; b < args[i].part0[N]; ++b) items.push_back(make_int2(i, b));
        }
        P.nllitems = (int)items.size();
        BT_CUDA(dalloc((void **)&P.lldesc, (size_t)count * sizeof(BatchTensor)));
        BT_CUDA(dalloc((void **)&P.llargs, (size_t)count * sizeof(LLTotalArgs)));
        BT_CUDA(dalloc((void **)&P.llitems, items.size() * sizeof(int2)));
        BT_CUDA(cudaMemcpy(P.lldesc, desc0.data(), (size_t)count * sizeof(BatchTensor), cudaMemcpyHostToDevice));
        BT_CUDA(cudaMemcpy(P.llargs, args.data(), (size_t)count * sizeof(LLTotalArgs), cudaMemcpyHostToDevice));
        BT_CUDA(cudaMemcpy(P.llitems, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
    }
    if (smem_max > kMaxPhiSmem) {
        drop_cache_locked();
        return fail(c0, CPAPR_E_ARG, "batch: tile_nnz too large for the shared-memory stage");
    }
    for (int n = 0; n < N; ++n) P.modes[n].smem = smem_max;  // one occupancy for the whole plan
    P.grid = persistent_grid<T>(N - 1, smem_max);
    if (graph_flag)
        for (int n = 0; n < N; ++n) {
            cpapr_status st = build_graph<T>(c0, P, n, tol, max_inner, P.grid);
            if (st != CPAPR_OK) {
                drop_cache_locked();
                return st;
            }
        }
    }  // plan built
    const int grid = P.grid;
    const bool graph = graph_flag != 0;

    struct Track {
        int outer = 0, total = 0;
        bool conv = false, active = true;
        double kkt = 0.0;
    };
    std::vector<Track> tr(count);
    std::vector<int32_t> flags((size_t)count * 2);
    std::vector<InnerState> hs((size_t)count * N);
    cpapr_status st = CPAPR_OK;
    for (int k = 0; k < max_outer && st == CPAPR_OK; ++k) {
        bool any = false;
        for (int i = 0; i < count; ++i) {
            flags[2 * i] = tr[i].active ? 0 : 1;
            flags[2 * i + 1] = ctxs[i]->k_total > 0 ? 1 : 0;
            any = any || tr[i].active;
        }
        if (!any) break;
        BT_CUDA(cudaMemcpyAsync(P.flags, flags.data(), flags.size() * 4, cudaMemcpyHostToDevice, s));
        for (int n = 0; n < N; ++n) {
            ModePlan &mp = P.modes[n];
            batch_sb_kernel<T><<<mp.nchunks, 256, 0, s>>>(mp.desc, mp.chunks, P.flags);
            BT_CUDA(cudaGetLastError());
            if (mp.nechunks > 0) {
                batch_empty_kkt_kernel<T><<<mp.nechunks, 256, 0, s>>>(mp.desc, mp.echunks, P.flags);
                BT_CUDA(cudaGetLastError());
            }
            if (mp.npitems > 0) {
                BT_CUDA(launch_pi_batch<T>(mp, N - 1, P.flags, s));
                c0->launches += 1;
            }
            if (graph) {
                BT_CUDA(cudaGraphLaunch(mp.exec, s));
            } else {
                for (int l = 0; l < max_inner && st == CPAPR_OK; ++l)
                    st = enqueue_inner_body<T>(c0, P, n, tol, max_inner, 0ull, 0, grid);
                if (st != CPAPR_OK) break;
            }
            batch_colsum_kernel<T><<<mp.nchunks, 256, 0, s>>>(mp.desc, mp.chunks, P.flags, P.col_count);
            batch_scale_kernel<T><<<mp.nchunks, 256, 0, s>>>(mp.desc, mp.chunks, P.flags);
            BT_CUDA(cudaGetLastError());
        }
        if (st != CPAPR_OK) break;
        gather_states_kernel<<<(unsigned)ceil_div((int64_t)count * N, 256), 256, 0, s>>>(P.state_ptrs, count * N,
                                                                                      P.states);
        BT_CUDA(cudaGetLastError());
        BT_CUDA(cudaMemcpyAsync(hs.data(), P.states, hs.size() * sizeof(InnerState), cudaMemcpyDeviceToHost, s));
        BT_CUDA(cudaStreamSynchronize(s));
        c0->launches += 1 + (int64_t)N * 3;
        for (int i = 0; i < count; ++i) {
            if (!tr[i].active) continue;
            cpapr_ctx *c = ctxs[i];
            c->k_total += 1;
            tr[i].outer += 1;
            bool all_first = true;
            double kmax = 0.0;
            for (int n = 0; n < N; ++n) {
                const InnerState &x = hs[(size_t)i * N + n];
                tr[i].total += x.used;
                if (!(x.passed && x.used == 1)) all_first = false;
                kmax = std::max(kmax, x.viol);
            }
            tr[i].kkt = kmax;
            if (all_first) {
                tr[i].conv = true;
                tr[i].active = false;
            }
        }
        int used_max = 0;
        for (int n = 0; n < N; ++n) {
            int um = 0;
            for (int i = 0; i < count; ++i) um = std::max(um, hs[(size_t)i * N + n].used);
            used_max += um * P.modes[n].body_kernels;
        }
        c0->launches += used_max;
    }
#undef BT_CUDA
    if (st != CPAPR_OK) {
        drop_cache_locked();
        return st;
    }
    // final log-likelihoods, three launches for the whole batch: B = A^(0)
    // Lambda, the tile sums of x log m along mode 0 (rows formed in place),
    // and every tensor's total; one copy back
    std::vector<double> ll(count, 0.0);
    {
        const ModePlan &m0 = P.modes[0];
        batch_scale_b_kernel<T><<<m0.nchunks, 256, 0, s>>>(m0.desc, m0.chunks);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && m0.ntiles > 0) e = launch_ll_batch<T>(P, N - 1, grid, s);
        if (e == cudaSuccess) {
            // the column sums of the totals run on the FP64 factors (masters in the FP32 form)
            batch_ll_total_kernel<double><<<P.nllitems, 256, 0, s>>>(P.llargs, P.llitems);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ll.data(), P.ll, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c0, e, "batch log-likelihood");
        c0->launches += 3;
    }
    for (int i = 0; i < count; ++i) {
        results[i].outer_iters = tr[i].outer;
        results[i].total_inner = tr[i].total;
        results[i].converged = tr[i].conv ? 1 : 0;
        results[i].reserved = 0;
        results[i].loglik = ll[i];
        results[i].kkt_viol = tr[i].kkt;
    }
    return CPAPR_OK;
}

}  // namespace

// Drops the cached batch plan if it refers to ctx (called when a context is
// destroyed or its tiling changes).
void batch_forget(cpapr_ctx *ctx) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    if (!g_cache) return;
    for (cpapr_ctx *c : g_cache->key)
        if (c == ctx) {
            drop_cache_locked();
            return;
        }
}

// Batched solve through the persistent kernels; contexts must share the
// device, the precision and the number of modes.
cpapr_status batch_mu_solve_persistent(cpapr_ctx *const *ctxs, int count, double tol, int max_outer, int max_inner,
                                       cpapr_result *results) {
    if (count == 0) return CPAPR_OK;
    for (int i = 1; i < count; ++i)
        if (ctxs[i]->N != ctxs[0]->N || ctxs[i]->device != ctxs[0]->device)
            return fail(ctxs[i], CPAPR_E_ARG, "batched solve needs one device and one number of modes");
    if (ctxs[0]->esize == 8) return batch_solve_t<double>(ctxs, count, tol, max_outer, max_inner, results);
    return batch_solve_t<float>(ctxs, count, tol, max_outer, max_inner, results);
}

}  // namespace cpapr
