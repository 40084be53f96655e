// Kernels of the multiplicative-update loop around Phi (Algorithm 1 of
// arXiv 2307.03276):
//   B <- (A^(n) + S) Lambda            sb_kernel
//   B <- B * Phi unless KKT passed     update_kernel (also the loop bookkeeping)
//   lambda <- e^T B; A <- B Lambda^-1  colsum_partial_kernel + normalise_kernel
//   log-likelihood total               ll_total_kernel (column sums, tile
//                                      partials and the model total at once)
// and the model I/O helpers.  All reductions that decide or normalise run in
// FP64 whatever the working precision.  In the FP32 form the factors and B
// have FP64 masters (A64, B64): S, the update and the normalisation compute
// on the masters in FP64 and write FP32 copies for the Phi kernels.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.cuh"
#include "ll_total.cuh"

namespace cpapr {

static unsigned grid_for(int64_t n, int threads = 256, int64_t cap = 152 * 8) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), cap));
}


// ---------------------------------------------------------------------------
// B <- (A + S) Lambda.  S(i,r) = kappa when this is not the first outer
// iteration, A(i,r) < kappa_tol and the previous Phi(i,r) > 1 (Chi and
// Kolda's shift away from inadmissible zeros).  Also resets the mode's
// inner-loop state.
// ---------------------------------------------------------------------------
// A: the FP64 factor (the master in the FP32 form); Bm: FP64 master of B
// (FP32 form) or null.
template <typename T>
__global__ void sb_kernel(const double *__restrict__ A, const T *__restrict__ phi_prev,
                          const double *__restrict__ lambda, double *__restrict__ Bm, T *__restrict__ B, int64_t rows,
                          int Rp, int shift, double kappa, double kappa_tol, InnerState *inner) {
    if (inner && blockIdx.x == 0 && threadIdx.x == 0) {
        inner->l = 0;
        inner->done = 0;
        inner->used = 0;
        inner->passed = 0;
        inner->counter = 0;
        inner->kkt[0] = 0ull;
        inner->kkt[1] = 0ull;
        inner->viol = 0.0;
    }
    const int64_t n = rows * Rp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e & (Rp - 1));  // Rp is a power of two
        const double a = A[e];
        const double s = (shift && a < kappa_tol && (double)phi_prev[e] > 1.0) ? kappa : 0.0;
        const double b = (a + s) * lambda[c];
        if (Bm) Bm[e] = b;
        B[e] = (T)b;
    }
}

cpapr_status launch_sb(cpapr_ctx *ctx, int n, bool shift, InnerState *inner) {
    const int64_t rows = ctx->dims[n];
    ProfScope ps(ctx, K_SB);
    count_launch(ctx);
    if (ctx->esize == 8)
        sb_kernel<double><<<grid_for(rows * ctx->Rp), 256, 0, ctx->stream>>>(
            factor64(ctx, n), (const double *)ctx->Phi[n], ctx->lambda, nullptr, (double *)ctx->B, rows, ctx->Rp,
            shift ? 1 : 0, ctx->opt.kappa, ctx->opt.kappa_tol, inner);
    else
        sb_kernel<float><<<grid_for(rows * ctx->Rp), 256, 0, ctx->stream>>>(
            factor64(ctx, n), (const float *)ctx->Phi[n], ctx->lambda, ctx->B64, (float *)ctx->B, rows, ctx->Rp,
            shift ? 1 : 0, ctx->opt.kappa, ctx->opt.kappa_tol, inner);
    CPAPR_CUDA(ctx, cudaGetLastError());
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// B <- B * Phi when the KKT check of this inner iteration failed.  Every
// block reads the same published violation; the last block to finish does
// the bookkeeping (iteration counter, done flag, next violation slot, and
// the graph's loop condition).
// ---------------------------------------------------------------------------
// B: the working-precision B; Bm: its FP64 master (FP32 form) or null.
template <typename T>
__global__ void update_kernel(T *__restrict__ B, double *__restrict__ Bm, const T *__restrict__ P, int64_t n,
                              InnerState *inner, double tol, int max_inner, cudaGraphConditionalHandle cond,
                              int use_cond) {
    __shared__ int s_l, s_done;
    __shared__ double s_viol;
    if (threadIdx.x == 0) {
        s_l = *((volatile int32_t *)&inner->l);
        s_done = *((volatile int32_t *)&inner->done);
        s_viol = __longlong_as_double((long long)inner->kkt[s_l & 1]);
    }
    __syncthreads();
    const int l = s_l, done = s_done;
    const double viol = s_viol;
    if (!done && !(viol < tol)) {
        if constexpr (sizeof(T) == 4) {
            // FP32 form: on the FP64 master, in pairs (n is even: rows of Rp >= 4 values)
            for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n / 2;
                 e += (int64_t)gridDim.x * blockDim.x)
                master_mul(reinterpret_cast<double2 *>(Bm), reinterpret_cast<float2 *>(B),
                           reinterpret_cast<const float2 *>(P), e);
        } else {
            // 16-byte vectors: n is a whole number of them (rows of Rp values)
            using V = typename Vec16<T>::type;
            V *Bv = reinterpret_cast<V *>(B);
            const V *Pv = reinterpret_cast<const V *>(P);
            const int64_t nv = n / Vec16<T>::n;
            for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nv;
                 e += (int64_t)gridDim.x * blockDim.x)
                Bv[e] = vmul(Bv[e], Pv[e]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&inner->counter, 1u);
        if (prev == gridDim.x - 1) {
            inner->counter = 0;
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
            __threadfence();
            if (use_cond) cudaGraphSetConditional(cond, (!now_done && l + 1 < max_inner) ? 1u : 0u);
        }
    }
}

cpapr_status launch_update(cpapr_ctx *ctx, int n, double tol, int max_inner, InnerState *inner,
                           unsigned long long cond_handle, int use_cond) {
    const int64_t nel = ctx->dims[n] * ctx->Rp;
    ProfScope ps(ctx, K_UPDATE);
    count_launch(ctx);
    const unsigned g = grid_for(nel, 256, 152 * 4);
    if (ctx->esize == 8)
        update_kernel<double><<<g, 256, 0, ctx->stream>>>((double *)ctx->B, nullptr, (const double *)ctx->Phi[n], nel,
                                                           inner, tol, max_inner,
                                                           (cudaGraphConditionalHandle)cond_handle, use_cond);
    else
        update_kernel<float><<<g, 256, 0, ctx->stream>>>((float *)ctx->B, ctx->B64, (const float *)ctx->Phi[n], nel,
                                                          inner, tol, max_inner,
                                                          (cudaGraphConditionalHandle)cond_handle, use_cond);
    CPAPR_CUDA(ctx, cudaGetLastError());
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// column sums (FP64), in a fixed order: block p sums rows p, p+P, ... per
// column; the partials are then added in block order.
// ---------------------------------------------------------------------------
// With `counter` set, the block that finishes last (an atomic count, no
// waiting) adds the partials in block order into colsum[0..Rp) and resets
// the counter.
template <typename T>
__global__ void colsum_partial_kernel(const T *__restrict__ M, int64_t rows, int Rp, double *__restrict__ part,
                                      unsigned int *counter = nullptr, double *__restrict__ colsum = nullptr) {
    __shared__ double sm[256];
    __shared__ bool last;
    const int c = threadIdx.x % Rp;
    const int rl = threadIdx.x / Rp;
    const int nrl = blockDim.x / Rp;
    double s = 0.0;
    if (rl < nrl)
        for (int64_t i = (int64_t)blockIdx.x * nrl + rl; i < rows; i += (int64_t)gridDim.x * nrl)
            s += (double)M[i * Rp + c];
    sm[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < Rp) {
        double t = 0.0;
        for (int k = 0; k < nrl; ++k) t += sm[k * Rp + threadIdx.x];
        part[(int64_t)blockIdx.x * Rp + threadIdx.x] = t;
    }
    if (!counter) return;
    __threadfence();  // every writer's partial is visible device-wide before the count
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int r = threadIdx.x; r < Rp; r += blockDim.x) {
        double t = 0.0;
        for (unsigned p = 0; p < gridDim.x; ++p) t += __ldcg(part + (int64_t)p * Rp + r);
        colsum[r] = t;
    }
    if (threadIdx.x == 0) *counter = 0;
}

static int colsum_parts(int64_t rows, int Rp) {
    const int nrl = std::max(1, 256 / Rp);
    return (int)std::max<int64_t>(1, std::min<int64_t>(kColParts, ceil_div(rows, nrl * 4)));
}

// A(i,c) = B(i,c) / lambda_c (lambda = the column sums of B, finished by
// colsum_partial_kernel), or A kept when lambda_c = 0 (an all-zero column).
// B is the FP64 B (the master in the FP32 form); Am is the FP64 master of A
// (FP32 form; A is then its FP32 copy) or null.
template <typename T>
__global__ void normalise_kernel(const double *__restrict__ B, T *__restrict__ A, double *__restrict__ Am,
                                 int64_t rows, int Rp, const double *__restrict__ lambda) {
    // one reciprocal per column (no overflow: lambda >= 2^-1000, else a plain
    // division); lambda = 0 marks an all-zero column, whose A stays
    __shared__ double lam[256], inv[256];
    for (int c = threadIdx.x; c < Rp; c += blockDim.x) {
        const double l = lambda[c];
        lam[c] = l;
        inv[c] = l >= 0x1p-1000 ? 1.0 / l : 0.0;
    }
    __syncthreads();
    const int64_t n = rows * Rp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e & (Rp - 1));  // Rp is a power of two
        const double l = lam[c];
        if (l > 0.0) {
            const double v = inv[c] != 0.0 ? B[e] * inv[c] : B[e] / l;
            if (Am) Am[e] = v;
            A[e] = (T)v;
        }
    }
}

cpapr_status launch_normalise(cpapr_ctx *ctx, int n) {
    const int64_t rows = ctx->dims[n];
    const int Rp = ctx->Rp;
    const int parts = colsum_parts(rows, Rp);
    // A^(n) changes: materialised rows of another mode that contain it go stale
    if (n != ctx->pi_mode_built) ctx->pi_mode_built = -1;
    ProfScope ps(ctx, K_NORM);
    count_launch(ctx, 2);
    // llcount[1]: the column-sum counter (llcount[0] belongs to the log-likelihood total)
    // the column sums and the division run on the FP64 B (the master in the FP32 form)
    const double *B64 = ctx->B64 ? ctx->B64 : (const double *)ctx->B;
    colsum_partial_kernel<double><<<parts, 256, 0, ctx->stream>>>(B64, rows, Rp, ctx->colpart, ctx->llcount + 1,
                                                                  ctx->lambda);
    if (ctx->esize == 8)
        normalise_kernel<double><<<grid_for(rows * Rp), 256, 0, ctx->stream>>>(B64, (double *)ctx->A[n], nullptr,
                                                                               rows, Rp, ctx->lambda);
    else
        normalise_kernel<float><<<grid_for(rows * Rp), 256, 0, ctx->stream>>>(B64, (float *)ctx->A[n], ctx->A64[n],
                                                                              rows, Rp, ctx->lambda);
    CPAPR_CUDA(ctx, cudaGetLastError());
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// B = A^(n) diag(lambda)
// ---------------------------------------------------------------------------
// A: the FP64 factor (the master in the FP32 form); Bm: FP64 master of B or null
template <typename T>
__global__ void scale_b_kernel(const double *__restrict__ A, const double *__restrict__ lambda,
                               double *__restrict__ Bm, T *__restrict__ B, int64_t n, int Rp) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double b = A[e] * lambda[e & (Rp - 1)];  // Rp is a power of two
        if (Bm) Bm[e] = b;
        B[e] = (T)b;
    }
}

cpapr_status launch_scale_b(cpapr_ctx *ctx, int n, void *dstB) {
    count_launch(ctx);
    const int64_t nel = ctx->dims[n] * ctx->Rp;
    // the FP32 form refreshes B's master only when dstB is the context's B
    if (ctx->esize == 8)
        scale_b_kernel<double><<<grid_for(nel), 256, 0, ctx->stream>>>(factor64(ctx, n), ctx->lambda, nullptr,
                                                                       (double *)dstB, nel, ctx->Rp);
    else
        scale_b_kernel<float><<<grid_for(nel), 256, 0, ctx->stream>>>(
            factor64(ctx, n), ctx->lambda, dstB == ctx->B ? ctx->B64 : nullptr, (float *)dstB, nel, ctx->Rp);
    CPAPR_CUDA(ctx, cudaGetLastError());
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// log-likelihood total of one tensor in one launch (ll_total_body)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) ll_total_kernel(const LLTotalArgs a) {
    ll_total_body<T>(a, (int)blockIdx.x);
}

LLTotalArgs ll_total_args(const cpapr_ctx *ctx, const double *llpart, int nll, double *dst) {
    LLTotalArgs a{};
    int blocks = 0;
    for (int m = 0; m < ctx->N; ++m) {
        a.A[m] = factor64(ctx, m);  // the column sums run on the FP64 factors
        a.rows[m] = ctx->dims[m];
        a.part0[m] = blocks;
        blocks += colsum_parts(ctx->dims[m], ctx->Rp);
    }
    a.part0[ctx->N] = blocks;
    a.N = ctx->N;
    a.Rp = ctx->Rp;
    a.lambda = ctx->lambda;
    a.part = ctx->colpart;
    a.counter = ctx->llcount;
    a.llpart = llpart;
    a.nll = nll;
    a.dst = dst;
    return a;
}

cpapr_status launch_ll_total(cpapr_ctx *ctx, const double *llpart, int nll, double *dst) {
    const LLTotalArgs a = ll_total_args(ctx, llpart, nll, dst);
    const int blocks = a.part0[ctx->N];
    ll_total_kernel<double><<<blocks, 256, 0, ctx->stream>>>(a);
    count_launch(ctx);
    CPAPR_CUDA(ctx, cudaGetLastError());
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// random initial model (SplitMix64, counter-based; Steele, Lea, Flood 2014)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void rand_fill_kernel(double *__restrict__ dst, int64_t rows, int R, int Rp, uint64_t base) {
    const int64_t n = rows * Rp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / Rp;
        const int c = (int)(e % Rp);
        double v = 0.0;
        if (c < R) {
            const uint64_t k = (uint64_t)(i * R + c);
            v = (double)(sm64_mix(base + (k + 1) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
        }
        dst[e] = v;
    }
}

// A = stage / colsum (columns with a zero sum stay as they are); lambda *= colsum.
// Am: FP64 master of A (FP32 form) or null.
template <typename T>
__global__ void init_scale_kernel(const double *__restrict__ stage, T *__restrict__ A, double *__restrict__ Am,
                                  int64_t rows, int Rp, const double *__restrict__ part, int nparts,
                                  double *__restrict__ lambda) {
    __shared__ double cs[256];
    for (int c = threadIdx.x; c < Rp; c += blockDim.x) {
        double s = 0.0;
        for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * Rp + c];
        cs[c] = s;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < Rp; c += blockDim.x) lambda[c] = lambda[c] * cs[c];
    const int64_t n = rows * Rp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double s = cs[e % Rp];
        const double v = s > 0.0 ? stage[e] / s : stage[e];
        if (Am) Am[e] = v;
        A[e] = (T)v;
    }
}

__global__ void fill_lambda_kernel(double *__restrict__ lambda, int R, int Rp) {
    for (int c = threadIdx.x; c < Rp; c += blockDim.x) lambda[c] = c < R ? 1.0 : 0.0;
}

cpapr_status launch_init_random(cpapr_ctx *ctx, uint64_t seed) {
    const int Rp = ctx->Rp;
    fill_lambda_kernel<<<1, 256, 0, ctx->stream>>>(ctx->lambda, ctx->R, Rp);
    count_launch(ctx, 1 + 3 * ctx->N);
    CPAPR_CUDA(ctx, cudaGetLastError());
    for (int m = 0; m < ctx->N; ++m) {
        const int64_t rows = ctx->dims[m];
        const uint64_t base = sm64_mix(seed + (uint64_t)(200 + m + 1) * 0x9E3779B97F4A7C15ull);
        rand_fill_kernel<<<grid_for(rows * Rp), 256, 0, ctx->stream>>>(ctx->stage, rows, ctx->R, Rp, base);
        const int parts = colsum_parts(rows, Rp);
        colsum_partial_kernel<double><<<parts, 256, 0, ctx->stream>>>(ctx->stage, rows, Rp, ctx->colpart);
        if (ctx->esize == 8)
            init_scale_kernel<double><<<grid_for(rows * Rp), 256, 0, ctx->stream>>>(
                ctx->stage, (double *)ctx->A[m], nullptr, rows, Rp, ctx->colpart, parts, ctx->lambda);
        else
            init_scale_kernel<float><<<grid_for(rows * Rp), 256, 0, ctx->stream>>>(
                ctx->stage, (float *)ctx->A[m], ctx->A64[m], rows, Rp, ctx->colpart, parts, ctx->lambda);
        CPAPR_CUDA(ctx, cudaGetLastError());
    }
    return CPAPR_OK;
}

// ---------------------------------------------------------------------------
// model I/O: caller matrices are rows x R doubles (host or device); the
// device keeps rows x Rp of the working type with zero padding columns.
// ---------------------------------------------------------------------------
// dst64: an FP64 copy to write as well (a factor's master in the FP32 form) or null
template <typename T>
__global__ void convert_kernel(const double *__restrict__ src, T *__restrict__ dst, int64_t n,
                               int32_t *__restrict__ errflag, double *__restrict__ dst64) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[e];
        if (!(v >= 0.0) || isinf(v)) atomicOr(errflag + 2, 1);
        if (dst64) dst64[e] = v;
        dst[e] = (T)v;
    }
}

template <typename T>
__global__ void widen_kernel(const T *__restrict__ src, double *__restrict__ dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (double)src[e];
}

static cpapr_status upload_matrix2(cpapr_ctx *ctx, const double *src, int64_t rows, void *dst, double *dst64) {
    const int R = ctx->R, Rp = ctx->Rp;
    const int64_t n = rows * Rp;
    CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->stage, 0, (size_t)n * 8, ctx->stream));
    if (rows > 0)
        CPAPR_CUDA(ctx, cudaMemcpy2DAsync(ctx->stage, (size_t)Rp * 8, src, (size_t)R * 8, (size_t)R * 8, (size_t)rows,
                                          cudaMemcpyDefault, ctx->stream));
    count_launch(ctx);
    if (ctx->esize == 8)
        convert_kernel<double><<<grid_for(n), 256, 0, ctx->stream>>>(ctx->stage, (double *)dst, n, ctx->errflag,
                                                                     nullptr);
    else
        convert_kernel<float><<<grid_for(n), 256, 0, ctx->stream>>>(ctx->stage, (float *)dst, n, ctx->errflag,
                                                                    dst64);
    CPAPR_CUDA(ctx, cudaGetLastError());
    return CPAPR_OK;
}

cpapr_status upload_matrix(cpapr_ctx *ctx, const double *src, int64_t rows, void *dst) {
    return upload_matrix2(ctx, src, rows, dst, nullptr);
}

cpapr_status upload_factor(cpapr_ctx *ctx, int m, const double *src) {
    return upload_matrix2(ctx, src, ctx->dims[m], ctx->A[m], ctx->A64[m]);
}

cpapr_status download_matrix(cpapr_ctx *ctx, const void *src, int64_t rows, double *dst) {
    const int R = ctx->R, Rp = ctx->Rp;
    const int64_t n = rows * Rp;
    const double *from = (const double *)src;
    if (ctx->esize != 8) {
        widen_kernel<float><<<grid_for(n), 256, 0, ctx->stream>>>((const float *)src, ctx->stage, n);
        count_launch(ctx);
        CPAPR_CUDA(ctx, cudaGetLastError());
        from = ctx->stage;
    }
    if (rows > 0)
        CPAPR_CUDA(ctx, cudaMemcpy2DAsync(dst, (size_t)R * 8, from, (size_t)Rp * 8, (size_t)R * 8, (size_t)rows,
                                          cudaMemcpyDefault, ctx->stream));
    return CPAPR_OK;
}

}  // namespace cpapr
