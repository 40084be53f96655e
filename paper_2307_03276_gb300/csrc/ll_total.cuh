// Log-likelihood total: the sum of the per-tile partials of sum x log m,
// minus the model total sum_r lambda_r prod_m colsum_m(r) (the log-likelihood
// of the Poisson model with the constant sum log x! dropped).  Blocks
// [part0[m], part0[m+1]) take column partial sums of factor m; the last block
// to finish (atomic election, no waiting) adds the partials of every column
// in part order, the tile partials with a fixed tree, and writes the result.
// Shared by the single-tensor launch (mu.cu) and the batched one (batch.cu).
#pragma once

#include "internal.cuh"

namespace cpapr {

struct LLTotalArgs {
    const void *A[kMaxModes];
    int64_t rows[kMaxModes];
    int part0[kMaxModes + 1];  // first block of each mode; part0[N] = number of blocks
    int N, Rp;
    const double *lambda;
    double *part;           // [blocks][Rp]
    unsigned int *counter;  // zero between launches
    const double *llpart;   // per-tile sums of x log m
    int nll;
    double *dst;
};

// One block of the total: `block` in [0, part0[N]); the blocks of one total
// may come from one launch or from a launch shared with other tensors.
template <typename T>
__device__ __forceinline__ void ll_total_body(const LLTotalArgs &a, int block) {
    __shared__ double sm[256];
    __shared__ double cs[kMaxModes][256];
    __shared__ bool last;
    const int tid = threadIdx.x;
    int m = 0;
    while (m + 1 < a.N && block >= a.part0[m + 1]) ++m;
    const int Rp = a.Rp;
    const int p = block - a.part0[m];
    const int nparts = a.part0[m + 1] - a.part0[m];
    const int c = tid % Rp, rl = tid / Rp, nrl = blockDim.x / Rp;
    const T *M = reinterpret_cast<const T *>(a.A[m]);
    double s = 0.0;
    if (rl < nrl)
        for (int64_t i = (int64_t)p * nrl + rl; i < a.rows[m]; i += (int64_t)nparts * nrl) s += (double)M[i * Rp + c];
    sm[tid] = s;
    __syncthreads();
    if (tid < Rp) {
        double t = 0.0;
        for (int k = 0; k < nrl; ++k) t += sm[k * Rp + tid];
        a.part[(int64_t)block * Rp + tid] = t;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(a.counter, 1u) == (unsigned)a.part0[a.N] - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // sum of the tile partials: per-thread strided sums, then a tree
    double v = 0.0;
    for (int i = tid; i < a.nll; i += 256) v += __ldcg(a.llpart + i);
    sm[tid] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) sm[tid] += sm[tid + w];
        __syncthreads();
    }
    // column sums of every factor, partials in order
    if (tid < Rp)
        for (int mm = 0; mm < a.N; ++mm) {
            double t = 0.0;
            for (int q = a.part0[mm]; q < a.part0[mm + 1]; ++q) t += __ldcg(a.part + (int64_t)q * Rp + tid);
            cs[mm][tid] = t;
        }
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int cc = 0; cc < Rp; ++cc) {
            double pr = a.lambda[cc];
            for (int mm = 0; mm < a.N; ++mm) pr *= cs[mm][cc];
            tot += pr;
        }
        *a.dst = sm[0] - tot;
        *a.counter = 0u;  // ready for the next launch
    }
}

// Arguments of one tensor's total (blocks = part0[N]); host side, mu.cu.
LLTotalArgs ll_total_args(const cpapr_ctx *ctx, const double *llpart, int nll, double *dst);

}  // namespace cpapr
