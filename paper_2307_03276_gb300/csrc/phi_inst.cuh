// Instantiates the Phi tile kernels for one working type (PHI_T) and one
// gathered-mode count (PHI_NM1; 0 = runtime count) and exposes a launcher.
// Included by the small phi_<type>_<nm1>.cu units so that the template
// instantiations compile in parallel.
#include "phi_kernels.cuh"

#ifndef PHI_T
#error "define PHI_T"
#endif
#ifndef PHI_NM1
#error "define PHI_NM1"
#endif
#ifndef PHI_FN
#error "define PHI_FN"
#endif

namespace cpapr {

namespace {
constexpr int kThreads = sizeof(PHI_T) == 8 ? 128 : 256;
// nonzeros per batch (U <= G when G > 1: after the reduce-scatter every lane
// finishes one of them, so a nonzero costs G / U divisions; one lane per
// nonzero takes two at a time for memory-level parallelism).  FP64 at 16
// ranks per lane has no registers to spare for a second batch entry; FP64 at
// 8 or fewer takes two: with four its kernel with the dot on the FP32 pipe
// needed 178 registers and ran 37% slower on the 3-way tensor (1.63 vs 1.19
// ms on GB300), and both kernels share the batch size.
template <int RPL, int G>
constexpr int unroll_for() {
    if (sizeof(PHI_T) == 8) return RPL >= 16 ? (G >= 2 ? 2 : 1) : 2;
    return G >= 4 ? 4 : 2;
}

// win: persisting-L2 window for the launch, or null for a plain launch
template <int RPL, typename K>
cudaError_t launch(K k, const PhiArgs &a, cudaStream_t s, const cudaAccessPolicyWindow *win) {
    const size_t smem = phi_smem_bytes(a.T, a.pi ? 0 : a.nm1, (int)sizeof(PHI_T), kThreads, RPL);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (a.ntiles <= 0) return cudaGetLastError();
    if (!win) {
        k<<<a.ntiles, kThreads, smem, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow = *win;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.ntiles);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

template <int RPL, int G, int OP, bool PI>
cudaError_t run(const PhiArgs &a, cudaStream_t s, const cudaAccessPolicyWindow *win) {
    constexpr int U = unroll_for<RPL, G>();
    // the log-likelihood's underflow fallback needs more registers than four
    // blocks per SM allow (measured: 7% faster unconstrained)
    if constexpr (phi_occ4<PHI_T, RPL>() && OP != OP_LL) {
        return launch<RPL>(phi_tile_kernel_occ4<PHI_T, PHI_NM1, RPL, G, OP, kThreads, U, PI>, a, s, win);
    } else {
        // FP64 Phi with 8 or fewer ranks per lane: the launcher's choice of the
        // kernel that takes the dot on the FP32 pipe
        if constexpr (sizeof(PHI_T) == 8 && OP == OP_PHI && RPL <= 8) {
            if (a.dfdot) return launch<RPL>(phi_tile_kernel_df<PHI_T, PHI_NM1, RPL, G, OP, kThreads, U, PI>, a, s, win);
        }
        return launch<RPL>(phi_tile_kernel<PHI_T, PHI_NM1, RPL, G, OP, kThreads, U, PI>, a, s, win);
    }
}
// log-likelihood: FP64 can stream the materialised rows, FP32 always gathers
template <int RPL, int G>
cudaError_t run_ll(const PhiArgs &a, cudaStream_t s, const cudaAccessPolicyWindow *win) {
    if constexpr (sizeof(PHI_T) == 8) {
        if (a.pi) return run<RPL, G, OP_LL, true>(a, s, win);
    }
    return run<RPL, G, OP_LL, false>(a, s, win);
}
}  // namespace

// Returns cudaErrorInvalidValue when (rpl, lanes) has no instantiation.
// Phi reads the materialised Khatri-Rao rows when a.pi is set.
cudaError_t PHI_FN(const PhiArgs &a, int rpl, int lanes, int op, cudaStream_t s, const cudaAccessPolicyWindow *win) {
#define CPAPR_CASE(R_, G_)                                                                          \
    if (rpl == R_ && lanes == G_) {                                                                 \
        if (op == OP_PHI)                                                                           \
            return a.pi ? run<R_, G_, OP_PHI, true>(a, s, win) : run<R_, G_, OP_PHI, false>(a, s, win); \
        if (op == OP_MTTKRP) return run<R_, G_, OP_MTTKRP, false>(a, s, win);                      \
        return run_ll<R_, G_>(a, s, win);                                                           \
    }
#if PHI_IS_DOUBLE
    CPAPR_CASE(2, 1)
    CPAPR_CASE(4, 1)
    CPAPR_CASE(8, 1)
    CPAPR_CASE(16, 1)
    CPAPR_CASE(8, 2)
    CPAPR_CASE(16, 2)
    CPAPR_CASE(8, 4)
    CPAPR_CASE(16, 4)
    CPAPR_CASE(8, 8)
    CPAPR_CASE(16, 8)
    CPAPR_CASE(8, 16)
#else
    CPAPR_CASE(4, 1)
    CPAPR_CASE(8, 1)
    CPAPR_CASE(16, 1)
    CPAPR_CASE(4, 2)
    CPAPR_CASE(8, 2)
    CPAPR_CASE(4, 4)
    CPAPR_CASE(8, 4)
    CPAPR_CASE(4, 8)
    CPAPR_CASE(8, 8)
    CPAPR_CASE(4, 16)
    CPAPR_CASE(8, 16)
#endif
#undef CPAPR_CASE
    return cudaErrorInvalidValue;
}

}  // namespace cpapr
