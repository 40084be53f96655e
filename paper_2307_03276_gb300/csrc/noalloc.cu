// cpapr_phi_noalloc: Phi^(n) without any device allocation in the call.
//
// Who needs this: a caller whose device memory is owned by someone else (a
// framework's caching allocator that has reserved the GPU, a fixed memory
// budget), or whose calls sit in a loop that must not block on the driver's
// allocator, cannot let the library call cudaMalloc/cudaFree per call.
// cpapr_phi itself allocates nothing either, but the Phi kernel's scratch
// (the per-tile partial rows of rows that span tiles, which the last tile to
// arrive adds up) lives in a buffer sized at cpapr_create time and grown
// with a stream-ordered allocation when the tiling changes.  This variant takes that scratch from a fixed array in
// device memory that the library image carries, so the call itself only
// launches kernels and copies between device buffers.
//
// The array is file-scope `static __device__` storage of
// CPAPR_NOALLOC_SCRATCH_BYTES bytes: every GPU that loads the library holds it
// until the process exits.  In host code its name is only a host-side stand-in,
// so the device address is looked up with cudaGetSymbolAddress, once per
// device, by the first call on a context of that device (with the context's
// device made current for the call and the caller's device restored after).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace cpapr {
cpapr_status launch_phi_given_carry(cpapr_ctx *ctx, int n, const void *B, void *out, void *carry);
}

using namespace cpapr;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CPAPR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Makes ctx->device current for the lifetime of the guard and puts the
// caller's device back afterwards, on every return path.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
        else if (err == cudaSuccess) prev = -1;  // already current: nothing to restore
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Device address of the scratch array on ctx->device (which the caller has
// made current), looked up once per device.
cpapr_status scratch_address(cpapr_ctx *ctx, void **out) {
    const int dev = ctx->device;
    if (dev < 0 || dev >= kMaxDevices) return fail(ctx, CPAPR_E_ARG, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(ctx, CPAPR_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CPAPR_OK;
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" cpapr_status cpapr_phi_noalloc(cpapr_ctx *ctx, int32_t mode, const double *B, double *out) {
    if (!ctx) return fail(nullptr, CPAPR_E_ARG, "ctx is NULL");
    if (ctx->sticky) return CPAPR_E_CUDA;
    if (mode < 0 || mode >= ctx->N) return fail(ctx, CPAPR_E_ARG, "mode out of range");
    if (!ctx->model_set) return fail(ctx, CPAPR_E_STATE, "no model set");
    if (!out || !is_device_pointer(out)) return fail(ctx, CPAPR_E_ARG, "out must be a device pointer");
    if (B && !is_device_pointer(B)) return fail(ctx, CPAPR_E_ARG, "B must be NULL or a device pointer");
    const ModeLayout &L = ctx->mode[mode];
    const int64_t need = (int64_t)2 * L.ntiles * ctx->Rp * (int64_t)ctx->esize;
    if (need > (int64_t)CPAPR_NOALLOC_SCRATCH_BYTES)
        return fail(ctx, CPAPR_E_RANGE,
                    "cpapr_phi_noalloc: this mode needs " + std::to_string(need) + " bytes of scratch (2 x " +
                        std::to_string(L.ntiles) + " tiles x " + std::to_string(ctx->Rp) +
                        " ranks); the fixed scratch holds " + std::to_string((long long)CPAPR_NOALLOC_SCRATCH_BYTES) +
                        ": use cpapr_phi, or a larger tile_nnz");
    DeviceGuard guard(ctx->device);
    if (guard.err != cudaSuccess)
        return fail(ctx, CPAPR_E_CUDA, std::string("selecting the context's device: ") + cudaGetErrorString(guard.err));
    void *scratch = nullptr;
    CPAPR_TRY(scratch_address(ctx, &scratch));
    if (ctx->nnz == 0) {
        CPAPR_CUDA(ctx, cudaMemsetAsync(out, 0, (size_t)ctx->dims[mode] * ctx->R * 8, ctx->stream));
    } else {
        if (B)
            CPAPR_TRY(upload_matrix(ctx, B, ctx->dims[mode], ctx->B));
        else
            CPAPR_TRY(launch_scale_b(ctx, mode, ctx->B));
        // the per-tile partials land in the fixed scratch; every slot a
        // finishing tile reads is written earlier in this launch, so nothing
        // is cleared (the materialised rows, if the mode uses them, live in
        // the context's buffer and are rebuilt for this call)
        CPAPR_TRY(launch_pi_build(ctx, mode));
        CPAPR_TRY(launch_phi_given_carry(ctx, mode, ctx->B, ctx->outbuf, scratch));
        CPAPR_TRY(download_matrix(ctx, ctx->outbuf, ctx->dims[mode], out));
    }
    // Did a tile's bounded staging wait give up?  Such a tile never wrote its
    // rows nor counted its partials: clear the flag and every mode's
    // partial counters (plain memsets, no allocation) and report it.
    int32_t waited_out = 0;
    CPAPR_CUDA(ctx, cudaMemcpyAsync(&waited_out, ctx->errflag + 3, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (waited_out) {
        CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->errflag + 3, 0, 4, ctx->stream));
        for (int n = 0; n < ctx->N; ++n)
            if (ctx->mode[n].splitcnt)
                CPAPR_CUDA(ctx, cudaMemsetAsync(ctx->mode[n].splitcnt, 0,
                                                (size_t)std::max(ctx->mode[n].nsplit, 1) * 4, ctx->stream));
        CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return fail(ctx, CPAPR_E_TIMEOUT, "a device-side staging wait gave up; out is incomplete");
    }
    return CPAPR_OK;
}
