// CP-APR MU driver (Algorithm 1 of arXiv 2307.03276).
//
// Per outer iteration and mode n, everything stays on the device:
//   sb_kernel                    B <- (A^(n) + S) Lambda, inner state reset
//   pi_build_kernel              Khatri-Rao rows of mode n (if materialised)
//   inner loop (<= max_inner):   Phi tile kernel with the KKT violation
//                                folded in, then update_kernel
//                                (B <- B * Phi unless the check passed)
//   normalise                    lambda <- e^T B, A^(n) <- B Lambda^-1
// The inner loop runs either as plain stream launches whose kernels return
// at once after the check passed, or as a CUDA graph holding a conditional
// WHILE node whose body is {Phi, update}; update_kernel clears the
// loop condition on the device, so no host round trip decides the exit.
// The host reads the per-mode inner states back once per outer iteration to
// test outer convergence (every mode passed its check at the first inner
// iteration).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace cpapr {

cpapr_status configure_mode(cpapr_ctx *ctx, int n, int lanes, int tile, int reduction);

static cpapr_status build_inner_graph(cpapr_ctx *ctx, int n, double tol, int max_inner) {
    if (ctx->graph_exec[n]) {
        if (ctx->graph_max_inner[n] == max_inner && ctx->graph_tol[n] == tol) return CPAPR_OK;
        cudaGraphExecDestroy(ctx->graph_exec[n]);
        ctx->graph_exec[n] = nullptr;
    }
    cudaGraph_t g = nullptr;
    CPAPR_CUDA(ctx, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "cudaGraphConditionalHandleCreate");
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "cudaGraphAddNode(conditional)");
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "cudaStreamBeginCaptureToGraph");
    }
    InnerState *inner = ctx->inner + n;
    ctx->graph_capture_kernels = 0;
    cpapr_status st = launch_phi(ctx, n, OP_PHI, ctx->B, ctx->Phi[n], inner);
    if (st == CPAPR_OK) st = launch_update(ctx, n, tol, max_inner, inner, (unsigned long long)h, 1);
    ctx->graph_body_kernels[n] = ctx->graph_capture_kernels;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(ctx->stream, &captured);
    if (st != CPAPR_OK) {
        cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "cudaStreamEndCapture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    ctx->graph_exec[n] = exec;
    ctx->graph_max_inner[n] = max_inner;
    ctx->graph_tol[n] = tol;
    return CPAPR_OK;
}

// Enqueues one mode's part of an outer iteration (no host synchronisation).
static cpapr_status enqueue_mode(cpapr_ctx *ctx, int n, double tol, int max_inner, bool shift) {
    InnerState *inner = ctx->inner + n;
    CPAPR_TRY(launch_sb(ctx, n, shift, inner));
    CPAPR_TRY(launch_empty_kkt(ctx, n, ctx->B, inner));
    // the other modes' factors are fixed for this inner loop: their
    // Khatri-Rao rows are built once here if the mode streams them
    CPAPR_TRY(launch_pi_build(ctx, n));
    if (ctx->opt.use_graph) {
        CPAPR_TRY(build_inner_graph(ctx, n, tol, max_inner));
        CPAPR_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec[n], ctx->stream));
    } else {
        for (int l = 0; l < max_inner; ++l) {
            CPAPR_TRY(launch_phi(ctx, n, OP_PHI, ctx->B, ctx->Phi[n], inner));
            CPAPR_TRY(launch_update(ctx, n, tol, max_inner, inner, 0ull, 0));
        }
    }
    CPAPR_TRY(launch_normalise(ctx, n));
    return CPAPR_OK;
}

// Enqueues the log-likelihood of the current model and its copy to *host
// (complete after the context's stream is synchronised).
cpapr_status loglik_enqueue(cpapr_ctx *ctx, double *host) {
    CPAPR_TRY(launch_loglik(ctx, ctx->scalars));
    CPAPR_CUDA(ctx, cudaMemcpyAsync(host, ctx->scalars, 8, cudaMemcpyDeviceToHost, ctx->stream));
    return CPAPR_OK;
}

static cpapr_status loglik_now(cpapr_ctx *ctx, double *host) {
    CPAPR_TRY(loglik_enqueue(ctx, host));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CPAPR_OK;
}

cpapr_status launch_loglik_host(cpapr_ctx *ctx, double *host) { return loglik_now(ctx, host); }

cpapr_status batch_mu_solve_persistent(cpapr_ctx *const *ctxs, int count, double tol, int max_outer, int max_inner,
                                       cpapr_result *results);

cpapr_status mu_solve(cpapr_ctx *ctx, double tol, int max_outer, int max_inner, cpapr_result *res,
                      int32_t *inner_trace, double *ll_trace, double *kkt_trace) {
    const int N = ctx->N;
    std::vector<InnerState> hs(N);
    int outer = 0, total_inner = 0;
    bool conv = false;
    double kkt_last = 0.0;
    for (int k = 0; k < max_outer; ++k) {
        const bool shift = ctx->k_total > 0;
        for (int n = 0; n < N; ++n) CPAPR_TRY(enqueue_mode(ctx, n, tol, max_inner, shift));
        CPAPR_CUDA(ctx, cudaMemcpyAsync(hs.data(), ctx->inner, sizeof(InnerState) * N, cudaMemcpyDeviceToHost,
                                        ctx->stream));
        CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->k_total += 1;
        ++outer;
        bool all_first = true;
        double kmax = 0.0;
        for (int n = 0; n < N; ++n) {
            total_inner += hs[n].used;
            if (ctx->opt.use_graph) ctx->launches += (int64_t)hs[n].used * ctx->graph_body_kernels[n];
            if (!(hs[n].passed && hs[n].used == 1)) all_first = false;
            kmax = std::max(kmax, hs[n].viol);
            if (inner_trace) inner_trace[(int64_t)k * N + n] = hs[n].used;
        }
        kkt_last = kmax;
        if (kkt_trace) kkt_trace[k] = kmax;
        if (ll_trace) CPAPR_TRY(loglik_now(ctx, &ll_trace[k]));
        if (all_first) {
            conv = true;
            break;
        }
    }
    double ll = 0.0;
    CPAPR_TRY(loglik_now(ctx, &ll));
    res->outer_iters = outer;
    res->total_inner = total_inner;
    res->converged = conv ? 1 : 0;
    res->reserved = 0;
    res->loglik = ll;
    res->kkt_viol = kkt_last;
    return CPAPR_OK;
}

// Batch.  Contexts that share the device and the number of modes run through
// the persistent batched kernels (batch.cu).  Otherwise the contexts' outer
// iterations advance in lock step: the work of all still-running contexts is
// enqueued on their streams before any host synchronisation, so one round
// trip per outer iteration covers the batch.
cpapr_status batch_mu_solve(cpapr_ctx *const *ctxs, int count, double tol, int max_outer, int max_inner,
                            cpapr_result *results) {
    if (count == 0) return CPAPR_OK;
    bool uniform = true;
    for (int i = 1; i < count; ++i)
        uniform = uniform && ctxs[i]->N == ctxs[0]->N && ctxs[i]->device == ctxs[0]->device;
    if (uniform) return batch_mu_solve_persistent(ctxs, count, tol, max_outer, max_inner, results);
    struct Track {
        int outer = 0, total = 0;
        bool conv = false, active = true;
        double kkt = 0.0;
    };
    std::vector<Track> tr(count);
    std::vector<std::vector<InnerState>> hs(count);
    for (int i = 0; i < count; ++i) hs[i].resize(ctxs[i]->N);
    for (int k = 0; k < max_outer; ++k) {
        bool any = false;
        for (int i = 0; i < count; ++i) {
            if (!tr[i].active) continue;
            any = true;
            cpapr_ctx *c = ctxs[i];
            const bool shift = c->k_total > 0;
            for (int n = 0; n < c->N; ++n) CPAPR_TRY(enqueue_mode(c, n, tol, max_inner, shift));
            CPAPR_CUDA(c, cudaMemcpyAsync(hs[i].data(), c->inner, sizeof(InnerState) * c->N, cudaMemcpyDeviceToHost,
                                          c->stream));
        }
        if (!any) break;
        for (int i = 0; i < count; ++i) {
            if (!tr[i].active) continue;
            cpapr_ctx *c = ctxs[i];
            CPAPR_CUDA(c, cudaStreamSynchronize(c->stream));
            c->k_total += 1;
            tr[i].outer += 1;
            bool all_first = true;
            double kmax = 0.0;
            for (int n = 0; n < c->N; ++n) {
                tr[i].total += hs[i][n].used;
                if (c->opt.use_graph) c->launches += (int64_t)hs[i][n].used * c->graph_body_kernels[n];
                if (!(hs[i][n].passed && hs[i][n].used == 1)) all_first = false;
                kmax = std::max(kmax, hs[i][n].viol);
            }
            tr[i].kkt = kmax;
            if (all_first) {
                tr[i].conv = true;
                tr[i].active = false;
            }
        }
    }
    for (int i = 0; i < count; ++i) {
        double ll = 0.0;
        CPAPR_TRY(loglik_now(ctxs[i], &ll));
        results[i].outer_iters = tr[i].outer;
        results[i].total_inner = tr[i].total;
        results[i].converged = tr[i].conv ? 1 : 0;
        results[i].reserved = 0;
        results[i].loglik = ll;
        results[i].kkt_viol = tr[i].kkt;
    }
    return CPAPR_OK;
}

// ---- tuned-choice cache -------------------------------------------------------
// One text line per shape class:
//   cpapr-tune-1 <key> <lanes> <tile> <reduction> <pi> <ms>
// The key names what the best choice depends on: the precision, the number
// of modes, the padded rank and power-of-two buckets of the nonzeros, of the
// mode's rows and of the nonzeros per non-empty row (how many rows a tile
// crosses).  The last line of a key wins.
struct TuneChoice {
    int lanes = 0, tile = 0, reduction = 0, pi = 0;
};

static int log2_bucket(double v) { return v >= 1.0 ? (int)std::lround(std::log2(v)) : 0; }

static std::string tune_key(const cpapr_ctx *ctx, int n) {
    const ModeLayout &L = ctx->mode[n];
    const double rows = (double)ctx->dims[n];
    const double nonempty = std::max(1.0, rows - (double)L.nempty);
    char buf[160];
    std::snprintf(buf, sizeof buf, "%s/N%d/Rp%d/nnz2^%d/rows2^%d/per_row2^%d", ctx->esize == 8 ? "f64" : "f32", ctx->N,
                  ctx->Rp, log2_bucket((double)ctx->nnz), log2_bucket(rows), log2_bucket((double)ctx->nnz / nonempty));
    return buf;
}

static std::mutex g_tune_mu;

static bool tune_lookup(const char *path, const std::string &key, TuneChoice *out) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512], k[256];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        TuneChoice c;
        float ms = 0.f;
        if (std::sscanf(line, "cpapr-tune-1 %255s %d %d %d %d %f", k, &c.lanes, &c.tile, &c.reduction, &c.pi, &ms) == 6 &&
            key == k) {
            *out = c;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

static void tune_store(const char *path, const std::string &key, const TuneChoice &c, float ms) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE *f = std::fopen(path, "a");
    if (!f) return;  // an unwritable cache only costs the next create its timing
    std::fprintf(f, "cpapr-tune-1 %s %d %d %d %d %.6f\n", key.c_str(), c.lanes, c.tile, c.reduction, c.pi, ms);
    std::fclose(f);
}

// A cached choice this tensor can run (else it is ignored).
static bool choice_fits(const cpapr_ctx *ctx, const TuneChoice &c) {
    if (!phi_config_supported((int)ctx->esize, ctx->N - 1, ctx->Rp, c.lanes)) return false;
    if (c.tile < 64 || c.tile > (1 << 20) || c.tile % 4) return false;
    if (c.reduction != CPAPR_REDUCE_ATOMIC && c.reduction != CPAPR_REDUCE_SEGMENTED) return false;
    if (c.pi != 0 && c.pi != 1) return false;
    if (c.pi && !pi_fits(ctx)) return false;
    return phi_smem_for((int)ctx->esize, ctx->N - 1, c.tile, ctx->Rp, c.lanes) <= kMaxPhiSmem;
}

// Times each supported (lanes, tile, reduction, Pi form) choice on the
// tensor's own data, one Phi per candidate after a warm-up, and keeps the
// fastest per mode -- the analogue of the paper's Kokkos policy grid search
// (league / team / vector sizes, Experiments 3 to 6), chosen per mode
// because the paper finds the best policy differs across modes.  Each
// candidate runs as a Phi of the MU inner loop does: with the mode's inner
// state, so the segmented form publishes its fused KKT violation and the
// atomic form pays for zeroing its output and its separate KKT pass.  With a
// cache file, modes whose shape class it holds take the cached choice.
cpapr_status autotune(cpapr_ctx *ctx) {
    if (ctx->nnz == 0) return CPAPR_OK;
    const int Rp = ctx->Rp;
    const char *cache = ctx->opt.tune_cache;
    std::vector<std::string> keys(ctx->N);
    std::vector<int> todo;
    for (int n = 0; n < ctx->N; ++n) {
        keys[n] = tune_key(ctx, n);
        TuneChoice c;
        if (cache && tune_lookup(cache, keys[n], &c) && choice_fits(ctx, c)) {
            CPAPR_TRY(configure_mode(ctx, n, c.lanes, c.tile, c.reduction));
            CPAPR_TRY(configure_pi(ctx, n, c.pi));
        } else if (ctx->opt.autotune) {
            todo.push_back(n);
        }
    }
    if (todo.empty()) return CPAPR_OK;
    cudaEvent_t e0, e1;
    CPAPR_CUDA(ctx, cudaEventCreate(&e0));
    CPAPR_CUDA(ctx, cudaEventCreate(&e1));
    // a neutral model for timing: uniform factors
    std::vector<double> ones((size_t)ctx->Imax * ctx->R, 1.0 / 64.0);
    for (int m = 0; m < ctx->N; ++m) CPAPR_TRY(upload_factor(ctx, m, ones.data()));
    std::vector<double> lam(Rp, 1.0);
    CPAPR_CUDA(ctx, cudaMemcpyAsync(ctx->lambda, lam.data(), Rp * 8, cudaMemcpyHostToDevice, ctx->stream));
    CPAPR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int n : todo) {
        CPAPR_TRY(launch_scale_b(ctx, n, ctx->B));
        InnerState *inner = ctx->inner + n;
        float best = 1e30f;
        TuneChoice bc;
        bc.lanes = ctx->mode[n].lanes;
        bc.tile = ctx->mode[n].tile_nnz;
        bc.reduction = ctx->mode[n].reduction;
        bc.pi = ctx->mode[n].pi;
        const int tiles[] = {1024, 2048, 4096, 8192};
        // the materialised Khatri-Rao rows are a candidate where their buffer
        // fits (the fixed cost of building them once per inner loop is not
        // timed: it is spread over the inner iterations)
        const int npi = pi_fits(ctx) ? 2 : 1;
        for (int lanes = 1; lanes <= 32; lanes <<= 1) {
            if (!phi_config_supported((int)ctx->esize, ctx->N - 1, Rp, lanes)) continue;
            for (int tile : tiles) {
                // MTTKRP and the log-likelihood share the mode's tiles and stage every
                // coordinate stream: keep room for two of their blocks per SM
                if (phi_smem_for((int)ctx->esize, ctx->N - 1, tile, Rp, lanes) > kMaxPhiSmem / 2) continue;
                for (int cand = 0; cand < 2 * npi; ++cand) {
                    const int red = cand % 2 ? CPAPR_REDUCE_SEGMENTED : CPAPR_REDUCE_ATOMIC;
                    const int pi = cand / 2;
                    CPAPR_TRY(configure_mode(ctx, n, lanes, tile, red));
                    CPAPR_TRY(configure_pi(ctx, n, pi));
                    if (pi) CPAPR_TRY(launch_pi_build(ctx, n));
                    // a fresh inner state: not done, violation slots clear
                    CPAPR_CUDA(ctx, cudaMemsetAsync(inner, 0, sizeof(InnerState), ctx->stream));
                    CPAPR_TRY(launch_phi(ctx, n, OP_PHI, ctx->B, ctx->outbuf, inner));
                    CPAPR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
                    for (int rep = 0; rep < 3; ++rep) CPAPR_TRY(launch_phi(ctx, n, OP_PHI, ctx->B, ctx->outbuf, inner));
                    CPAPR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
                    CPAPR_CUDA(ctx, cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CPAPR_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best) {
                        best = ms;
                        bc.lanes = lanes;
                        bc.tile = tile;
                        bc.reduction = red;
                        bc.pi = pi;
                    }
                }
            }
        }
        CPAPR_TRY(configure_mode(ctx, n, bc.lanes, bc.tile, bc.reduction));
        CPAPR_TRY(configure_pi(ctx, n, bc.pi));
        CPAPR_CUDA(ctx, cudaMemsetAsync(inner, 0, sizeof(InnerState), ctx->stream));
        if (cache) tune_store(cache, keys[n], bc, best / 3.f);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // leave no model behind: the caller sets one
    ctx->model_set = false;
    return CPAPR_OK;
}

}  // namespace cpapr
