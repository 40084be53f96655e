#!/usr/bin/env python3
"""CP-APR MU Phi^(n) throughput on GB300 (one JSON line on stdout).

Workload (default): the 4-way 200,000 x 200,000 x 10,000 x 365 count tensor
with 50,000,000 distinct nonzeros, Zipf(1.1) coordinates in modes 1-2 and
uniform ones in modes 3-4, geometric(0.5) counts, rank R = 16, seeded
synthetic (a stand-in for the FROSTT tensors of the paper, which are not
available here).  --workload c2 selects the 3-way 1e5 x 1e5 x 1e3 tensor
with 1e7 nonzeros and R = 32.

One step = one outer iteration of Algorithm 1 over every mode (S and B, up to
10 inner iterations of Phi with the KKT check and the multiplicative update,
lambda normalisation) followed by the Poisson log-likelihood.  The unit is a
nonzero visited by a Phi^(n) evaluation; `value` = Phi nonzero visits of all
ranks / the slowest rank's device time for the K timed steps, with every
other kernel of the step counted as overhead.  The per-mode layouts (4.8 GB
of index and value streams for the 4-way tensor) exceed the 129 MB L2, so no
flush is needed between steps; the factor matrices stay L2-resident by
design.

Reported beside it: the FP32 form of the same step, the FP64 step with the
Khatri-Rao rows formed in place, the 3-way tensor's FP64 and FP32 steps, the
roofline of the dominant kernel (the Phi tile kernel), an end-to-end number
through the C ABI from pinned host buffers, MTTKRP kernel throughput, the
batched solver, the time to KKT tolerance 1e-4 (a small tensor solved to the
tolerance, the headline tensor to a violation level FP64 and FP32 both
reach, the 64-tensor batch), the clocks seen during the timed region and the
FP64 oracle timed on the host's cores (all of them, and one).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  torchrun --nproc-per-node N bench.py --gpus N ...   (replicas: one per GPU)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Φ^(n) nonzeros/s and HBM GB/s (FP64 vs FP32 vs batched, 1 GB300)"
UNIT = "nnz/s"
TOL = 1e-4
MAX_INNER = 10
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}
# GB300: 152 SMs x 2 FP64 FMA per SM per clock x 2 FLOP x 2.07 GHz (nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# random-row gather from an L2-resident table, 128-byte rows, measured on this GB300
L2_GATHER_GBS = 7450.0


# DRAM bytes per Phi launch by mode (dram__bytes_read.sum + dram__bytes_write.sum) from ncu captures of
# the kernel configuration named in the key (workload, dtype, Pi form, lanes per mode, tile per mode).
# "nnz" is the nonzero count of the captured tensor: the 4-way workload was captured on a copy with the
# same dims, rank and distributions but 1e7 nonzeros (a few GB on the device, as the capture rules ask);
# its traffic is scaled to the full tensor per mode as (bytes - io) * nnz_full / nnz + io, where io is
# the algorithmic B read plus Phi write (2 R b_f I_n), the only part that does not grow with the
# nonzeros.  "l2_read" is lts__t_sectors_srcunit_tex_op_read.sum x 32 bytes (the L2 bytes read by L1
# misses: the gathered factor rows the L1 did not hold) for a fused configuration.  A run in any other
# configuration reports traffic null; an entry is dropped when its kernel changes.
NCU_TRAFFIC = {
    ("c2_3way_1e5x1e5x1e3_1e7_r32", "f64", "materialised", (4, 4, 4), (1024, 1024, 1024)):
        {"bytes": [2668266240 + 18964736, 2667915520 + 16923904, 2642699520 + 6055680], "nnz": 10_000_000,
         "source": "ncu capture of the FP64 materialised-Pi tile kernel, modes 0-2"},
    ("c2_3way_1e5x1e5x1e3_1e7_r32", "f32", "fused", (8, 8, 8), (2048, 2048, 2048)):
        {"bytes": [149920512 + 9855744, 149870848 + 6829568, 150985472 + 916480], "nnz": 10_000_000,
         "l2_read": [46078048 * 32, 45825406 * 32, 56520460 * 32],
         "source": "ncu capture of the FP32 fused-Pi tile kernel, modes 0-2"},
    ("c3_4way_2e5x2e5x1e4x365_5e7_r16", "f64", "materialised", (2, 2, 2, 2), (2048, 2048, 2048, 2048)):
        {"bytes": [1386862336 + 12523776, 1386850048 + 12308224, 1362785024 + 3010048, 1361540096 + 3038976],
         "nnz": 10_000_000,
         "source": "ncu capture of the FP64 materialised-Pi tile kernel, modes 0-3, on the 4-way tensor's "
                   "1e7-nonzero copy (same dims), scaled to 5e7 nonzeros"},
    ("c3_4way_2e5x2e5x1e4x365_5e7_r16", "f32", "materialised", (4, 4, 4, 4), (4096, 4096, 4096, 4096)):
        {"bytes": [694905088 + 3333888, 694989056 + 212992, 682062336 + 261888, 681425920 + 171520],
         "nnz": 10_000_000,
         "source": "ncu capture of the FP32 materialised-Pi tile kernel, modes 0-3, on the 4-way tensor's "
                   "1e7-nonzero copy (same dims), scaled to 5e7 nonzeros"},
}


def layout_bytes(T) -> int:
    """Bytes of the per-mode sorted layouts that every step streams: the other
    modes' int32 coordinates, the FP64 values and one row-start bit per
    nonzero, for each mode."""
    return T.nmodes * (T.nnz * (4 * (T.nmodes - 1) + 8) + T.nnz // 8)


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    except OSError:
        return dict(FALLBACK_PEAKS)


# ---------------------------------------------------------------------------
# byte and FLOP models (per Phi^(n) launch over the whole tensor)
# ---------------------------------------------------------------------------

def phi_bytes(dims, nnz, R, n, value_bytes, factor_bytes, materialised=False) -> float:
    """Compulsory HBM bytes of one Phi^(n).  Fused Khatri-Rao rows: the mode-n
    index and value streams, the row offsets, one read of every other factor
    and of B, one write of Phi.  Materialised rows (the paper's Pi): the
    values, the Pi stream (R values per nonzero), the row offsets, one read
    of B and one write of Phi."""
    N = len(dims)
    if materialised:
        return nnz * (value_bytes + R * factor_bytes) + 4 * (dims[n] + 1) + factor_bytes * R * 2 * dims[n]
    other = sum(dims) - dims[n]
    return nnz * (4 * (N - 1) + value_bytes) + 4 * (dims[n] + 1) + factor_bytes * R * (other + 2 * dims[n])


def phi_flops(N, nnz, R, materialised=False) -> float:
    """Fused: (N-2)R Khatri-Rao products, 2R dot, max + divide, 2R scale-add
    per nonzero.  Materialised: the products are done once per inner loop by
    the Pi build, so a Phi costs 4R + 2 (the paper's own count)."""
    return nnz * (4 * R + 2) if materialised else nnz * ((N + 2) * R + 2)


def phi_fp64_pipe_flops(N, nnz, R, materialised=False, dot_on_fp32=True) -> float:
    """The part of phi_flops the FP64 Phi kernel runs on the FP64 pipe: with
    the divisor x / max(<B, pi>, eps) on the FP32 pipe (8 or fewer ranks per
    lane, eps >= 2^-43) the dot's 2R and the max and divide leave it, leaving
    the scale-add and, fused, the Khatri-Rao products."""
    return phi_flops(N, nnz, R, materialised) - (nnz * (2 * R + 2) if dot_on_fp32 else 0)


def phi_gather_bytes(N, nnz, R, factor_bytes, materialised=False) -> float:
    """Factor-row bytes the Phi walk gathers per launch: the N-1 other modes'
    rows per nonzero with fused Khatri-Rao rows; none with materialised rows
    (those are streamed).  The B row is read once per run of a row and kept in
    registers along it, so it is not counted."""
    return 0.0 if materialised else float(nnz) * (N - 1) * R * factor_bytes


# ---------------------------------------------------------------------------
# multi-GPU plumbing (replicas)
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return dist


def barrier(dist, use_cuda: bool):
    if dist is None:
        return
    if use_cuda:
        import torch
        dist.barrier(device_ids=[torch.cuda.current_device()])
    else:
        dist.barrier()


def aggregate(dist, units: float, seconds: float, use_cuda: bool = False):
    """Whole-job units (sum over ranks) and time (max over ranks)."""
    if dist is None:
        return units, seconds
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if use_cuda else torch.device("cpu")
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    s = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3][k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def gpu_selector() -> str | None:
    try:
        import torch
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[0] if vis else None


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(name: str):
    from paper_2307_03276_gb300 import synth
    spec = synth.SPECS[name]
    T = synth.generate(spec)
    lam = np.ones(T.rank)
    fs = synth.random_factors(T.dims, T.rank, spec.seed + 17)
    return T, lam, fs


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_phi_rate(T, lam, fs, S, seconds, threads):
    """Phi^(n) evaluations of the FP64 oracle over the first S nonzeros,
    modes cycled, for about `seconds`: (nnz/s, evaluations, elapsed)."""
    import oracle
    idx = np.ascontiguousarray(T.idx[:, :S])
    vals = np.ascontiguousarray(T.vals[:S])
    done, n = 0, 0
    t0 = time.perf_counter()
    while True:
        B = fs[n] * lam[None, :]
        if threads == 1:
            oracle.phi(T.dims, idx, vals, fs, B, n)
        else:
            oracle.phi_threads(T.dims, idx, vals, fs, B, n, threads)
        done += S
        n = (n + 1) % T.nmodes
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return done / dt, done // S, dt


def cpu_baseline(T, lam, fs, seconds: float = 10.0, sample: int = 1_000_000) -> dict:
    """The FP64 oracle as it stands on a bounded sample of the same tensor:
    on all the host's cores (each thread owns a range of Phi's rows) and,
    beside it, on one core."""
    import oracle
    oracle.build()
    cores = host_cores()
    S1 = min(sample, T.nnz)
    Sm = min(sample * max(1, min(cores, 8)), T.nnz)
    v1, k1, d1 = _oracle_phi_rate(T, lam, fs, S1, seconds / 2, 1)
    vm, km, dm = _oracle_phi_rate(T, lam, fs, Sm, seconds / 2, cores)
    return {"value": vm, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"Phi^(n) over the first {Sm:,} of {T.nnz:,} nonzeros (random draw order), modes cycled, "
                      f"{km} evaluations in {dm:.1f} s, FP64, Neumaier row sums, {cores} threads (each owns a range "
                      f"of Phi's rows; bit-identical to one thread)",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": f"Phi^(n) over the first {S1:,} nonzeros, modes cycled, {k1} evaluations "
                                        f"in {d1:.1f} s, one thread"}}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def timed_solve(cp, torch, T, lam, fs, precision, steps, warmup, dist, use_cuda, clocks=None, pi_mode=0):
    stream = torch.cuda.current_stream()
    t = cp.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, profile=1, use_graph=0,
                  stream=stream.cuda_stream, pi_mode=pi_mode)
    t.set_model(lam, fs)
    for _ in range(warmup):
        t.mu_solve(TOL, 1, MAX_INNER, trace=True, ll_trace=False)
    for k in range(7):
        t.kernel_stats(k, reset=True)
    launches0 = t.info().kernel_launches
    inner = np.zeros(T.nmodes, dtype=np.int64)
    barrier(dist, use_cuda)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        r = t.mu_solve(TOL, 1, MAX_INNER, trace=True, ll_trace=False)
        inner += r["inner"].sum(axis=0)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    barrier(dist, use_cuda)
    ms = e0.elapsed_time(e1)
    stats = {k: t.kernel_stats(k) for k in range(7)}
    launches = t.info().kernel_launches - launches0
    info = t.info()
    # MTTKRP kernel time (outside the timed region)
    for k in (cp.K_MTTKRP,):
        t.kernel_stats(k, reset=True)
    for n in range(T.nmodes):
        t.mttkrp(n)
    for n in range(T.nmodes):
        t.mttkrp(n)
    mt = t.kernel_stats(cp.K_MTTKRP)
    t.close()
    return {"ms": ms, "inner": inner, "stats": stats, "launches": launches, "clocks": clk, "info": info,
            "mttkrp": mt, "last": r}


KKT_MAX_OUTER = 30          # headline workload: outer iterations recorded for the common violation level
KKT_SMALL_MAX_OUTER = 6000  # the 100 x 80 x 60 tensor: solved to the tolerance
KKT_BATCH_MAX_OUTER = 100   # the 64-tensor batch: converged tensors counted


def _solve_timed(cp, torch, t, lam, fs, max_outer, trace=False):
    """Sets the model, runs one mu_solve call of up to max_outer outer
    iterations and returns (result, device ms of the call)."""
    stream = torch.cuda.current_stream()
    t.set_model(lam, fs)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = t.mu_solve(TOL, max_outer, MAX_INNER, trace=trace, ll_trace=False)
    e1.record(stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1)


def time_to_kkt(cp, torch, T, lam, fs, max_outer=KKT_MAX_OUTER, solve_to_tol=False):
    """Time to KKT tolerance through the library's default path (CUDA-graph
    inner loops), FP64 and FP32 from the same initial model.

    solve_to_tol: Algorithm 1 runs until every mode passes its check at the
    first inner iteration (converged) or max_outer.  Otherwise the violation
    of every outer iteration is recorded first (one solve with the trace);
    the common level is the largest of the FP64 and FP32 best violations
    (a level both reach), and each form is then timed, from the same start,
    for exactly the outer iterations it needs to first reach that level
    (the iterates are reproducible run to run, so the second solve repeats
    the first)."""
    stream = torch.cuda.current_stream()
    out = {"workload": T.name, "kkt_tol": TOL, "max_outer": max_outer, "max_inner": MAX_INNER}
    forms = (("fp64", cp.CPAPR_FP64), ("fp32", cp.CPAPR_FP32))
    tensors = {name: cp.Tensor(T.dims, T.idx, T.vals, T.rank, precision=prec, stream=stream.cuda_stream)
               for name, prec in forms}
    try:
        for name, t in tensors.items():
            _solve_timed(cp, torch, t, lam, fs, 1)  # warm-up: graphs, plans, pools
        traces = {}
        for name, t in tensors.items():
            r, ms = _solve_timed(cp, torch, t, lam, fs, max_outer, trace=True)
            traces[name] = np.asarray(r["kkt_trace"])
            ll = r["loglik"]
            out[name] = {"ms": ms, "outer_iters": r["outer_iters"], "total_inner": r["total_inner"],
                         "converged": bool(r["converged"]), "kkt_viol": r["kkt_viol"],
                         "kkt_viol_min": float(traces[name].min()),
                         "loglik": ll if np.isfinite(ll) else None, "loglik_finite": bool(np.isfinite(ll)),
                         "phi_nnz_per_s": r["total_inner"] * T.nnz / (ms / 1e3)}
        if solve_to_tol:
            out["fp32_speedup"] = out["fp64"]["ms"] / out["fp32"]["ms"]
        else:
            level = max(float(tr.min()) for tr in traces.values())
            out["common_level"] = level
            for name, t in tensors.items():
                k = int(np.flatnonzero(traces[name] <= level)[0]) + 1
                r, ms = _solve_timed(cp, torch, t, lam, fs, k, trace=True)
                out[name]["to_common_level"] = {"outer_iters": k, "ms": ms, "total_inner": r["total_inner"],
                                                "kkt_viol": r["kkt_viol"]}
            out["fp32_speedup_at_common_level"] = (out["fp64"]["to_common_level"]["ms"]
                                                   / out["fp32"]["to_common_level"]["ms"])
    finally:
        for t in tensors.values():
            t.close()
    l64, l32 = out["fp64"]["loglik"], out["fp32"]["loglik"]
    out["loglik_rel_diff"] = abs(l32 - l64) / abs(l64) if (l64 is not None and l32 is not None) else None
    return out


def batch_time_to_kkt(cp, torch, max_outer=KKT_BATCH_MAX_OUTER, count=64, per_tensor=True):
    """The 64-tensor batch solved to KKT tolerance 1e-4 (or max_outer) by the
    batched solver and by one mu_solve per tensor (the plain path), FP64 and
    FP32, from the same initial models; converged tensors are counted.  The
    batched and per-tensor solves run the same iterates (the same inner
    iteration counts), so converged tensors reach the tolerance at the same
    outer iteration in both."""
    from paper_2307_03276_gb300 import synth
    tensors = [synth.generate(sp) for sp in synth.batch_specs(count=count)]
    stream = torch.cuda.current_stream()
    out = {"workload": f"c4_batch{count}_3way", "kkt_tol": TOL, "max_outer": max_outer, "tensors": count}
    modes = ("batched", "per_tensor") if per_tensor else ("batched",)
    for pname, prec in (("fp64", cp.CPAPR_FP64), ("fp32", cp.CPAPR_FP32)):
        for mode in modes:
            ts = [cp.Tensor(T.dims, T.idx, T.vals, T.rank, precision=prec, stream=stream.cuda_stream) for T in tensors]
            init = [(np.ones(T.rank), synth.random_factors(T.dims, T.rank, T.seed + 3)) for T in tensors]

            def solve(mo):
                for t, (lam, fs) in zip(ts, init):
                    t.set_model(lam, fs)
                if mode == "batched":
                    return cp.cpapr_batch_mu_solve([t.ctx for t in ts], TOL, mo, MAX_INNER)
                return [t.mu_solve(TOL, mo, MAX_INNER) for t in ts]

            solve(1)  # warm-up
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = solve(max_outer)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            for t in ts:
                t.close()
            conv = [r for r in res if r["converged"]]
            out[f"{pname}_{mode}"] = {
                "ms": ms, "converged": len(conv), "outer_iters_max": max(r["outer_iters"] for r in res),
                "converged_outer_iters_max": max((r["outer_iters"] for r in conv), default=0),
                "unconverged_kkt_viol_max": max((r["kkt_viol"] for r in res if not r["converged"]), default=0.0),
                "total_inner": sum(r["total_inner"] for r in res),
                "phi_nnz_per_s": sum(r["total_inner"] * T.nnz for r, T in zip(res, tensors)) / (ms / 1e3)}
    if per_tensor:
        base = out["fp64_per_tensor"]["ms"]
        out["speedup_vs_fp64_per_tensor"] = {k: base / out[k]["ms"] for k in
                                             ("fp64_batched", "fp32_batched", "fp32_per_tensor")}
    return out


def run_time_to_kkt(args):
    import torch
    from paper_2307_03276_gb300 import build, cpapr as cp
    torch.cuda.set_device(0)
    build.build()
    if args.workload == "c4":
        print(json.dumps({"probe": "time_to_kkt", **batch_time_to_kkt(cp, torch, args.max_outer)}), flush=True)
        return
    T, lam, fs = make_workload(args.workload)
    r = time_to_kkt(cp, torch, T, lam, fs, args.max_outer, solve_to_tol=args.workload == "c1")
    print(json.dumps({"probe": "time_to_kkt", **r}), flush=True)


def batched_run(cp, torch, precision, steps, warmup, count=64, tuned=True):
    """64 uneven 3-way tensors (dims log-uniform up to 20000 x 20000 x 500, nnz
    log-uniform 1e3..1e6, R in {8, 16, 32}): one outer iteration per step for
    the whole batch through the persistent batched solver, and the same work
    as one cpapr_mu_solve per tensor.  With `tuned`, also the batched step
    with contexts whose tiles (and FP64 Pi forms) the autotuner chose per
    shape class through a cache file (tuning time reported apart)."""
    from paper_2307_03276_gb300 import synth
    specs = synth.batch_specs(count=count)
    tensors = [synth.generate(s) for s in specs]
    stream = torch.cuda.current_stream()
    out = {"workload": f"c4_batch{count}_3way", "tensors": count, "nnz_total": int(sum(T.nnz for T in tensors)),
           "ranks": sorted({int(T.rank) for T in tensors})}
    cache_dir = tempfile.mkdtemp(prefix="cpapr_tune_")
    modes = ("batched", "per_tensor", "batched_tuned") if tuned else ("batched", "per_tensor")
    for mode in modes:
        extra = {}
        t0 = time.perf_counter()
        if mode == "batched_tuned":
            extra = {"autotune": 1, "tune_cache": os.path.join(cache_dir, "tune.txt")}
        ts = [cp.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, stream=stream.cuda_stream, **extra)
              for T in tensors]
        create_s = time.perf_counter() - t0
        for T, t in zip(tensors, ts):
            t.set_model(np.ones(T.rank), synth.random_factors(T.dims, T.rank, T.seed + 3))

        def step():
            if mode != "per_tensor":
                res = cp.cpapr_batch_mu_solve([t.ctx for t in ts], TOL, 1, MAX_INNER)
            else:
                res = [t.mu_solve(TOL, 1, MAX_INNER) for t in ts]
            return sum(r["total_inner"] * T.nnz for r, T in zip(res, tensors))

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        units = 0
        e0.record(stream)
        for _ in range(steps):
            units += step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[mode] = {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps}
        if mode == "batched_tuned":
            out[mode]["create_with_tuning_s"] = create_s
            with open(extra["tune_cache"]) as f:
                out[mode]["shape_classes_tuned"] = len(f.read().splitlines())
            out[mode]["tiles_mode0"] = sorted({int(t.info().tile_nnz[0]) for t in ts})
        for t in ts:
            t.close()
    out["speedup_vs_per_tensor"] = out["batched"]["value"] / out["per_tensor"]["value"]
    if tuned:
        out["tuned_vs_heuristic"] = out["batched_tuned"]["value"] / out["batched"]["value"]
    return out


KERNEL_NAMES = ("phi_tile", "pi_build", "mu_update", "normalise", "s_and_b", "loglik", "mttkrp")


def kernel_breakdown(stats, steps):
    """Device milliseconds per step of each kernel kind (library CUDA events)."""
    return {KERNEL_NAMES[k]: stats[k][1] / steps for k in range(7) if stats[k][0]}


def ncu_traffic(T, dtype, mat, info, inner_per_mode):
    """Measured DRAM bytes per Phi launch for this configuration (scaled to the
    tensor's nonzeros where the capture ran on a smaller copy), weighted by the
    launches of each mode, with its source and, where captured, the L2 bytes
    read by L1 misses per launch; (None, None, None) if not captured."""
    N = T.nmodes
    form = "materialised" if all(mat) else ("fused" if not any(mat) else "mixed")
    key = (T.name, dtype, form, tuple(info.rank_lanes)[:N], tuple(info.tile_nnz)[:N])
    if key not in NCU_TRAFFIC:
        return None, None, None
    ent = NCU_TRAFFIC[key]
    fb = 8 if dtype == "f64" else 4
    scale = T.nnz / ent["nnz"]
    per_mode = []
    for n in range(N):
        io = 2.0 * T.rank * fb * T.dims[n]
        per_mode.append((ent["bytes"][n] - io) * scale + io)
    w = [float(inner_per_mode[n]) for n in range(N)]
    tot = max(sum(w), 1.0)
    l2 = None
    if "l2_read" in ent:
        l2 = sum(w[n] * ent["l2_read"][n] * scale for n in range(N)) / tot
    return sum(w[n] * per_mode[n] for n in range(N)) / tot, ent["source"], l2


def roofline_for(T, inner_per_mode, stats, precision, peaks, cp, pi_modes=None, info=None):
    """Roofline of the Phi tile kernel from its measured average duration.
    pi_modes: per mode, whether Phi streamed materialised Khatri-Rao rows."""
    N, nnz, R = T.nmodes, T.nnz, T.rank
    fb = 8 if precision == cp.CPAPR_FP64 else 4
    mat = [bool(pi_modes and pi_modes[n] == cp.CPAPR_PI_MATERIALISED) for n in range(N)]
    traffic, traffic_src, l2_read = (ncu_traffic(T, "f64" if fb == 8 else "f32", mat, info, inner_per_mode)
                                     if info is not None else (None, None, None))
    launches, total_ms = stats[cp.K_PHI]
    byts = sum(inner_per_mode[n] * phi_bytes(T.dims, nnz, R, n, fb, fb, mat[n]) for n in range(N))
    fl = sum(inner_per_mode[n] * phi_flops(N, nnz, R, mat[n]) for n in range(N))
    # FP64: the dot runs on the FP32 pipe where a lane holds 8 or fewer ranks
    lanes = list(info.rank_lanes)[:N] if info is not None else [max(1, T.rank // 8)] * N
    rp = info.rank_padded if info is not None else max(2, 1 << (R - 1).bit_length())
    on32 = [rp // max(lanes[n], 1) <= 8 for n in range(N)]
    fl64 = sum(inner_per_mode[n] * phi_fp64_pipe_flops(N, nnz, R, mat[n], on32[n]) for n in range(N))
    gath = sum(inner_per_mode[n] * phi_gather_bytes(N, nnz, R, fb, mat[n]) for n in range(N))
    sec = total_ms / 1e3
    hbm = {"achieved": byts / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    hbm["frac"] = hbm["achieved"] / hbm["peak"]
    l2g = None
    if gath > 0:
        # gathered rows include the L1's hits; the ceiling is for rows the L2 serves, so the
        # fraction uses the L2 sectors that ncu counted for this configuration (null if not captured)
        l2g = {"gathered": gath / sec / 1e9, "l2_served": None, "peak": L2_GATHER_GBS, "unit": "GB/s",
               "frac": None}
        if l2_read is not None:
            l2g["l2_served"] = l2_read / (total_ms / max(launches, 1) / 1e3) / 1e9
            l2g["frac"] = l2g["l2_served"] / L2_GATHER_GBS
    form = "materialised Pi" if all(mat) else ("fused Pi" if not any(mat) else "mixed")
    if precision == cp.CPAPR_FP64:
        ach = fl64 / sec / 1e12
        dot32 = all(on32)
        model = ("2R" if all(mat) else "NR") if dot32 else ("4R+2" if all(mat) else "(N+2)R+2")
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic,
                "kernel": f"phi_tile_kernel<double> ({form})",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz",
                "flop_model": f"{model} FP64 FLOPs per nonzero on the FP64 pipe"
                              + (" (the dot's 2R and the max and divide run on the FP32 pipe)" if dot32 else ""),
                "paper_flop_model": {"achieved": fl / sec / 1e12, "unit": "TFLOP/s",
                                     "per_nonzero": "4R+2" if all(mat) else "(N+2)R+2"}}
    else:
        roof = {"bound": "hbm", "achieved": hbm["achieved"], "peak": hbm["peak"], "unit": "GB/s",
                "frac": hbm["frac"], "traffic": traffic, "kernel": f"phi_tile_kernel<float> ({form})",
                "peak_source": f"{peaks['source']} hbm_gbs"}
    roof["traffic_unit"] = "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    roof["traffic_source"] = traffic_src
    roof["algorithmic_bytes_per_launch"] = byts / max(sum(inner_per_mode[n] for n in range(N)), 1)
    roof["avg_launch_ms"] = total_ms / max(launches, 1)
    roof["launches"] = launches
    roof["hbm"] = hbm
    if l2g is not None:
        roof["l2_gather"] = l2g
    # the paper's word count Q = nnz(5R+2) 8-byte words per Phi (Eq. "Q"), which
    # counts every factor access whether it hits a cache or not: context only
    qb = sum(inner_per_mode[n] * nnz * (5 * R + 2) * 8.0 for n in range(N))
    roof["paper_model"] = {"achieved": qb / sec / 1e9, "unit": "GB/s", "words_per_nonzero": 5 * R + 2}
    roof["flops_tflops"] = fl / sec / 1e12
    return roof


def e2e_run(cp, torch, T, lam, fs, precision, steps, warmup):
    """Through the C ABI from pinned host buffers: create (H2D + index build),
    set_model, one outer iteration + log-likelihood, get_model (D2H), destroy."""
    stream = torch.cuda.current_stream()
    idx_p = torch.from_numpy(T.idx).pin_memory()
    val_p = torch.from_numpy(T.vals).pin_memory()
    lam_p = torch.from_numpy(lam).pin_memory()
    fs_p = [torch.from_numpy(np.ascontiguousarray(A)).pin_memory() for A in fs]
    lam_o = torch.empty(T.rank, dtype=torch.float64).pin_memory()
    fs_o = [torch.empty(A.shape, dtype=torch.float64).pin_memory() for A in fs]
    opt = cp.cpapr_default_options(precision=precision, use_graph=0, stream=stream.cuda_stream)
    rows = [idx_p[m] for m in range(T.nmodes)]
    units = 0
    launches = 0

    def step():
        nonlocal units, launches
        ctx = cp.cpapr_create(T.dims, rows, val_p, T.rank, opt)
        try:
            cp.cpapr_set_model(ctx, lam_p, fs_p)
            r = cp.cpapr_mu_solve(ctx, TOL, 1, MAX_INNER, trace=True, ll_trace=False)
            import ctypes
            arr = (ctypes.c_void_p * T.nmodes)(*[A.data_ptr() for A in fs_o])
            cp._check(cp.load().cpapr_get_model(ctx, lam_o.data_ptr(), arr), ctx)
            launches += cp.cpapr_get_info(ctx).kernel_launches
            return int(r["inner"].sum()) * T.nnz
        finally:
            cp.cpapr_destroy(ctx)

    for _ in range(warmup):
        step()
    units = 0
    launches = 0
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        units += step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h2d = T.idx.nbytes + T.vals.nbytes + lam.nbytes + sum(A.nbytes for A in fs)
    d2h = lam.nbytes + sum(A.nbytes for A in fs)
    return {"value": units / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": ms / steps, "gpu_launches_per_step": launches / max(steps, 1)}


def run_ours(args):
    import torch
    from paper_2307_03276_gb300 import build, cpapr as cp
    world, rank, local = dist_env()
    use_cuda = torch.cuda.is_available()
    if not use_cuda:
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dist = dist_init(world, use_cuda)
    build.build()
    peaks = load_peaks()
    T, lam, fs = make_workload(args.workload)
    prim = cp.CPAPR_FP64 if args.precision == "fp64" else cp.CPAPR_FP32
    other = cp.CPAPR_FP32 if prim == cp.CPAPR_FP64 else cp.CPAPR_FP64
    clocks = ClockSampler(gpu_selector())

    res = timed_solve(cp, torch, T, lam, fs, prim, args.steps, args.warmup, dist, use_cuda, clocks)
    units = float(res["inner"].sum()) * T.nnz
    units_all, sec = aggregate(dist, units, res["ms"] / 1e3, use_cuda)
    roof = roofline_for(T, res["inner"], res["stats"], prim, peaks, cp, list(res["info"].pi_mode)[:T.nmodes],
                        res["info"])
    out = {"metric": METRIC, "value": units_all / sec, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prim == cp.CPAPR_FP64 else "f32",
           "data": "synthetic (seeded Zipf/Poisson count tensor; FROSTT stand-in)",
           "config": {"workload": T.name, "dims": list(T.dims), "nnz": T.nnz, "rank": T.rank,
                      "precision": args.precision, "step": "1 outer MU iteration (all modes, <=10 inner) + loglik",
                      "kkt_tol": TOL, "max_inner": MAX_INNER, "parallelism": f"replicas x{world}",
                      "l2": f"inputs larger than L2 (mode layouts {layout_bytes(T) / 1e6:,.0f} MB > 129 MB), no flush",
                      "graph": False, "tile_nnz": list(res["info"].tile_nnz)[:T.nmodes],
                      "rank_lanes": list(res["info"].rank_lanes)[:T.nmodes]},
           "roofline": roof, "gpu_launches": int(res["launches"]), "clocks": res["clocks"],
           "inner_iterations_per_mode": res["inner"].tolist(),
           "kernel_ms_per_step": kernel_breakdown(res["stats"], args.steps)}
    kern = {}
    mt_l, mt_ms = res["mttkrp"]
    kern["mttkrp_" + args.precision] = {"nnz_per_s": T.nnz * mt_l / (mt_ms / 1e3), "avg_launch_ms": mt_ms / max(mt_l, 1)}
    if not args.no_variants:
        r2 = timed_solve(cp, torch, T, lam, fs, other, args.steps, args.warmup, dist, use_cuda)
        u2, s2 = aggregate(dist, float(r2["inner"].sum()) * T.nnz, r2["ms"] / 1e3, use_cuda)
        name = "fp32" if other == cp.CPAPR_FP32 else "fp64"
        out["variants"] = {name: {"value": u2 / s2, "unit": UNIT, "ms_per_step": s2 * 1e3 / args.steps,
                                  "dtype": "f32" if other == cp.CPAPR_FP32 else "f64",
                                  "roofline": roofline_for(T, r2["inner"], r2["stats"], other, peaks, cp,
                                                           list(r2["info"].pi_mode)[:T.nmodes], r2["info"]),
                                  "inner_iterations_per_mode": r2["inner"].tolist(),
                                  "kernel_ms_per_step": kernel_breakdown(r2["stats"], args.steps),
                                  "loglik_last": r2["last"]["loglik"]}}
        mt_l, mt_ms = r2["mttkrp"]
        kern["mttkrp_" + name] = {"nnz_per_s": T.nnz * mt_l / (mt_ms / 1e3), "avg_launch_ms": mt_ms / max(mt_l, 1)}
        if prim == cp.CPAPR_FP64 and T.nmodes >= 3:
            # the same FP64 step with the Khatri-Rao rows formed inside every Phi
            r3 = timed_solve(cp, torch, T, lam, fs, prim, args.steps, args.warmup, dist, use_cuda,
                             pi_mode=cp.CPAPR_PI_FUSED)
            u3, s3 = aggregate(dist, float(r3["inner"].sum()) * T.nnz, r3["ms"] / 1e3, use_cuda)
            out["variants"]["fp64_fused_pi"] = {
                "value": u3 / s3, "unit": UNIT, "ms_per_step": s3 * 1e3 / args.steps, "dtype": "f64",
                "roofline": roofline_for(T, r3["inner"], r3["stats"], prim, peaks, cp,
                                         list(r3["info"].pi_mode)[:T.nmodes], r3["info"]),
                "inner_iterations_per_mode": r3["inner"].tolist(),
                "kernel_ms_per_step": kernel_breakdown(r3["stats"], args.steps),
                "loglik_last": r3["last"]["loglik"]}
        for pname, prec in (("fp64", cp.CPAPR_FP64), ("fp32", cp.CPAPR_FP32)):
            b = batched_run(cp, torch, prec, args.steps, args.warmup)
            ub, sb = aggregate(dist, b["batched"]["value"] * b["batched"]["ms_per_step"] * args.steps / 1e3,
                               b["batched"]["ms_per_step"] * args.steps / 1e3, use_cuda)
            b["batched"]["value"] = ub / sb
            out["variants"]["batched_" + pname] = b
        if args.workload != "c2":
            # the 3-way 1e7-nonzero tensor, FP64 and FP32 steps
            from paper_2307_03276_gb300 import synth
            T2, lam2, fs2 = make_workload("c2")
            c2 = {"workload": T2.name, "dims": list(T2.dims), "nnz": T2.nnz, "rank": T2.rank}
            k2 = min(args.steps, 10)
            for pname, prec in (("fp64", cp.CPAPR_FP64), ("fp32", cp.CPAPR_FP32)):
                r4 = timed_solve(cp, torch, T2, lam2, fs2, prec, k2, args.warmup, dist, use_cuda)
                u4, s4 = aggregate(dist, float(r4["inner"].sum()) * T2.nnz, r4["ms"] / 1e3, use_cuda)
                c2[pname] = {"value": u4 / s4, "unit": UNIT, "steps": k2, "ms_per_step": s4 * 1e3 / k2,
                             "dtype": "f64" if prec == cp.CPAPR_FP64 else "f32",
                             "roofline": roofline_for(T2, r4["inner"], r4["stats"], prec, peaks, cp,
                                                      list(r4["info"].pi_mode)[:T2.nmodes], r4["info"]),
                             "kernel_ms_per_step": kernel_breakdown(r4["stats"], k2)}
            out["variants"]["c2"] = c2
            del T2
        if world == 1:
            # time to KKT tolerance 1e-4: the small tensor solved to the
            # tolerance, the headline tensor to a violation level FP64 and FP32
            # both reach, and the 64-tensor batch (batched vs per tensor)
            T1, lam1, fs1 = make_workload("c1")
            out["variants"]["time_to_kkt"] = {
                "c1_to_tolerance": time_to_kkt(cp, torch, T1, lam1, fs1, KKT_SMALL_MAX_OUTER, solve_to_tol=True),
                "headline_common_level": time_to_kkt(cp, torch, T, lam, fs, KKT_MAX_OUTER),
                "batch": batch_time_to_kkt(cp, torch, KKT_BATCH_MAX_OUTER)}
    out["kernels"] = kern
    if not args.no_e2e:
        e2e = e2e_run(cp, torch, T, lam, fs, prim, max(2, args.steps // 2), 1)
        ue, se = aggregate(dist, e2e["value"] * e2e["ms_per_step"] * max(2, args.steps // 2) / 1e3,
                           e2e["ms_per_step"] * max(2, args.steps // 2) / 1e3, use_cuda)
        e2e["value"] = ue / se
        out["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(T, lam, fs, seconds=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_kernel_only(args):
    """Phi^(n) for every mode, `steps` rounds: a small target for ncu captures.
    With --workload c4: `steps` batched outer iterations of the 64-tensor
    batch with plain stream launches (no graphs, so every kernel is visible
    to a launch list)."""
    import torch
    from paper_2307_03276_gb300 import build, cpapr as cp
    torch.cuda.set_device(0)
    build.build()
    prec = cp.CPAPR_FP64 if args.precision == "fp64" else cp.CPAPR_FP32
    if args.workload == "c4":
        from paper_2307_03276_gb300 import synth
        tensors = [synth.generate(sp) for sp in synth.batch_specs(count=64)]
        ts = [cp.Tensor(T.dims, T.idx, T.vals, T.rank, precision=prec, use_graph=0) for T in tensors]
        for T, t in zip(tensors, ts):
            t.set_model(np.ones(T.rank), synth.random_factors(T.dims, T.rank, T.seed + 3))
        inner = 0
        for _ in range(args.steps):
            inner += sum(r["total_inner"] for r in cp.cpapr_batch_mu_solve([t.ctx for t in ts], TOL, 1, MAX_INNER))
        for t in ts:
            t.close()
        print(json.dumps({"kernel": "batch", "precision": args.precision, "workload": "c4_batch64_3way",
                          "outer_iterations": args.steps, "inner_iterations": inner}))
        return
    if args.nnz or args.rank:
        # the same workload with fewer nonzeros (same dims and distributions)
        # and/or another rank: a capture target of a few GB for ncu
        from paper_2307_03276_gb300 import synth
        base = synth.SPECS[args.workload]
        spec = synth.scaled(base, args.nnz or base.nnz, rank=args.rank or None)
        T = synth.generate(spec)
        lam, fs = np.ones(T.rank), synth.random_factors(T.dims, T.rank, spec.seed + 17)
    else:
        T, lam, fs = make_workload(args.workload)
    with cp.Tensor(T.dims, T.idx, T.vals, T.rank, precision=prec, profile=1, use_graph=0) as t:
        t.set_model(lam, fs)
        for _ in range(args.steps):
            for n in range(T.nmodes):
                t.phi(n)
        launches, ms = t.kernel_stats(cp.K_PHI)
        info = t.info()
    print(json.dumps({"kernel": "phi_tile_kernel", "precision": args.precision, "workload": T.name, "rank": T.rank,
                      "nnz": T.nnz, "pi_mode": list(info.pi_mode)[:T.nmodes],
                      "launches": launches, "avg_ms": ms / max(launches, 1),
                      "tile_nnz": list(info.tile_nnz)[:T.nmodes], "rank_lanes": list(info.rank_lanes)[:T.nmodes]}))


def run_r_sweep(args):
    """Phi^(n) and MTTKRP over R in {8, 16, 32, 64} on one tensor (default: the
    5-way 5e4 x 5e4 x 5e3 x 1e3 x 24 workload, 1e8 nonzeros), each rank with the
    autotuner choosing lanes, tile, reduction and Pi form per mode; one JSON
    line with nonzeros/s and the roofline fractions per rank and precision."""
    import torch
    from paper_2307_03276_gb300 import build, cpapr as cp, synth
    torch.cuda.set_device(0)
    build.build()
    peaks = load_peaks()
    spec = synth.SPECS[args.workload]
    T = synth.generate(spec)
    N = T.nmodes
    ranks = [int(r) for r in args.ranks.split(",")]
    precs = [cp.CPAPR_FP64, cp.CPAPR_FP32] if args.precision == "both" else (
        [cp.CPAPR_FP64] if args.precision == "fp64" else [cp.CPAPR_FP32])
    out = {"sweep": "rank", "workload": T.name, "dims": list(T.dims), "nnz": T.nnz, "results": []}
    for R in ranks:
        fs = synth.random_factors(T.dims, R, spec.seed + 17)
        lam = np.ones(R)
        for prec in precs:
            fb = 8 if prec == cp.CPAPR_FP64 else 4
            with cp.Tensor(T.dims, T.idx, T.vals, R, precision=prec, profile=1, use_graph=0, autotune=1) as t:
                info = t.info()
                t.set_model(lam, fs)
                for n in range(N):
                    t.phi(n)
                for k in range(7):
                    t.kernel_stats(k, reset=True)
                reps = max(1, args.steps)
                for _ in range(reps):
                    for n in range(N):
                        t.phi(n)
                for n in range(N):
                    t.mttkrp(n)
                for _ in range(reps):
                    for n in range(N):
                        t.mttkrp(n)
                pl, pms = t.kernel_stats(cp.K_PHI)
                bl, bms = t.kernel_stats(cp.K_PI)
                ml, mms = t.kernel_stats(cp.K_MTTKRP)
                pim = list(info.pi_mode)[:N]
            mat = [m == cp.CPAPR_PI_MATERIALISED for m in pim]
            per = pms / max(pl, 1)
            byts = sum(phi_bytes(T.dims, T.nnz, R, n, fb, fb, mat[n]) for n in range(N)) / N
            rp = int(info.rank_padded)
            fl = sum(phi_fp64_pipe_flops(N, T.nnz, R, mat[n], rp // max(int(info.rank_lanes[n]), 1) <= 8)
                     for n in range(N)) / N
            mb = sum(phi_bytes(T.dims, T.nnz, R, n, fb, fb, False) for n in range(N)) / N
            mper = mms / max(ml, 1)
            row = {"rank": R, "dtype": "f64" if prec == cp.CPAPR_FP64 else "f32",
                   "rank_lanes": list(info.rank_lanes)[:N], "tile_nnz": list(info.tile_nnz)[:N],
                   "reduction": list(info.reduction)[:N], "pi_mode": pim,
                   "phi_ms_per_launch": per, "phi_nnz_per_s": T.nnz / (per / 1e3),
                   "phi_hbm_frac": byts / (per / 1e3) / 1e9 / peaks["hbm_gbs"],
                   "phi_fp64_frac": (fl / (per / 1e3) / 1e12 / FP64_PEAK_TFLOPS) if fb == 8 else None,
                   "pi_build_ms_per_launch": (bms / bl) if bl else None,
                   "mttkrp_ms_per_launch": mper, "mttkrp_nnz_per_s": T.nnz / (mper / 1e3),
                   "mttkrp_hbm_frac": mb / (mper / 1e3) / 1e9 / peaks["hbm_gbs"]}
            out["results"].append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    out["peaks"] = {"hbm_gbs": peaks["hbm_gbs"], "source": peaks["source"], "fp64_tflops": FP64_PEAK_TFLOPS}
    print(json.dumps(out), flush=True)


PPA_WINDOW = 16


def ppa_phi_ms(cp, T, lam, fs, precision, pi_mode, reduction, modes, reps):
    """Average Phi (and Pi build) launch time over `modes`, heuristic tiling."""
    with cp.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, profile=1, use_graph=0,
                   pi_mode=pi_mode, reduction=reduction) as t:
        t.set_model(lam, fs)
        for n in modes:
            t.phi(n)
        t.kernel_stats(cp.K_PHI, reset=True)
        t.kernel_stats(cp.K_PI, reset=True)
        for _ in range(reps):
            for n in modes:
                t.phi(n)
        pl, pms = t.kernel_stats(cp.K_PHI)
        bl, bms = t.kernel_stats(cp.K_PI)
        info = t.info()
    return {"phi_ms": pms / max(pl, 1), "pi_build_ms": (bms / bl) if bl else 0.0,
            "tile_nnz": list(info.tile_nnz)[:T.nmodes], "rank_lanes": list(info.rank_lanes)[:T.nmodes]}


def run_ppa(args):
    """Pressure-point probes after the paper's performance analysis (Section
    "Pressure Point Analysis"), on GB300.

    Data reuse: Phi^(0) of a 3-way 1e5 x 1e5 x 1e3 tensor with 1e7 nonzeros
    and R = 32 whose mode-0 rows are uniform, once with modes 1 and 2 uniform
    over their full range and once with them confined to their first
    PPA_WINDOW rows (every factor row gathered stays cache-resident; the
    tensor, its streams and B/Phi keep their sizes).  The paper hard-codes
    the gathered row instead; here the input carries the access pattern, so
    the kernels run unchanged and their results stay exact.

    Atomics: the paper swaps the atomic row update for an unsynchronised one
    (wrong results, timing only).  The segmented reduction here is the
    non-atomic form that stays correct, so the probe times the 3-way Zipf
    workload with reduction = atomic against reduction = segmented."""
    import torch
    from paper_2307_03276_gb300 import build, cpapr as cp, synth
    torch.cuda.set_device(0)
    build.build()
    reps = max(1, args.steps)
    c2 = synth.C2
    out = {"probe": "pressure_points", "reuse": [], "atomic": []}
    layouts = {"full": (("uniform",),) * 3,
               "window": (("uniform",), ("window", PPA_WINDOW), ("window", PPA_WINDOW))}
    forms = [(cp.CPAPR_FP64, cp.CPAPR_PI_FUSED), (cp.CPAPR_FP64, cp.CPAPR_PI_MATERIALISED),
             (cp.CPAPR_FP32, cp.CPAPR_PI_FUSED), (cp.CPAPR_FP32, cp.CPAPR_PI_MATERIALISED)]
    for name, modes in layouts.items():
        spec = synth.TensorSpec(c2.dims, c2.nnz, c2.rank, modes, c2.values, 1102,
                                f"ppa_3way_1e5x1e5x1e3_1e7_r32_{name}")
        T = synth.generate(spec)
        fs = synth.random_factors(T.dims, T.rank, 5)
        lam = np.ones(T.rank)
        for prec, pim in forms:
            r = ppa_phi_ms(cp, T, lam, fs, prec, pim, cp.CPAPR_REDUCE_SEGMENTED, [0], reps)
            r.update({"tensor": name, "window_rows": PPA_WINDOW if name == "window" else None,
                      "dtype": "f64" if prec == cp.CPAPR_FP64 else "f32",
                      "pi": "fused" if pim == cp.CPAPR_PI_FUSED else "materialised", "mode": 0})
            out["reuse"].append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
        del T
    T, lam, fs = make_workload("c2")
    for prec, pim in [(cp.CPAPR_FP64, cp.CPAPR_PI_MATERIALISED), (cp.CPAPR_FP32, cp.CPAPR_PI_FUSED)]:
        for red, rname in [(cp.CPAPR_REDUCE_SEGMENTED, "segmented"), (cp.CPAPR_REDUCE_ATOMIC, "atomic")]:
            r = ppa_phi_ms(cp, T, lam, fs, prec, pim, red, list(range(T.nmodes)), reps)
            r.update({"workload": T.name, "dtype": "f64" if prec == cp.CPAPR_FP64 else "f32",
                      "pi": "fused" if pim == cp.CPAPR_PI_FUSED else "materialised", "reduction": rname,
                      "phi_nnz_per_s": T.nnz / (r["phi_ms"] / 1e3)})
            out["atomic"].append(r)
            print(json.dumps(r), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The FP64 oracle on all the host's cores (each thread owns a range of
    Phi rows), on bounded samples of the same workload; the one-core figure
    rides along."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    T, lam, fs = make_workload(args.workload)
    import oracle
    oracle.build()
    cores = host_cores()
    S = min(args.ref_sample * max(1, min(cores, 8)), T.nnz)
    idx = np.ascontiguousarray(T.idx[:, :S])
    vals = np.ascontiguousarray(T.vals[:S])
    for k in range(args.warmup):
        n = k % T.nmodes
        oracle.phi_threads(T.dims, idx, vals, fs, fs[n] * lam[None, :], n, cores)
    t0 = time.perf_counter()
    for k in range(args.steps):
        n = k % T.nmodes
        oracle.phi_threads(T.dims, idx, vals, fs, fs[n] * lam[None, :], n, cores)
    dt = time.perf_counter() - t0
    value = S * args.steps / dt
    v1, k1, d1 = _oracle_phi_rate(T, lam, fs, min(args.ref_sample, T.nnz), 3.0, 1)
    sample = (f"each step: Phi^(n) (n cycling) over the first {S:,} of {T.nnz:,} nonzeros (random draw order) "
              f"of the same tensor, FP64, {cores} threads")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Zipf/Poisson count tensor; FROSTT stand-in)",
           "config": {"workload": T.name, "dims": list(T.dims), "nnz": T.nnz, "rank": T.rank, "precision": "fp64",
                      "step": "Phi^(n) over a bounded sample", "parallelism": f"host, {cores} threads"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                              "sample": f"Phi^(n) over the first {min(args.ref_sample, T.nnz):,} "
                                                        f"nonzeros, {k1} evaluations in {d1:.1f} s"}},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "c5"],
                    help="c4 (the 64-tensor batch) applies to --time-to-kkt and --kernel-only only")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "both"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-sample", type=int, default=1_000_000)
    ap.add_argument("--r-sweep", action="store_true",
                    help="Phi and MTTKRP over --ranks on --workload (default c5) with autotuned choices")
    ap.add_argument("--ranks", default="8,16,32,64")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only run Phi^(n) for every mode --steps times (profiling target)")
    ap.add_argument("--nnz", type=int, default=0,
                    help="with --kernel-only: the workload scaled to this many nonzeros (same dims)")
    ap.add_argument("--rank", type=int, default=0, help="with --kernel-only: the workload at this rank")
    ap.add_argument("--time-to-kkt", action="store_true",
                    help="full solve at KKT tolerance 1e-4 (FP64 and FP32) on --workload")
    ap.add_argument("--max-outer", type=int, default=KKT_MAX_OUTER)
    ap.add_argument("--ppa", action="store_true",
                    help="pressure-point probes: factor-row reuse and atomic vs segmented reduction")
    args = ap.parse_args(argv)
    if args.ppa:
        run_ppa(args)
        return
    if args.time_to_kkt:
        run_time_to_kkt(args)
        return
    if args.workload == "c4" and not args.kernel_only:
        raise SystemExit("--workload c4 (the 64-tensor batch) applies to --time-to-kkt and --kernel-only only")
    if args.r_sweep:
        if "--workload" not in (argv if argv is not None else sys.argv):
            args.workload = "c5"
        if "--precision" not in (argv if argv is not None else sys.argv):
            args.precision = "both"
        run_r_sweep(args)
        return
    if args.precision == "both":
        raise SystemExit("--precision both applies to --r-sweep only")
    if args.kernel_only:
        run_kernel_only(args)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
