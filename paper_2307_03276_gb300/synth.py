"""Seeded synthetic sparse count tensors and initial models.

This module only draws inputs: coordinates, counts and U(0,1) factor
entries.  It holds none of the CP-APR arithmetic, so both the CUDA path and
the CPU oracle can consume its output without sharing any method code.

Random numbers come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
i-th draw of a stream with base ``b`` is ``mix64(b + (i + 1) * GOLDEN)``,
which is exactly the i-th output of a SplitMix64 generator started at state
``b``.  Being counter-based it vectorises in numpy and gives identical bits on
every machine and numpy version.

The workloads stand in for the FROSTT tensors the paper measures (Table
"Tensors used for evaluation"): 3- to 5-way count tensors with millions of
nonzeros and power-law (Zipf) mode distributions.  Those datasets are not
available here, so seeded stand-ins of that shape are drawn instead.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
import math
import os

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (uint64 in, uint64 out, wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_base(seed: int, stream: int) -> np.uint64:
    """Base state of sub-stream ``stream`` of seed ``seed``."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed % (1 << 64)) + np.uint64(stream + 1) * GOLDEN
    return np.uint64(mix64(np.array([s], dtype=np.uint64))[0])


def raw64(base: np.uint64, start: int, n: int) -> np.ndarray:
    """Draws ``start .. start+n-1`` of the SplitMix64 stream at ``base``."""
    ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(base + ctr * GOLDEN)


def uniform01(base: np.uint64, start: int, n: int) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each draw times 2^-53."""
    return (raw64(base, start, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# distributions (inverse-CDF tables; deterministic)
# ---------------------------------------------------------------------------

def _inverse_cdf(cdf: np.ndarray, u: np.ndarray) -> np.ndarray:
    k = np.searchsorted(cdf, u, side="right")
    return np.minimum(k, len(cdf) - 1).astype(np.int64)


def zipf_table(n: int, alpha: float) -> np.ndarray:
    w = np.arange(1, n + 1, dtype=np.float64) ** (-alpha)
    c = np.cumsum(w)
    return c / c[-1]


def alias_table(weights: np.ndarray):
    """Walker's alias table built with Vose's linear algorithm (M. D. Vose,
    IEEE Trans. Softw. Eng. 17(9), 1991): returns (prob, alias) such that
    drawing k uniform on [0, n) and keeping k with probability prob[k], else
    taking alias[k], samples index i with probability weights[i] / sum."""
    n = weights.size
    p = (weights / weights.sum() * n).tolist()
    prob = [1.0] * n
    alias = list(range(n))
    small = [i for i in range(n) if p[i] < 1.0]
    large = [i for i in range(n) if p[i] >= 1.0]
    while small and large:
        s = small.pop()
        g = large.pop()
        prob[s] = p[s]
        alias[s] = g
        p[g] = (p[g] + p[s]) - 1.0
        (small if p[g] < 1.0 else large).append(g)
    return np.array(prob), np.array(alias, dtype=np.int64)


def _alias_draw(prob: np.ndarray, alias: np.ndarray, u: np.ndarray) -> np.ndarray:
    x = u * prob.size
    k = np.minimum(x.astype(np.int64), prob.size - 1)
    return np.where((x - k) < prob[k], k, alias[k])


def poisson_table(mu: float) -> np.ndarray:
    pmf = [math.exp(-mu)]
    k = 0
    while True:
        k += 1
        pmf.append(pmf[-1] * mu / k)
        if k > mu and pmf[-1] < 1e-18:
            break
    c = np.cumsum(np.array(pmf))
    return c / c[-1]


def geometric_table(p: float, kmax: int = 64) -> np.ndarray:
    k = np.arange(kmax, dtype=np.float64)
    c = np.cumsum(p * (1.0 - p) ** k)
    return c / c[-1]


# ---------------------------------------------------------------------------
# workload specs
# ---------------------------------------------------------------------------

@dataclass
class TensorSpec:
    """Shape and statistics of one synthetic count tensor."""
    dims: tuple
    nnz: int
    rank: int
    modes: tuple            # per mode: ("zipf", alpha), ("uniform",) or ("window", W)
    values: tuple           # ("poisson1", mu) -> Poisson(mu)+1, ("geometric", p) -> {1,2,..}
    seed: int
    name: str = ""


@dataclass
class SparseTensor:
    dims: tuple
    idx: np.ndarray         # int64 [N, nnz], 0-based coordinates, unsorted
    vals: np.ndarray        # float64 [nnz]
    rank: int
    seed: int
    name: str = ""
    spec: TensorSpec | None = field(default=None, repr=False)

    @property
    def nmodes(self) -> int:
        return len(self.dims)

    @property
    def nnz(self) -> int:
        return int(self.vals.shape[0])


# The five workloads: a small one the oracle solves in seconds, three large
# single tensors (3-, 4- and 5-way) and a batch of 64 small uneven tensors.
C1 = TensorSpec((100, 80, 60), 10_000, 10, (("uniform",),) * 3, ("poisson1", 1.0), 1001, "c1_3way_100x80x60_1e4_r10")
C2 = TensorSpec((100_000, 100_000, 1_000), 10_000_000, 32, (("zipf", 1.2),) * 3, ("poisson1", 2.0), 1002,
                "c2_3way_1e5x1e5x1e3_1e7_r32")
C3 = TensorSpec((200_000, 200_000, 10_000, 365), 50_000_000, 16,
                (("zipf", 1.1), ("zipf", 1.1), ("uniform",), ("uniform",)), ("geometric", 0.5), 1003,
                "c3_4way_2e5x2e5x1e4x365_5e7_r16")
C5 = TensorSpec((50_000, 50_000, 5_000, 1_000, 24), 100_000_000, 64, (("zipf", 1.3),) * 5, ("poisson1", 1.0), 1005,
                "c5_5way_5e4x5e4x5e3x1e3x24_1e8_r64")
SPECS = {"c1": C1, "c2": C2, "c3": C3, "c5": C5}


def scaled(spec: TensorSpec, nnz: int, dims: tuple | None = None, rank: int | None = None,
           seed: int | None = None) -> TensorSpec:
    """The same statistics at a smaller size (for oracle-sized parity cases)."""
    return TensorSpec(tuple(dims) if dims is not None else spec.dims, int(nnz),
                      rank if rank is not None else spec.rank, spec.modes, spec.values,
                      seed if seed is not None else spec.seed,
                      f"{spec.name}@nnz{nnz}")


def _draw_mode(spec: TensorSpec, m: int, base: np.uint64, start: int, n: int, cache: dict) -> np.ndarray:
    kind = spec.modes[m]
    dim = spec.dims[m]
    u = uniform01(base, start, n)
    if kind[0] == "uniform":
        return np.minimum((u * dim).astype(np.int64), dim - 1)
    if kind[0] == "window":
        # uniform over the first W rows of a mode that keeps its full size:
        # the factor rows read through this mode stay cache-resident (the
        # "data reuse" pressure point of the paper's performance analysis)
        w = min(int(kind[1]), dim)
        return np.minimum((u * w).astype(np.int64), w - 1)
    if kind[0] == "zipf":
        # P(k) proportional to (k + 1)^-alpha, sampled with an alias table
        key = ("zipf", m)
        if key not in cache:
            w = np.arange(1, dim + 1, dtype=np.float64) ** (-kind[1])
            prob, alias = alias_table(w)
            # seeded relabelling so that heavy rows are scattered over the mode
            relabel = np.argsort(uniform01(stream_base(spec.seed, 100 + m), 0, dim), kind="stable")
            cache[key] = (prob, alias, relabel.astype(np.int64))
        prob, alias, relabel = cache[key]
        return relabel[_alias_draw(prob, alias, u)]
    raise ValueError(f"unknown mode distribution {kind}")


def _chunked(fn, n: int, chunk: int = 1 << 22) -> None:
    """Runs fn(lo, hi) over [0, n) in chunks on a thread pool (numpy releases
    the GIL); the result does not depend on the chunking."""
    bounds = [(lo, min(lo + chunk, n)) for lo in range(0, n, chunk)]
    if len(bounds) <= 1:
        for lo, hi in bounds:
            fn(lo, hi)
        return
    workers = max(1, min(len(bounds), os.cpu_count() or 1, 16))
    with ThreadPoolExecutor(workers) as ex:
        for f in [ex.submit(fn, lo, hi) for lo, hi in bounds]:
            f.result()


def generate(spec: TensorSpec) -> SparseTensor:
    """Draws exactly ``spec.nnz`` distinct coordinates and their counts."""
    N = len(spec.dims)
    total = 1
    for d in spec.dims:
        total *= int(d)
    if total >= 2 ** 62:
        raise ValueError("coordinate space too large for 63-bit linear keys")
    if spec.nnz > total:
        raise ValueError("more nonzeros than coordinates")
    strides = [1] * N
    for m in range(N - 2, -1, -1):
        strides[m] = strides[m + 1] * int(spec.dims[m + 1])
    bases = [stream_base(spec.seed, m) for m in range(N)]
    cache: dict = {}
    # Keep the first spec.nnz distinct coordinates in draw order.  Each round
    # draws a batch, keeps its first occurrences that are not yet known, and
    # sizes the next batch from the shortfall.
    known = np.empty(0, dtype=np.int64)   # sorted distinct keys so far
    chosen: list = []
    count = 0
    drawn = 0
    batch = int(spec.nnz * 1.15) + 64
    for m in range(N):  # build the per-mode tables once, before the threads use them
        _draw_mode(spec, m, bases[m], 0, 1, cache)
    for _ in range(64):
        lin = np.empty(batch, dtype=np.int64)

        def fill(lo, hi, start=drawn, out=lin):
            acc = np.zeros(hi - lo, dtype=np.int64)
            for m in range(N):
                acc += _draw_mode(spec, m, bases[m], start + lo, hi - lo, cache) * strides[m]
            out[lo:hi] = acc

        _chunked(fill, batch)
        drawn += batch
        # first occurrence of each distinct key: smallest draw position per key
        order = np.argsort(lin)
        srt = lin[order]
        head = np.ones(srt.size, dtype=bool)
        head[1:] = srt[1:] != srt[:-1]
        firstpos = np.minimum.reduceat(order, np.flatnonzero(head))
        cand = lin[np.sort(firstpos)]
        if known.size:
            pos = np.minimum(np.searchsorted(known, cand), known.size - 1)
            cand = cand[known[pos] != cand]
        take = cand[:spec.nnz - count]
        chosen.append(take)
        count += take.size
        if count >= spec.nnz:
            break
        known = np.sort(np.concatenate([known, cand]), kind="stable")
        batch = int((spec.nnz - count) * 3) + 1024
    else:
        raise RuntimeError("could not draw enough distinct coordinates")
    lin = np.concatenate(chosen) if len(chosen) > 1 else chosen[0]
    idx = np.empty((N, lin.size), dtype=np.int64)
    rem = lin.copy()
    for m in range(N):
        idx[m] = rem // strides[m]
        rem -= idx[m] * strides[m]
    vb = stream_base(spec.seed, 50)
    u = uniform01(vb, 0, lin.size)
    if spec.values[0] == "poisson1":
        vals = (_inverse_cdf(poisson_table(spec.values[1]), u) + 1).astype(np.float64)
    elif spec.values[0] == "geometric":
        vals = (_inverse_cdf(geometric_table(spec.values[1]), u) + 1).astype(np.float64)
    else:
        raise ValueError(f"unknown value distribution {spec.values}")
    return SparseTensor(tuple(int(d) for d in spec.dims), idx, vals, spec.rank, spec.seed, spec.name, spec)


def random_factors(dims, rank: int, seed: int) -> list:
    """U(0,1) factor matrices, row-major I_m x R, one sub-stream per mode."""
    out = []
    for m, d in enumerate(dims):
        b = stream_base(seed, 200 + m)
        out.append(uniform01(b, 0, int(d) * rank).reshape(int(d), rank))
    return out


def random_tensor(dims, nnz: int, rank: int, seed: int, values=("poisson1", 1.0), modes=None) -> SparseTensor:
    """Small uniform (or given-distribution) tensor for tests."""
    if modes is None:
        modes = (("uniform",),) * len(dims)
    return generate(TensorSpec(tuple(dims), nnz, rank, tuple(modes), values, seed, f"rand{tuple(dims)}x{nnz}"))


# ---------------------------------------------------------------------------
# batch workload: 64 uneven 3-way tensors
# ---------------------------------------------------------------------------

def batch_specs(count: int = 64, seed: int = 1004, nnz_range=(1e3, 1e6),
                dim_lo=(50, 50, 50), dim_hi=(20_000, 20_000, 500), ranks=(8, 16, 32)) -> list:
    """Per-tensor specs: log-uniform dims and nnz, Zipf(1.2) modes, Poisson(1)+1 counts.
    nnz is capped at 10% of the coordinate space: Zipf-distributed coordinates
    cannot practically fill a larger share of a small space."""
    b = stream_base(seed, 0)
    specs = []
    for t in range(count):
        u = uniform01(b, 8 * t, 8)
        dims = tuple(int(round(math.exp(math.log(lo) + u[m] * (math.log(hi) - math.log(lo)))))
                     for m, (lo, hi) in enumerate(zip(dim_lo, dim_hi)))
        cap = 0.1 * dims[0] * dims[1] * dims[2]
        nnz = int(round(math.exp(math.log(nnz_range[0]) + u[3] * (math.log(nnz_range[1]) - math.log(nnz_range[0])))))
        nnz = int(min(nnz, cap))
        rank = ranks[min(int(u[4] * len(ranks)), len(ranks) - 1)]
        specs.append(TensorSpec(dims, nnz, rank, (("zipf", 1.2),) * 3, ("poisson1", 1.0),
                                seed * 1000 + t, f"c4_batch{t}"))
    return specs
