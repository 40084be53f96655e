"""Host logic of bench.py: byte/FLOP models and the multi-rank aggregation
(world size 2 over gloo on CPU, the same code path NCCL takes on GPUs)."""
import os
import socket

import numpy as np
import pytest

import bench


def test_byte_model_matches_hand_count():
    # 4-way 200,000 x 200,000 x 10,000 x 365, 5e7 nonzeros, R = 16, FP64, mode 0:
    # 5e7*(12+8) + 4*(2e5+1) + 8*16*(2e5+1e4+365 + 2*2e5) = 1.0789 GB
    b = bench.phi_bytes((200_000, 200_000, 10_000, 365), 50_000_000, 16, 0, 8, 8)
    assert b == 50_000_000 * 20 + 4 * 200_001 + 8 * 16 * (210_365 + 400_000)
    assert abs(b / 1e9 - 1.0789) < 1e-3
    assert bench.phi_flops(4, 10, 16) == 10 * (6 * 16 + 2)
    assert bench.phi_gather_bytes(3, 10, 32, 4) == 10 * 2 * 32 * 4


def test_byte_model_materialised_pi():
    # 3-way 1e5 x 1e5 x 1e3, 1e7 nonzeros, R = 32, FP64, mode 0, Pi streamed:
    # 1e7 * (8 + 32*8) + 4*(1e5 + 1) + 8*32*2*1e5 = 2.6916 GB; FLOPs 4R+2 per nonzero
    b = bench.phi_bytes((100_000, 100_000, 1_000), 10_000_000, 32, 0, 8, 8, materialised=True)
    assert b == 10_000_000 * (8 + 256) + 4 * 100_001 + 8 * 32 * 2 * 100_000
    assert abs(b / 1e9 - 2.6916) < 1e-4
    assert bench.phi_flops(3, 10, 32, materialised=True) == 10 * (4 * 32 + 2)
    assert bench.phi_gather_bytes(3, 10, 32, 8, materialised=True) == 0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    d = bench.dist_init(world, use_cuda=False)
    bench.barrier(d, use_cuda=False)
    u, s = bench.aggregate(d, units=100.0 * (rank + 1), seconds=0.5 + rank, use_cuda=False)
    q.put((rank, u, s))
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, u, s in got:
        assert u == 300.0 and s == 1.5


def test_window_mode_distribution():
    """A ("window", W) mode draws uniformly from the first W rows of a mode
    that keeps its full size (the data-reuse pressure-point input)."""
    from paper_2307_03276_gb300 import synth
    spec = synth.TensorSpec((500, 400, 300), 20_000, 4, (("uniform",), ("window", 8), ("window", 500)),
                            ("poisson1", 1.0), 7, "w")
    T = synth.generate(spec)
    assert T.dims == (500, 400, 300) and T.nnz == 20_000
    assert T.idx[1].min() == 0 and T.idx[1].max() == 7
    assert T.idx[2].max() == 299          # a window wider than the mode is the whole mode
    counts = np.bincount(T.idx[1], minlength=8)
    assert counts.min() > 0.8 * T.nnz / 8  # near-uniform over the window
    assert len({tuple(c) for c in T.idx.T}) == T.nnz


def test_roofline_line_is_strict_json():
    """The roofline object of a measured FP64 step: the FLOP model of the Pi
    form that ran, the measured traffic for a captured configuration, the
    paper's word count as context, and nothing a strict JSON parser rejects."""
    import json

    class CP:
        CPAPR_FP64, CPAPR_FP32, CPAPR_PI_MATERIALISED, K_PHI = 0, 1, 2, 0

    class Info:
        rank_lanes = (4, 4, 4)
        tile_nnz = (1024, 1024, 1024)
        rank_padded = 32

    class T:
        nmodes, nnz, rank = 3, 10_000_000, 32
        dims = (100_000, 100_000, 1_000)
        name = "c2_3way_1e5x1e5x1e3_1e7_r32"

    inner = np.array([10, 10, 10])
    r = bench.roofline_for(T, inner, {0: (30, 43.6)}, 0, {"hbm_gbs": 6682.5, "source": "measured"}, CP,
                           [2, 2, 2], Info())
    json.dumps(r, allow_nan=False)
    # 8 ranks per lane: the divisor runs on the FP32 pipe, the scale-add's 2R FP64 FLOPs per nonzero remain
    assert r["bound"] == "alu" and r["flop_model"].startswith("2R FP64 FLOPs per nonzero on the FP64 pipe")
    flops = 30 * 1e7 * (2 * 32)
    assert abs(r["achieved"] - flops / 43.6e-3 / 1e12) < 1e-9
    assert abs(r["paper_flop_model"]["achieved"] - 30 * 1e7 * (4 * 32 + 2) / 43.6e-3 / 1e12) < 1e-9
    assert r["traffic"] is not None and 2.6e9 < r["traffic"] < 2.8e9
    assert r["paper_model"]["words_per_nonzero"] == 162
    assert abs(r["paper_model"]["achieved"] - 30 * 1e7 * 162 * 8 / 43.6e-3 / 1e9) < 1e-6


def test_batch_workload_specs():
    """The 64-tensor batch: 3-way, dims within [50,50,50]-[20000,20000,500],
    nnz within [1e3, 1e6] and at most 10% of the coordinate space, R from
    {8, 16, 32}, every tensor seeded differently; the same specs on every call."""
    from paper_2307_03276_gb300 import synth
    specs = synth.batch_specs()
    assert len(specs) == 64 and specs == synth.batch_specs()
    assert len({s.seed for s in specs}) == 64
    for s in specs:
        assert len(s.dims) == 3
        assert all(lo <= d <= hi for d, lo, hi in zip(s.dims, (50, 50, 50), (20_000, 20_000, 500)))
        assert s.nnz <= 0.1 * s.dims[0] * s.dims[1] * s.dims[2] + 1
        assert s.nnz <= 1_000_000 and (s.nnz >= 1_000 or s.nnz >= int(0.1 * s.dims[0] * s.dims[1] * s.dims[2]))
        assert s.rank in (8, 16, 32)
    assert {s.rank for s in specs} == {8, 16, 32}
