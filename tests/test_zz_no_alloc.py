"""cpapr_phi_noalloc against cpapr_phi.

cpapr_phi_noalloc is for callers that cannot let the library allocate device
memory during a call -- their GPU memory belongs to another allocator, or the
call sits in a loop that must not block on cudaMalloc.  Its Phi kernel takes
its scratch (per-tile partial rows) from a fixed array the library keeps on
every GPU instead of a buffer the context allocated.  These tests call it
through the C ABI twice in a row with device buffers and compare each result
with the regular entry point, within the tolerances the parity tests use; they
check that neither the context's device memory nor torch's reserved memory
grows across the calls, and that a staging wait that gives up is reported
and leaves the next call correct.
"""
import numpy as np
import pytest
import torch

from paper_2307_03276_gb300 import cpapr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2307_03276_gb300 import build
    build.build()


def max_rel(got, want):
    nz = want != 0
    err = np.zeros_like(want)
    err[nz] = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
    err[~nz] = np.abs(got[~nz]) > 0
    return float(err.max())


@pytest.mark.parametrize("precision,tol,reduction", [
    (cpapr.CPAPR_FP64, 1e-12, cpapr.CPAPR_REDUCE_AUTO),
    (cpapr.CPAPR_FP32, 1e-5, cpapr.CPAPR_REDUCE_AUTO),
    # a context whose modes use atomic adds: the allocation-free call still
    # takes the segmented reduction through the fixed scratch
    (cpapr.CPAPR_FP64, 1e-12, cpapr.CPAPR_REDUCE_ATOMIC),
])
def test_noalloc_matches_phi_on_two_calls(precision, tol, reduction):
    T = synth.generate(synth.scaled(synth.C3, 300_000, dims=(40_000, 40_000, 10_000, 365)))
    fs = synth.random_factors(T.dims, T.rank, 31)
    lam = 0.5 + synth.uniform01(synth.stream_base(31, 1), 0, T.rank)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, tile_nnz=512, reduction=reduction) as t:
        t.set_model(lam, fs)
        assert max(t.info().nsplit[:T.nmodes]) > 0  # rows cut across tiles: the scratch is used
        if reduction == cpapr.CPAPR_REDUCE_ATOMIC:
            assert all(r == cpapr.CPAPR_REDUCE_ATOMIC for r in t.info().reduction[:T.nmodes])
        wants = [t.phi(n) for n in range(T.nmodes)]
        outs = [torch.full((T.dims[n], T.rank), float("nan"), dtype=torch.float64, device="cuda")
                for n in range(T.nmodes)]
        B = fs[1] * 1.5
        want_b = t.phi(1, B=B)
        Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        out_b = torch.zeros((T.dims[1], T.rank), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        held = t.info().device_bytes
        reserved = torch.cuda.memory_reserved()
        for _ in range(2):
            for n in range(T.nmodes):
                outs[n].fill_(float("nan"))
                cpapr.cpapr_phi_noalloc(t.ctx, n, outs[n])
                torch.cuda.synchronize()
                assert max_rel(outs[n].cpu().numpy(), wants[n]) <= tol, (n,)
            # explicit device B
            out_b.zero_()
            cpapr.cpapr_phi_noalloc(t.ctx, 1, out_b, B=Bd)
            torch.cuda.synchronize()
            assert max_rel(out_b.cpu().numpy(), want_b) <= tol
        assert t.info().device_bytes == held
        assert torch.cuda.memory_reserved() == reserved


def test_noalloc_timeout_is_reported_and_next_call_is_correct(monkeypatch):
    """With the host-side injection every tile's staging barrier expects 16
    bytes more than its copies bring, so each bounded wait runs out (about a
    second) and the tile is skipped.  The call must say so (CPAPR_E_TIMEOUT)
    and leave the partial counters of the rows that span tiles cleared: the
    next call, without the injection, equals cpapr_phi.  Nothing faults."""
    rng = np.random.default_rng(12)
    dims = (40, 30, 20)
    nnz = 256
    idx = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.int64)
    idx[0, : nnz // 2] = 7  # one row spanning several tiles
    vals = rng.integers(1, 4, nnz).astype(np.float64)
    fs = synth.random_factors(dims, 8, 3)
    with cpapr.Tensor(dims, idx, vals, 8, tile_nnz=64, pi_mode=cpapr.CPAPR_PI_FUSED) as t:
        t.set_model(np.ones(8), fs)
        assert t.info().ntiles[0] == 4 and t.info().nsplit[0] > 0
        want = t.phi(0)
        out = torch.zeros((dims[0], 8), dtype=torch.float64, device="cuda")
        monkeypatch.setenv("CPAPR_FAULT_STAGE_WAIT", "1")
        with pytest.raises(cpapr.CpaprError) as e:
            cpapr.cpapr_phi_noalloc(t.ctx, 0, out)
        assert e.value.status == 6
        monkeypatch.delenv("CPAPR_FAULT_STAGE_WAIT")
        for _ in range(2):
            out.fill_(float("nan"))
            cpapr.cpapr_phi_noalloc(t.ctx, 0, out)
            torch.cuda.synchronize()
            assert max_rel(out.cpu().numpy(), want) <= 1e-12


def test_noalloc_keeps_the_callers_current_device():
    T = synth.random_tensor((60, 50, 40), 3_000, 8, 91)
    fs = synth.random_factors(T.dims, 8, 5)
    with cpapr.Tensor(T.dims, T.idx, T.vals, 8) as t:
        t.set_model(np.ones(8), fs)
        out = torch.zeros((T.dims[0], 8), dtype=torch.float64, device="cuda")
        before = torch.cuda.current_device()
        cpapr.cpapr_phi_noalloc(t.ctx, 0, out)
        assert torch.cuda.current_device() == before


def test_noalloc_rejects_oversize_scratch_and_host_buffers():
    rng = np.random.default_rng(8)
    nnz, dims, R = 300_000, (2_000, 1_500, 900), 128
    idx = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.int64)
    vals = rng.integers(1, 4, nnz).astype(np.float64)
    fs = synth.random_factors(dims, R, 9)
    with cpapr.Tensor(dims, idx, vals, R, tile_nnz=64) as t:
        t.set_model(np.ones(R), fs)
        out = torch.zeros((dims[0], R), dtype=torch.float64, device="cuda")
        with pytest.raises(cpapr.CpaprError) as e:
            cpapr.cpapr_phi_noalloc(t.ctx, 0, out)
        assert e.value.status == 2 and "scratch" in str(e.value)
    with cpapr.Tensor(dims, idx, vals, 8) as t:
        t.set_model(np.ones(8), [A[:, :8].copy() for A in fs])
        with pytest.raises(cpapr.CpaprError) as e:
            cpapr.cpapr_phi_noalloc(t.ctx, 0, np.zeros((dims[0], 8)))
        assert e.value.status == 1
