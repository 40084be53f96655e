"""cpapr_phi_noalloc against cpapr_phi.

cpapr_phi_noalloc is for callers that cannot let the library allocate device
memory during a call -- their GPU memory belongs to another allocator, or the
call sits in a loop that must not block on cudaMalloc.  Its Phi kernel takes
its scratch (per-tile partial rows) from a fixed array the library keeps on
every GPU instead of a buffer the context allocated.  These tests call it
through the C ABI twice in a row with device buffers and compare each result
with the regular entry point, within the tolerances the parity tests use.
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


@pytest.mark.parametrize("precision,tol", [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 1e-5)])
def test_noalloc_matches_phi_on_two_calls(precision, tol):
    T = synth.generate(synth.scaled(synth.C3, 300_000, dims=(40_000, 40_000, 10_000, 365)))
    fs = synth.random_factors(T.dims, T.rank, 31)
    lam = 0.5 + synth.uniform01(synth.stream_base(31, 1), 0, T.rank)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, tile_nnz=512) as t:
        t.set_model(lam, fs)
        assert max(t.info().nsplit[:T.nmodes]) > 0  # rows cut across tiles: the scratch is used
        for n in range(T.nmodes):
            want = t.phi(n)
            for _ in range(2):
                out = torch.full((T.dims[n], T.rank), float("nan"), dtype=torch.float64, device="cuda")
                cpapr.cpapr_phi_noalloc(t.ctx, n, out)
                torch.cuda.synchronize()
                assert max_rel(out.cpu().numpy(), want) <= tol, (n,)
        # explicit device B
        B = fs[1] * 1.5
        want = t.phi(1, B=B)
        Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        for _ in range(2):
            out = torch.zeros((T.dims[1], T.rank), dtype=torch.float64, device="cuda")
            cpapr.cpapr_phi_noalloc(t.ctx, 1, out, B=Bd)
            torch.cuda.synchronize()
            assert max_rel(out.cpu().numpy(), want) <= tol


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
