"""Batched CP-APR MU (cpapr_batch_mu_solve): many uneven tensors in one
persistent launch per step, against solving each tensor alone and against
the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2307_03276_gb300 import cpapr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2307_03276_gb300 import build
    build.build()
    oracle.build()


def batch_tensors(count=7, seed=77):
    specs = synth.batch_specs(count=count, seed=seed, nnz_range=(300, 30_000), dim_hi=(2_000, 2_000, 200))
    out = []
    for k, sp in enumerate(specs):
        if k == 0:  # a rank-1 tensor converges after two outer iterations and gets masked
            sp = synth.TensorSpec(sp.dims, sp.nnz, 1, sp.modes, sp.values, sp.seed, sp.name)
        T = synth.generate(sp)
        out.append(T)
    return out


def models(tensors):
    res = []
    for T in tensors:
        fs = synth.random_factors(T.dims, T.rank, T.seed + 3)
        res.append((np.ones(T.rank), fs))
    return res


@pytest.mark.parametrize("use_graph", [1, 0])
def test_batch_fp64_equals_individual_solves_and_oracle(use_graph):
    Ts = batch_tensors()
    ms = models(Ts)
    tol, mo, mi = 1e-4, 6, 5
    batch = [cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, use_graph=use_graph) for T in Ts]
    for t, (lam, fs) in zip(batch, ms):
        t.set_model(lam, fs)
    res = cpapr.cpapr_batch_mu_solve([t.ctx for t in batch], tol, mo, mi)
    for T, t, (lam, fs), r in zip(Ts, batch, ms, res):
        lb, fb = t.get_model()
        with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as s:
            s.set_model(lam, fs)
            ri = s.mu_solve(tol, mo, mi)
            li, fi = s.get_model()
        assert (r["outer_iters"], r["total_inner"], r["converged"]) == (ri["outer_iters"], ri["total_inner"],
                                                                          ri["converged"])
        # same kernels and tiles; only the column sums are added in another fixed order
        np.testing.assert_allclose(lb, li, rtol=1e-12)
        for a, b in zip(fb, fi):
            np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-15 * b.max())
        ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=tol, max_outer=mo, max_inner=mi)
        assert r["outer_iters"] == ref["outer_iters"] and r["total_inner"] == ref["total_inner"]
        np.testing.assert_allclose(lb, ref["lambda"], rtol=1e-10)
        for a, b in zip(fb, ref["factors"]):
            np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-14 * b.max())
        assert abs(r["loglik"] - ref["loglik"][-1]) <= 1e-11 * abs(ref["loglik"][-1])
        # the batched log-likelihood launches against the single-tensor one on the same final model
        assert abs(r["loglik"] - t.loglik()) <= 1e-13 * abs(r["loglik"])
        t.close()
    assert res[0]["converged"] and res[0]["outer_iters"] == 2


def test_batch_fp32_close_to_individual():
    Ts = batch_tensors(seed=78)
    ms = models(Ts)
    batch = [cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=cpapr.CPAPR_FP32) for T in Ts]
    for t, (lam, fs) in zip(batch, ms):
        t.set_model(lam, fs)
    res = cpapr.cpapr_batch_mu_solve([t.ctx for t in batch], 1e-4, 3, 5)
    for T, t, (lam, fs), r in zip(Ts, batch, ms, res):
        lb, fb = t.get_model()
        ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-4, max_outer=3, max_inner=5)
        np.testing.assert_allclose(lb, ref["lambda"], rtol=1e-4)
        assert abs(r["loglik"] - ref["loglik"][-1]) <= 1e-5 * abs(ref["loglik"][-1])
        assert abs(r["loglik"] - t.loglik()) <= 1e-6 * abs(r["loglik"])
        t.close()


def test_batch_mixed_modes_falls_back():
    """Tensors with different numbers of modes still solve (lock-step path)."""
    a = synth.random_tensor((30, 20, 10), 800, 4, 5)
    b = synth.random_tensor((12, 10, 8, 6), 900, 4, 6)
    ts = []
    for T in (a, b):
        t = cpapr.Tensor(T.dims, T.idx, T.vals, T.rank)
        t.set_model(np.ones(4), synth.random_factors(T.dims, 4, 9))
        ts.append(t)
    res = cpapr.cpapr_batch_mu_solve([t.ctx for t in ts], 1e-4, 2, 3)
    for T, t, r in zip((a, b), ts, res):
        ref = oracle.mu_solve(T.dims, T.idx, T.vals, np.ones(4), synth.random_factors(T.dims, 4, 9), tol=1e-4,
                              max_outer=2, max_inner=3)
        np.testing.assert_allclose(t.get_model()[0], ref["lambda"], rtol=1e-10)
        t.close()


@pytest.mark.parametrize("precision", [cpapr.CPAPR_FP64, cpapr.CPAPR_FP32])
def test_batch_with_an_empty_tensor(precision):
    """A tensor without nonzeros rides along in a batch: it gets no tiles, its
    log-likelihood is the model total alone, and the other tensors' results
    match their oracle solves."""
    a = synth.random_tensor((40, 30, 20), 2_000, 8, 11)
    ts = []
    for dims, T in (((40, 30, 20), a), ((25, 15, 10), None)):
        if T is None:
            t = cpapr.Tensor(dims, np.zeros((3, 0), dtype=np.int64), np.zeros(0), 8, precision=precision)
        else:
            t = cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision)
        t.set_model(np.ones(8), synth.random_factors(dims, 8, 12))
        ts.append(t)
    res = cpapr.cpapr_batch_mu_solve([t.ctx for t in ts], 1e-4, 2, 3)
    ref = oracle.mu_solve(a.dims, a.idx, a.vals, np.ones(8), synth.random_factors(a.dims, 8, 12), tol=1e-4,
                          max_outer=2, max_inner=3)
    rt = 1e-11 if precision == cpapr.CPAPR_FP64 else 1e-5
    assert abs(res[0]["loglik"] - ref["loglik"][-1]) <= rt * abs(ref["loglik"][-1])
    for t, r in zip(ts, res):
        ll = t.loglik()
        assert np.isfinite(r["loglik"]) and abs(r["loglik"] - ll) <= 1e-12 * max(1.0, abs(ll))
        t.close()


def _sample_rows(T, n, k=4):
    counts = np.bincount(T.idx[n], minlength=T.dims[n])
    nonempty = np.flatnonzero(counts)
    rng = np.random.default_rng(n + 300)
    rows = {int(np.argmax(counts)), int(nonempty[np.argmin(counts[nonempty])])}
    rows.update(int(r) for r in rng.choice(nonempty, size=min(k, nonempty.size), replace=False))
    return np.array(sorted(rows))


def _rel(got, want):
    nz = want != 0
    e = np.zeros_like(want)
    e[nz] = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
    e[~nz] = np.abs(got[~nz]) > 0
    return float(e.max())


@pytest.mark.parametrize("precision", [cpapr.CPAPR_FP64, cpapr.CPAPR_FP32])
def test_full_64_tensor_batch_equals_individual_solves(precision):
    """The 64-tensor batch at its full size (dims log-uniform up to
    20000 x 20000 x 500, 1e3..1e6 nonzeros, R from {8, 16, 32}): two outer
    iterations through the persistent batched solver against one mu_solve
    per tensor from the same start (same inner iteration counts; lambda and
    factors equal up to the order of the column sums), and sampled Phi rows
    of the final models of the three largest tensors against the oracle."""
    Ts = [synth.generate(sp) for sp in synth.batch_specs(count=64)]
    ms = models(Ts)
    tol, mo, mi = 1e-4, 2, 10
    fp64 = precision == cpapr.CPAPR_FP64
    batch = [cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision) for T in Ts]
    for t, (lam, fs) in zip(batch, ms):
        t.set_model(lam, fs)
    res = cpapr.cpapr_batch_mu_solve([t.ctx for t in batch], tol, mo, mi)
    largest = sorted(range(len(Ts)), key=lambda i: -Ts[i].nnz)[:3]
    for i, (T, t, (lam, fs), r) in enumerate(zip(Ts, batch, ms, res)):
        lb, fb = t.get_model()
        with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision) as s:
            s.set_model(lam, fs)
            ri = s.mu_solve(tol, mo, mi)
            li, fi = s.get_model()
        assert (r["outer_iters"], r["total_inner"]) == (ri["outer_iters"], ri["total_inner"]), i
        if fp64:
            np.testing.assert_allclose(lb, li, rtol=1e-12)
            for a, b in zip(fb, fi):
                np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-15 * b.max())
            assert abs(r["loglik"] - ri["loglik"]) <= 1e-12 * abs(ri["loglik"])
        else:
            # FP32 factors: the batched column sums round differently in the
            # last FP64 bits, which can move an FP32 factor entry by one ulp
            np.testing.assert_allclose(lb, li, rtol=1e-5)
            for a, b in zip(fb, fi):
                np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-7 * b.max())
            assert abs(r["loglik"] - ri["loglik"]) <= 1e-5 * abs(ri["loglik"])
        if i in largest:
            # Phi of the final batched model, sampled rows against the oracle
            for n in range(T.nmodes):
                rows = _sample_rows(T, n)
                mask = np.isin(T.idx[n], rows)
                idx = np.ascontiguousarray(T.idx[:, mask])
                vals = np.ascontiguousarray(T.vals[mask])
                want = oracle.phi(T.dims, idx, vals, fb, fb[n] * lb[None, :], n)[rows]
                got = t.phi(n)[rows]
                assert _rel(got, want) <= (1e-12 if fp64 else 1e-5), (i, n)
        t.close()


@pytest.mark.parametrize("precision", [cpapr.CPAPR_FP64, cpapr.CPAPR_FP32])
def test_batch_with_tuned_contexts_matches_oracle(tmp_path, precision):
    """Contexts whose tiles (and, in FP64, Pi forms) come from the tuning
    cache solve together: the batched solver keeps each context's tile as
    long as it fits its shared-memory budget, and the result matches the
    oracle's solve of each tensor."""
    Ts = batch_tensors(seed=79)
    ms = models(Ts)
    path = tmp_path / "tune.txt"
    batch = [cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, autotune=1, tune_cache=str(path))
             for T in Ts]
    assert path.exists() and len(path.read_text().splitlines()) >= 1
    for t, (lam, fs) in zip(batch, ms):
        t.set_model(lam, fs)
    res = cpapr.cpapr_batch_mu_solve([t.ctx for t in batch], 1e-4, 3, 5)
    fp64 = precision == cpapr.CPAPR_FP64
    for T, t, (lam, fs), r in zip(Ts, batch, ms, res):
        lb, fb = t.get_model()
        ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-4, max_outer=3, max_inner=5)
        assert r["total_inner"] == ref["total_inner"]
        np.testing.assert_allclose(lb, ref["lambda"], rtol=1e-10 if fp64 else 1e-5)
        assert abs(r["loglik"] - ref["loglik"][-1]) <= (1e-11 if fp64 else 1e-6) * abs(ref["loglik"][-1])
        t.close()
