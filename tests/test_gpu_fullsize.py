"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (default tiles and lanes), on sampled outputs the oracle computes one
by one: for every mode, the rows of Phi^(n) (and of MTTKRP) for the heaviest
slice, the lightest non-empty slice, random slices and an empty slice.  The
oracle evaluates exactly those rows from the sub-tensor of their nonzeros.
Properties that hold at any size check one full MU outer iteration.

Workloads: 3-way 1e5 x 1e5 x 1e3 (1e7 nonzeros, R = 32), 4-way
2e5 x 2e5 x 1e4 x 365 (5e7, R = 16), 5-way 5e4 x 5e4 x 5e3 x 1e3 x 24
(1e8, R = 64).
"""
import numpy as np
import pytest

import oracle
from paper_2307_03276_gb300 import cpapr, synth

pytestmark = pytest.mark.gpu

_T = {}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2307_03276_gb300 import build
    build.build()
    oracle.build()


def tensor(name):
    if name not in _T:
        _T[name] = synth.generate(synth.SPECS[name])
    return _T[name]


def model(T):
    fs = synth.random_factors(T.dims, T.rank, T.seed + 17)
    lam = 0.5 + synth.uniform01(synth.stream_base(T.seed, 77), 0, T.rank)
    return lam, fs


def sample_rows(T, n, k=5):
    counts = np.bincount(T.idx[n], minlength=T.dims[n])
    nonempty = np.flatnonzero(counts)
    rng = np.random.default_rng(n + 100)
    rows = {int(np.argmax(counts)), int(nonempty[np.argmin(counts[nonempty])])}
    rows.update(int(r) for r in rng.choice(nonempty, size=min(k, nonempty.size), replace=False))
    empty = np.flatnonzero(counts == 0)
    if empty.size:
        rows.add(int(empty[0]))
    return np.array(sorted(rows))


def sub_tensor(T, n, rows):
    mask = np.isin(T.idx[n], rows)
    return np.ascontiguousarray(T.idx[:, mask]), np.ascontiguousarray(T.vals[mask])


def rel_err(got, want):
    nz = want != 0
    e = np.zeros_like(want)
    e[nz] = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
    e[~nz] = np.abs(got[~nz]) > 0
    return float(e.max())


@pytest.mark.parametrize("name", ["c2", "c3", "c5"])
@pytest.mark.parametrize("precision,tol", [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 1e-5)])
def test_fullsize_phi_and_mttkrp_sampled_rows(name, precision, tol):
    T = tensor(name)
    lam, fs = model(T)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision) as t:
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            rows = sample_rows(T, n)
            idx, vals = sub_tensor(T, n, rows)
            want = oracle.phi(T.dims, idx, vals, fs, fs[n] * lam[None, :], n)[rows]
            got = t.phi(n)[rows]
            assert rel_err(got, want) <= tol, (name, n)
            if n == T.nmodes - 1:
                wm = oracle.mttkrp(T.dims, idx, vals, fs, n)[rows]
                assert rel_err(t.mttkrp(n)[rows], wm) <= tol, (name, n, "mttkrp")


@pytest.mark.parametrize("precision,tol", [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 2e-6)])
def test_fullsize_outer_iteration_properties(precision, tol):
    """One outer iteration on the 1e7-nonzero tensor: after B <- B*Phi the
    model's total mass equals sum(x), so sum(lambda) = sum(x); every factor
    column sums to one; the log-likelihood does not decrease."""
    T = tensor("c2")
    lam, fs = model(T)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision) as t:
        t.set_model(lam, fs)
        ll0 = t.loglik()
        res = t.mu_solve(tol=1e-4, max_outer=1, max_inner=10)
        lg, fg = t.get_model()
    total = T.vals.sum()
    assert abs(lg.sum() - total) <= tol * total
    for A in fg:
        np.testing.assert_allclose(A.sum(axis=0), 1.0, rtol=max(tol, 1e-12) * 10)
    assert res["loglik"] >= ll0
