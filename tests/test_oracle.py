"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a dense
brute-force evaluation of the printed formula, a closed form, or an
invariant that a dropped term, a wrong index or a swapped operand breaks.
The paper prints no worked numeric example, so there are no printed values
to pin against.
"""
import numpy as np
import pytest

from paper_2307_03276_gb300 import synth
from tests import _dense as D

EPS = 1e-10


def tiny(dims, nnz, R, seed, values=("poisson1", 1.0)):
    T = synth.random_tensor(dims, nnz, R, seed, values=values)
    fs = synth.random_factors(T.dims, R, seed + 7)
    return T, fs


CASES = [((5, 4, 3), 30, 3, 11), ((4, 3, 5, 2), 50, 4, 12), ((3, 4, 2, 3, 2), 60, 2, 13), ((6, 5, 4), 100, 1, 14)]


@pytest.mark.parametrize("dims,nnz,R,seed", CASES)
def test_phi_matches_dense_algorithm2(oracle, dims, nnz, R, seed):
    """Phi^(n) per nonzero equals (X_(n) ./ max(B Pi, eps)) Pi^T with dense matrices (Algorithm 2)."""
    T, fs = tiny(dims, nnz, R, seed)
    X = D.dense_tensor(T.dims, T.idx, T.vals)
    for n in range(len(dims)):
        B = synth.random_factors([dims[n]], R, seed + 100 + n)[0] * 3.0
        got = oracle.phi(T.dims, T.idx, T.vals, fs, B, n)
        want = D.phi_dense(X, fs, B, n, EPS)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dims,nnz,R,seed", CASES)
def test_mttkrp_matches_textbook(oracle, dims, nnz, R, seed):
    """MTTKRP equals X_(n) (A^(N) (.) ... (.) A^(1)) with the paper's Khatri-Rao order."""
    T, fs = tiny(dims, nnz, R, seed)
    X = D.dense_tensor(T.dims, T.idx, T.vals)
    for n in range(len(dims)):
        np.testing.assert_allclose(oracle.mttkrp(T.dims, T.idx, T.vals, fs, n), D.mttkrp_dense(X, fs, n),
                                   rtol=1e-13, atol=0)


def test_phi_epsilon_clamp(oracle):
    """A zero B row makes every denominator 0, so max(., eps) divides by eps (Algorithm 2's eps)."""
    T, fs = tiny((4, 3, 3), 20, 2, 21)
    X = D.dense_tensor(T.dims, T.idx, T.vals)
    B = synth.random_factors([4], 2, 22)[0]
    B[1, :] = 0.0
    got = oracle.phi(T.dims, T.idx, T.vals, fs, B, 0, eps=1e-3)
    np.testing.assert_allclose(got, D.phi_dense(X, fs, B, 0, 1e-3), rtol=1e-13)
    rows = T.idx[0] == 1
    if rows.any():
        pi = fs[1][T.idx[1][rows]] * fs[2][T.idx[2][rows]]
        np.testing.assert_allclose(got[1], (T.vals[rows][:, None] * pi).sum(0) / 1e-3, rtol=1e-13)


def test_per_slice_identity(oracle):
    """sum_r B[i,r] Phi[i,r] = sum of x over slice i when no denominator is clamped."""
    T = synth.generate(synth.scaled(synth.C1, 4000))
    fs = synth.random_factors(T.dims, 6, 31)
    for n in range(3):
        B = synth.random_factors([T.dims[n]], 6, 40 + n)[0] + 0.1
        P = oracle.phi(T.dims, T.idx, T.vals, fs, B, n)
        lhs = (B * P).sum(axis=1)
        rhs = np.bincount(T.idx[n], weights=T.vals, minlength=T.dims[n])
        np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-300)


def test_phi_homogeneity_and_permutation(oracle):
    """Phi(cB) = Phi(B)/c; shuffling nonzeros or relabelling a mode permutes nothing else."""
    T, fs = tiny((7, 6, 5), 120, 3, 51)
    B = synth.random_factors([7], 3, 52)[0]
    P = oracle.phi(T.dims, T.idx, T.vals, fs, B, 0)
    np.testing.assert_allclose(oracle.phi(T.dims, T.idx, T.vals, fs, 4.0 * B, 0), P / 4.0, rtol=1e-14)
    perm = np.random.default_rng(0).permutation(T.nnz)
    np.testing.assert_allclose(oracle.phi(T.dims, T.idx[:, perm], T.vals[perm], fs, B, 0), P, rtol=1e-14)
    # relabel mode 0 rows by sigma: Phi rows move with them
    sigma = np.random.default_rng(1).permutation(7)
    idx2 = T.idx.copy()
    idx2[0] = sigma[T.idx[0]]
    B2 = np.empty_like(B)
    B2[sigma] = B
    P2 = oracle.phi(T.dims, idx2, T.vals, fs, B2, 0)
    np.testing.assert_allclose(P2[sigma], P, rtol=1e-14)
    # relabel a non-output mode (1): Phi unchanged
    tau = np.random.default_rng(2).permutation(6)
    idx3 = T.idx.copy()
    idx3[1] = tau[T.idx[1]]
    fs3 = [fs[0], np.empty_like(fs[1]), fs[2]]
    fs3[1][tau] = fs[1]
    np.testing.assert_allclose(oracle.phi(T.dims, idx3, T.vals, fs3, B, 0), P, rtol=1e-14)


def test_duplicates_equal_coalesced(oracle):
    """Splitting a count over two identical coordinates gives the coalesced result (linearity in x)."""
    T, fs = tiny((5, 4, 3), 25, 2, 61)
    idx = np.concatenate([T.idx, T.idx[:, :5]], axis=1)
    vals = np.concatenate([T.vals, T.vals[:5] * 0.25])
    vals2 = T.vals.copy()
    vals2[:5] *= 1.25
    B = synth.random_factors([5], 2, 62)[0]
    for n in range(3):
        Bn = synth.random_factors([T.dims[n]], 2, 63 + n)[0]
        np.testing.assert_allclose(oracle.phi(T.dims, idx, vals, fs, Bn, n),
                                   oracle.phi(T.dims, T.idx, vals2, fs, Bn, n), rtol=1e-14)
    assert B.shape == (5, 2)


@pytest.mark.parametrize("dims,nnz,R,seed", CASES[:3])
def test_loglik_matches_dense(oracle, dims, nnz, R, seed):
    """LL = sum over all entries of x log m - m (0 log m = 0)."""
    T, fs = tiny(dims, nnz, R, seed)
    lam = np.linspace(0.5, 2.0, R)
    X = D.dense_tensor(T.dims, T.idx, T.vals)
    np.testing.assert_allclose(oracle.loglik(T.dims, T.idx, T.vals, lam, fs), D.loglik_dense(X, lam, fs),
                               rtol=1e-12)


def test_loglik_minus_inf_on_zero_model(oracle):
    T, fs = tiny((4, 3, 3), 20, 2, 71)
    fs[1][T.idx[1][0], :] = 0.0
    assert oracle.loglik(T.dims, T.idx, T.vals, np.ones(2), fs) == -np.inf


def test_mu_rank1_closed_form(oracle):
    """R = 1: one inner step sets B to the slice sums, so the solve returns lambda = sum(x)
    and A^(n) = mode-n marginals / sum(x) (the rank-1 Poisson MLE), converging at k = 2."""
    T = synth.generate(synth.scaled(synth.C1, 3000, rank=1))
    lam0, fs0 = np.ones(1), synth.random_factors(T.dims, 1, 81)
    out = oracle.mu_solve(T.dims, T.idx, T.vals, lam0, fs0, tol=1e-10, max_outer=5, max_inner=5)
    total = T.vals.sum()
    np.testing.assert_allclose(out["lambda"], [total], rtol=1e-14)
    for n in range(3):
        marg = np.bincount(T.idx[n], weights=T.vals, minlength=T.dims[n]) / total
        np.testing.assert_allclose(out["factors"][n][:, 0], marg, rtol=1e-13, atol=1e-300)
    assert out["converged"] and out["outer_iters"] == 2
    assert list(out["inner"][0]) == [2, 2, 2] and list(out["inner"][1]) == [1, 1, 1]


def test_mu_mass_conservation_and_monotone_ll(oracle):
    """After any B <- B*Phi, sum(B) = sum(x), so sum(lambda) = sum(x); with kappa = 0 the
    multiplicative update never lowers the log-likelihood."""
    T = synth.generate(synth.scaled(synth.C1, 2000, rank=4))
    lam0, fs0 = np.ones(4), synth.random_factors(T.dims, 4, 91)
    out = oracle.mu_solve(T.dims, T.idx, T.vals, lam0, fs0, tol=1e-6, max_outer=8, max_inner=3, kappa=0.0)
    np.testing.assert_allclose(out["lambda"].sum(), T.vals.sum(), rtol=1e-13)
    for A in out["factors"]:
        np.testing.assert_allclose(A.sum(axis=0), 1.0, rtol=1e-13)
    ll = out["loglik"]
    assert np.all(np.diff(ll) >= -1e-10 * np.abs(ll[:-1]))


@pytest.mark.parametrize("R,kappa", [(3, 0.0), (2, 0.01)])
def test_mu_matches_dense_outer_iterations(oracle, R, kappa):
    """Three outer iterations of Algorithm 1 with dense matrices, S included."""
    T, fs = tiny((5, 4, 3), 35, R, 101)
    lam = np.ones(R)
    if kappa:
        fs[0][1, 0] = 0.0   # an inadmissible zero that only S can move
    X = D.dense_tensor(T.dims, T.idx, T.vals)
    phi_prev = [np.zeros((d, R)) for d in T.dims]
    lam_d, fs_d = lam.copy(), [A.copy() for A in fs]
    inner_d = []
    for k in range(1, 4):
        lam_d, fs_d, inn = D.mu_outer_dense(X, lam_d, fs_d, k, 4, 1e-12, EPS, kappa, 1e-10, phi_prev)
        inner_d.append(inn)
    out = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-12, max_outer=3, max_inner=4, kappa=kappa)
    np.testing.assert_allclose(out["lambda"], lam_d, rtol=1e-11)
    for A, Ad in zip(out["factors"], fs_d):
        np.testing.assert_allclose(A, Ad, rtol=1e-10, atol=1e-300)
    assert out["inner"].tolist() == inner_d
    if kappa:
        assert out["factors"][0][1, 0] > 0.0


def test_mu_scooch_needed_for_inadmissible_zero(oracle):
    """Without S a zero entry of A stays zero forever (B*Phi keeps it 0)."""
    T, fs = tiny((5, 4, 3), 35, 2, 111)
    fs[0][2, 1] = 0.0
    out = oracle.mu_solve(T.dims, T.idx, T.vals, np.ones(2), fs, tol=1e-12, max_outer=4, max_inner=3, kappa=0.0)
    assert out["factors"][0][2, 1] == 0.0


def test_mu_converged_model_satisfies_kkt(oracle):
    """A converged solve leaves every mode with max|min(B, 1 - Phi)| < tol (dense recheck)."""
    T = synth.random_tensor((6, 5, 4), 60, 2, 121)
    lam0, fs0 = np.ones(2), synth.random_factors(T.dims, 2, 122)
    tol = 1e-4
    out = oracle.mu_solve(T.dims, T.idx, T.vals, lam0, fs0, tol=tol, max_outer=2000, max_inner=10)
    assert out["converged"]
    X = D.dense_tensor(T.dims, T.idx, T.vals)
    for n in range(3):
        assert D.kkt_dense(X, out["lambda"], out["factors"], n, EPS) < tol


def test_init_random_matches_splitmix_stream(oracle):
    """The C SplitMix64 stream reproduces synth's numpy stream; columns sum to one."""
    dims, R, seed = (7, 5, 6), 3, 2024
    lam, fs = oracle.init_random(dims, R, seed)
    raw = synth.random_factors(dims, R, seed)
    want_lam = np.prod([A.sum(axis=0) for A in raw], axis=0)
    np.testing.assert_allclose(lam, want_lam, rtol=1e-14)
    for A, W in zip(fs, raw):
        np.testing.assert_allclose(A, W / W.sum(axis=0), rtol=1e-14)


def test_oracle_rejects_out_of_range(oracle):
    T, fs = tiny((4, 3, 3), 10, 2, 131)
    idx = T.idx.copy()
    idx[1, 3] = 3
    with pytest.raises(ValueError):
        oracle.phi(T.dims, idx, T.vals, fs, np.ones((4, 2)), 0)


@pytest.mark.parametrize("inner", [1, 3])
def test_mu_two_way_is_kl_nmf(oracle, inner):
    """With N = 2 the MU loop is the Lee-Seung multiplicative update of
    non-negative matrix factorisation under the KL divergence, X ~ W H^T:
    with H's columns summing to one, W <- W * ((X / (W H^T)) H), then the
    column sums of W move into lambda, and the same for H with X^T.  Written
    here with plain dense matrix products (tol = 0: every inner iteration
    updates; one outer iteration, so no shift S)."""
    dims, R = (7, 5), 3
    T = synth.random_tensor(dims, 25, R, 31)
    X = np.zeros(dims)
    np.add.at(X, (T.idx[0], T.idx[1]), T.vals)
    A = [a / a.sum(axis=0, keepdims=True) for a in synth.random_factors(dims, R, 32)]
    lam = np.array([2.0, 5.0, 3.5])
    ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, A, tol=0.0, max_outer=1, max_inner=inner, kappa=0.0)
    W, H = A[0] * lam, A[1]
    for _ in range(inner):
        W = W * ((X / np.maximum(W @ H.T, EPS)) @ H)
    lam1 = W.sum(axis=0)
    A0 = W / lam1
    H = A[1] * lam1
    for _ in range(inner):
        H = H * ((X.T / np.maximum(H @ A0.T, EPS)) @ A0)
    lam2 = H.sum(axis=0)
    np.testing.assert_allclose(ref["lambda"], lam2, rtol=1e-12)
    np.testing.assert_allclose(ref["factors"][0], A0, rtol=1e-12)
    np.testing.assert_allclose(ref["factors"][1], H / lam2, rtol=1e-12)


def _golden():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "make_golden.py")
    spec = importlib.util.spec_from_file_location("make_golden", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_c1_golden_trajectory(oracle):
    """The oracle's ten-outer-iteration solve of the 100 x 80 x 60 workload
    reproduces the trajectory stored in tests/golden/c1_mu_oracle.txt
    (written by make_golden.py from the oracle alone): inner iterations per
    mode, KKT violation and log-likelihood per outer iteration, and lambda,
    whose sum is the total count (mass conservation)."""
    g = _golden()
    want = g.read()
    r = g.solve()
    assert r["outer_iters"] == want["outer_iters"] and bool(r["converged"]) == want["converged"]
    for k, (inner, kkt, ll) in enumerate(want["outer"]):
        assert list(r["inner"][k]) == inner
        assert abs(r["kkt"][k] - kkt) <= 1e-13 * kkt
        assert abs(r["loglik"][k] - ll) <= 1e-13 * abs(ll)
    np.testing.assert_allclose(r["lambda"], want["lambda"], rtol=1e-13)
    T = synth.generate(synth.C1)
    assert abs(want["lambda"].sum() - T.vals.sum()) <= 1e-12 * T.vals.sum()
    # the log-likelihood never decreases along the stored trajectory (kappa's shift aside, MU is an MM method)
    lls = [o[2] for o in want["outer"]]
    assert all(b >= a for a, b in zip(lls, lls[1:]))


@pytest.mark.parametrize("nthreads", [1, 3, 8, 64])
def test_threaded_phi_equals_single_threaded(oracle, nthreads):
    """The multi-threaded Phi of the CPU baseline (each thread owns a range of
    rows and sums them term by term in the given order) gives the plain
    oracle's bits: rows with thousands of terms, a skewed row, empty rows,
    more threads than a mode has rows."""
    T = synth.generate(synth.scaled(synth.C2, 20_000, dims=(300, 200, 50), rank=7))
    fs = synth.random_factors(T.dims, 7, 5)
    for n in range(3):
        B = fs[n] * 1.3
        want = oracle.phi(T.dims, T.idx, T.vals, fs, B, n)
        got = oracle.phi_threads(T.dims, T.idx, T.vals, fs, B, n, nthreads)
        assert np.array_equal(got, want)
