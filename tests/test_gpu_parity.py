"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (per entry, relative):
  FP64 Phi / MTTKRP 1e-12 -- all terms are non-negative, so only summation
      order differs; a segmented sum of k terms errs by about log2(k) ulps.
  FP32 Phi / MTTKRP 1e-5 -- each term carries about (N - 1 + R + 4) FP32
      roundings (factor conversion, Khatri-Rao product, dot, divide) and the
      row sums are Kahan-compensated.
  log-likelihood: FP64 1e-11 relative (a sum with cancellation against the
      model total), FP32 1e-5.
"""
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


def max_rel(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    nz = want != 0
    err = np.zeros_like(want)
    err[nz] = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
    err[~nz] = np.abs(got[~nz]) > 0
    return float(err.max()) if err.size else 0.0


def make_case(name):
    if name == "c1":
        return synth.generate(synth.C1)
    if name == "c2s":
        return synth.generate(synth.scaled(synth.C2, 200_000, dims=(20_000, 20_000, 1_000)))
    if name == "c3s":
        return synth.generate(synth.scaled(synth.C3, 300_000, dims=(40_000, 40_000, 10_000, 365)))
    if name == "c5s":
        return synth.generate(synth.scaled(synth.C5, 200_000, dims=(5_000, 5_000, 500, 100, 24), rank=8))
    if name == "c5s64":
        return synth.generate(synth.scaled(synth.C5, 100_000, dims=(5_000, 5_000, 500, 100, 24), rank=64))
    if name == "n2":
        return synth.random_tensor((300, 200), 5_000, 4, 77)
    if name == "n6":
        return synth.random_tensor((10, 9, 8, 7, 6, 5), 3_000, 8, 78)
    raise KeyError(name)


_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = make_case(name)
    return _cache[name]


def model_for(T, seed=5):
    fs = synth.random_factors(T.dims, T.rank, seed)
    lam = 0.5 + synth.uniform01(synth.stream_base(seed, 999), 0, T.rank)
    return lam, fs


CASES = ["c1", "c2s", "c3s", "c5s", "c5s64", "n2", "n6"]


PI_MODES = [cpapr.CPAPR_PI_FUSED, cpapr.CPAPR_PI_MATERIALISED]
# the FP64 form's dot product in FP64 and on the FP32 pipe (the automatic
# choice picks the latter only for launches of 608 tiles or more)
DOTS = [cpapr.CPAPR_DOT_FP64, cpapr.CPAPR_DOT_FP32_PIPE]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("reduction", [cpapr.CPAPR_REDUCE_SEGMENTED, cpapr.CPAPR_REDUCE_ATOMIC])
@pytest.mark.parametrize("pi_mode", PI_MODES)
@pytest.mark.parametrize("dot", DOTS)
def test_phi_fp64_matches_oracle(name, reduction, pi_mode, dot):
    T = case(name)
    lam, fs = model_for(T)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, reduction=reduction, pi_mode=pi_mode, fp64_dot=dot) as t:
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[n] * lam[None, :], n)
            got = t.phi(n)
            assert max_rel(got, want) <= 1e-12, (name, n)


@pytest.mark.parametrize("name", ["c1", "c2s", "c3s", "c5s64"])
@pytest.mark.parametrize("tile", [64, 320, 4096])
def test_phi_fp64_tile_sizes(name, tile):  # 64-nonzero tiles: 608 or more tiles, the FP32-pipe dot
    """Small tiles cut many rows across tiles and groups (rows finished by the
    last tile to arrive), large ones few."""
    T = case(name)
    lam, fs = model_for(T, 9)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, tile_nnz=tile) as t:
        t.set_model(lam, fs)
        info = t.info()
        for n in range(T.nmodes):
            want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[n] * lam[None, :], n)
            assert max_rel(t.phi(n), want) <= 1e-12, (name, tile, n, info.nsplit[n])


@pytest.mark.parametrize("name", ["c1", "c2s", "c3s", "c5s", "c5s64", "n6"])
def test_phi_fp32_matches_oracle(name):
    T = case(name)
    lam, fs = model_for(T)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=cpapr.CPAPR_FP32) as t:
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[n] * lam[None, :], n)
            assert max_rel(t.phi(n), want) <= 1e-5, (name, n)


@pytest.mark.parametrize("precision,tol", [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 1e-5)])
@pytest.mark.parametrize("rank", [16, 32, 64])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16])
def test_phi_rank_lanes(precision, tol, rank, lanes):
    """Every instantiated lanes-per-nonzero choice gives the same Phi (and MTTKRP)."""
    T = synth.generate(synth.scaled(synth.C3, 60_000, dims=(8_000, 8_000, 2_000, 365), rank=rank))
    lam, fs = model_for(T, 11)
    try:
        t = cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, rank_lanes=lanes, tile_nnz=1024)
    except cpapr.CpaprError as e:
        assert e.status == 1
        pytest.skip("lanes choice not instantiated for this rank/precision")
    with t:
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[n] * lam[None, :], n)
            assert max_rel(t.phi(n), want) <= tol, (lanes, n)
        assert max_rel(t.mttkrp(2), oracle.mttkrp(T.dims, T.idx, T.vals, fs, 2)) <= tol
        ll = oracle.loglik(T.dims, T.idx, T.vals, lam, fs)
        assert abs(t.loglik() - ll) <= (1e-11 if precision == cpapr.CPAPR_FP64 else 1e-5) * abs(ll)


@pytest.mark.parametrize("name", ["c1", "c3s", "c5s", "n6"])
@pytest.mark.parametrize("precision,tol", [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 1e-5)])
def test_mttkrp_matches_oracle(name, precision, tol):
    T = case(name)
    lam, fs = model_for(T)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision) as t:
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            assert max_rel(t.mttkrp(n), oracle.mttkrp(T.dims, T.idx, T.vals, fs, n)) <= tol, (name, n)


@pytest.mark.parametrize("name", ["c1", "c3s", "c5s"])
@pytest.mark.parametrize("precision,tol", [(cpapr.CPAPR_FP64, 1e-11), (cpapr.CPAPR_FP32, 1e-5)])
def test_loglik_matches_oracle(name, precision, tol):
    T = case(name)
    lam, fs = model_for(T)
    want = oracle.loglik(T.dims, T.idx, T.vals, lam, fs)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision) as t:
        t.set_model(lam, fs)
        got = t.loglik()
    assert abs(got - want) <= tol * abs(want), (got, want)


@pytest.mark.parametrize("name", ["c2s", "c3s", "c5s64"])
def test_loglik_from_materialised_rows(name):
    """After an outer iteration the last mode's materialised Khatri-Rao rows
    were built from the final factors of the other modes; the FP64
    log-likelihood then runs along that mode and streams them.  Both the
    solver's value and a later cpapr_loglik match the oracle on the final model."""
    T = case(name)
    lam, fs = model_for(T, 15)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, pi_mode=cpapr.CPAPR_PI_MATERIALISED) as t:
        t.set_model(lam, fs)
        r = t.mu_solve(tol=1e-4, max_outer=1, max_inner=3)
        got = t.loglik()
        lam2, fs2 = t.get_model()
    want = oracle.loglik(T.dims, T.idx, T.vals, lam2, fs2)
    assert abs(got - want) <= 1e-11 * abs(want), (got, want)
    assert abs(r["loglik"] - want) <= 1e-11 * abs(want), (r["loglik"], want)


def test_explicit_b_with_epsilon_clamp():
    """A zero row of B clamps every denominator of that slice to eps (Algorithm 2)."""
    T = case("c1")
    lam, fs = model_for(T)
    B = fs[0] * 2.0
    B[3] = 0.0
    B[7, :] = 1e-30
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as t:
        t.set_model(lam, fs)
        got = t.phi(0, B=B)
    want = oracle.phi(T.dims, T.idx, T.vals, fs, B, 0)
    assert max_rel(got, want) <= 1e-12


def test_phi_deterministic_segmented():
    T = case("c2s")
    lam, fs = model_for(T)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, tile_nnz=256) as t:
        t.set_model(lam, fs)
        a = t.phi(0)
        b = t.phi(0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("use_graph", [0, 1])
@pytest.mark.parametrize("dot", DOTS)
def test_mu_solve_fp64_matches_oracle_c1(use_graph, dot):
    """Ten outer iterations of Algorithm 1 on the 100x80x60 tensor."""
    T = case("c1")
    lam, fs = model_for(T, 21)
    ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-4, max_outer=10, max_inner=10)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, use_graph=use_graph, fp64_dot=dot) as t:
        t.set_model(lam, fs)
        res = t.mu_solve(tol=1e-4, max_outer=10, max_inner=10, trace=True)
        lam_g, fs_g = t.get_model()
    assert res["outer_iters"] == ref["outer_iters"]
    assert np.array_equal(res["inner"], ref["inner"])
    assert res["total_inner"] == ref["total_inner"]
    assert max_rel(lam_g, ref["lambda"]) <= 1e-10
    for A, Ar in zip(fs_g, ref["factors"]):
        np.testing.assert_allclose(A, Ar, rtol=1e-9, atol=1e-14 * Ar.max())
    np.testing.assert_allclose(res["loglik_trace"], ref["loglik"], rtol=1e-11)
    assert abs(res["loglik"] - ref["loglik"][-1]) <= 1e-11 * abs(ref["loglik"][-1])


def test_mu_solve_fp64_4way_two_outer():
    T = case("c3s")
    lam, fs = model_for(T, 22)
    ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-4, max_outer=2, max_inner=4)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as t:
        t.set_model(lam, fs)
        res = t.mu_solve(tol=1e-4, max_outer=2, max_inner=4, trace=True)
        lam_g, fs_g = t.get_model()
    assert np.array_equal(res["inner"], ref["inner"])
    assert max_rel(lam_g, ref["lambda"]) <= 1e-10
    for A, Ar in zip(fs_g, ref["factors"]):
        np.testing.assert_allclose(A, Ar, rtol=1e-9, atol=1e-14 * Ar.max())


@pytest.mark.parametrize("dot", DOTS)
def test_mu_solve_fp64_long_horizon(dot):
    """Twelve outer iterations of ten inner iterations on the 200,000-nonzero
    3-way Zipf tensor: the log-likelihood after every outer iteration, the
    final KKT violation and the model follow the oracle's trajectory (no
    drift: the two agree to a few ulps after 360 Phi evaluations), with the
    dot in FP64 and on the FP32 pipe."""
    T = case("c2s")
    lam, fs = model_for(T, 23)
    ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-4, max_outer=12, max_inner=10)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, fp64_dot=dot) as t:
        t.set_model(lam, fs)
        res = t.mu_solve(tol=1e-4, max_outer=12, max_inner=10, trace=True, ll_trace=True)
        lam_g, fs_g = t.get_model()
    assert res["outer_iters"] == ref["outer_iters"] and np.array_equal(res["inner"], ref["inner"])
    assert max_rel(res["loglik_trace"], ref["loglik"]) <= 1e-12
    assert abs(res["kkt_viol"] - ref["kkt"][-1]) <= 1e-9 * ref["kkt"][-1]
    assert max_rel(lam_g, ref["lambda"]) <= 1e-10
    for A, Ar in zip(fs_g, ref["factors"]):
        np.testing.assert_allclose(A, Ar, rtol=1e-8, atol=1e-14 * Ar.max())


def test_mu_solve_fp32_close_to_oracle():
    T = case("c1")
    lam, fs = model_for(T, 23)
    ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-4, max_outer=3, max_inner=5)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=cpapr.CPAPR_FP32) as t:
        t.set_model(lam, fs)
        res = t.mu_solve(tol=1e-4, max_outer=3, max_inner=5)
        lam_g, fs_g = t.get_model()
    assert max_rel(lam_g, ref["lambda"]) <= 1e-4
    assert abs(res["loglik"] - ref["loglik"][-1]) <= 1e-5 * abs(ref["loglik"][-1])


def test_solve_resumes_across_calls():
    """Two calls of one outer iteration equal one call of two (S from the 2nd on), bit for bit."""
    T = case("c1")
    lam, fs = model_for(T, 24)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as t:
        t.set_model(lam, fs)
        t.mu_solve(tol=1e-4, max_outer=1, max_inner=5)
        t.mu_solve(tol=1e-4, max_outer=1, max_inner=5)
        a = t.get_model()
        t.set_model(lam, fs)
        t.mu_solve(tol=1e-4, max_outer=2, max_inner=5)
        b = t.get_model()
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", [cpapr.CPAPR_FP64, cpapr.CPAPR_FP32])
def test_checkpoint_resume_is_bit_identical(precision):
    """Stop after two outer iterations, restore the state into a new context,
    continue: the same bits as running on without stopping (S included)."""
    T = case("c3s")
    lam, fs = model_for(T, 25)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision) as t:
        t.set_model(lam, fs)
        t.mu_solve(1e-4, 2, 4)
        state = cpapr.cpapr_get_state(t.ctx)
        r1 = t.mu_solve(1e-4, 2, 4)
        a = t.get_model()
    assert state["outer_done"] == 2
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision) as u:
        cpapr.cpapr_set_state(u.ctx, state)
        r2 = u.mu_solve(1e-4, 2, 4)
        b = u.get_model()
    assert r1 == r2
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)


def test_injected_allocation_failure_is_clean(monkeypatch):
    """A failing device allocation (injected on the host) surfaces as
    CPAPR_E_NOMEM from cpapr_create and leaves the library usable."""
    T = case("c1")
    for k in (1, 5, 12):
        monkeypatch.setenv("CPAPR_FAULT_ALLOC_AT", str(k))
        with pytest.raises(cpapr.CpaprError) as e:
            cpapr.Tensor(T.dims, T.idx, T.vals, T.rank)
        assert e.value.status == 4 and "injected" in str(e.value)
    monkeypatch.delenv("CPAPR_FAULT_ALLOC_AT")
    lam, fs = model_for(T)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as t:
        t.set_model(lam, fs)
        want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[0] * lam[None, :], 0)
        assert max_rel(t.phi(0), want) <= 1e-12


@pytest.mark.parametrize("precision,tol", [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 1e-5)])
def test_autotuned_context_matches_oracle(precision, tol):
    """The autotuner times (lanes, tile, reduction) per mode on the tensor and
    keeps the fastest; whatever it picks must give the same Phi."""
    T = case("c2s")
    lam, fs = model_for(T, 26)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, autotune=1) as t:
        info = t.info()
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            assert info.tile_nnz[n] in (1024, 2048, 4096, 8192)
            want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[n] * lam[None, :], n)
            assert max_rel(t.phi(n), want) <= tol


def test_init_random_matches_oracle():
    T = case("c1")
    lo, fo = oracle.init_random(T.dims, T.rank, 4242)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as t:
        t.init_random(4242)
        lg, fg = t.get_model()
    assert max_rel(lg, lo) <= 1e-13
    for a, b in zip(fg, fo):
        assert max_rel(a, b) <= 1e-13


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_empty_tensor():
    dims = (5, 4, 3)
    idx = np.zeros((3, 0), dtype=np.int64)
    vals = np.zeros(0)
    fs = synth.random_factors(dims, 2, 1)
    lam = np.ones(2)
    with cpapr.Tensor(dims, idx, vals, 2) as t:
        t.set_model(lam, fs)
        for n in range(3):
            assert np.all(t.phi(n) == 0.0)
            assert np.all(t.mttkrp(n) == 0.0)
        ll = t.loglik()
    assert abs(ll - oracle.loglik(dims, idx, vals, lam, fs)) <= 1e-12 * abs(ll)


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 7, 5), (9, 1, 4, 1)])
def test_single_nonzero_and_unit_modes(dims):
    idx = np.array([[d - 1] for d in dims], dtype=np.int64)
    vals = np.array([3.0])
    fs = synth.random_factors(dims, 3, 2)
    lam = np.ones(3)
    with cpapr.Tensor(dims, idx, vals, 3) as t:
        t.set_model(lam, fs)
        for n in range(len(dims)):
            want = oracle.phi(dims, idx, vals, fs, fs[n], n)
            assert max_rel(t.phi(n), want) <= 1e-12


def test_heavy_row_spanning_many_tiles():
    """One row holds 60% of the nonzeros and spans hundreds of tiles."""
    rng = np.random.default_rng(3)
    nnz = 200_000
    dims = (50, 3000, 2000)
    i0 = np.where(rng.random(nnz) < 0.6, 17, rng.integers(0, 50, nnz))
    idx = np.stack([i0, rng.integers(0, 3000, nnz), rng.integers(0, 2000, nnz)]).astype(np.int64)
    vals = rng.integers(1, 5, nnz).astype(np.float64)
    fs = synth.random_factors(dims, 16, 4)
    lam = np.ones(16)
    for prec, tol in [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 1e-5)]:
        with cpapr.Tensor(dims, idx, vals, 16, tile_nnz=512, precision=prec) as t:
            t.set_model(lam, fs)
            want = oracle.phi(dims, idx, vals, fs, fs[0], 0)
            assert max_rel(t.phi(0), want) <= tol


def test_empty_slices_and_duplicates():
    rng = np.random.default_rng(5)
    dims = (200, 30, 20)
    nnz = 3000
    idx = np.stack([rng.integers(0, 50, nnz) * 4, rng.integers(0, 30, nnz), rng.integers(0, 20, nnz)]).astype(np.int64)
    idx = np.concatenate([idx, idx[:, :100]], axis=1)
    vals = np.concatenate([rng.integers(1, 4, nnz), rng.integers(1, 4, 100)]).astype(np.float64)
    fs = synth.random_factors(dims, 4, 6)
    lam = np.ones(4)
    with cpapr.Tensor(dims, idx, vals, 4, tile_nnz=128) as t:
        t.set_model(lam, fs)
        for n in range(3):
            want = oracle.phi(dims, idx, vals, fs, fs[n], n)
            assert max_rel(t.phi(n), want) <= 1e-12


@pytest.mark.parametrize("rank", [1, 3, 10, 33, 128])
def test_ranks_not_power_of_two(rank):
    T = synth.random_tensor((40, 30, 20), 4000, rank, 90 + rank)
    lam, fs = model_for(T)
    for prec, tol in [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 1e-5)]:
        with cpapr.Tensor(T.dims, T.idx, T.vals, rank, precision=prec) as t:
            t.set_model(lam, fs)
            for n in range(3):
                want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[n] * lam[None, :], n)
                assert max_rel(t.phi(n), want) <= tol, (rank, prec, n)


@pytest.mark.parametrize("name", ["c1", "c2s", "c3s", "c5s64", "n6"])
@pytest.mark.parametrize("precision", [cpapr.CPAPR_FP64, cpapr.CPAPR_FP32])
def test_materialised_pi_equals_fused(name, precision):
    """Phi from the materialised Khatri-Rao rows (Algorithm 3's Pi, built
    once per mode) is bit-identical to Phi with the rows formed per nonzero:
    the products are taken in the same order and the Phi arithmetic is the
    same (given the same tiles: the automatic tile size depends on the form).
    The info block reports the choice."""
    T = case(name)
    lam, fs = model_for(T, 12)
    got = {}
    for pm in PI_MODES:
        with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, pi_mode=pm, tile_nnz=1024,
                          fp64_dot=cpapr.CPAPR_DOT_FP32_PIPE) as t:
            t.set_model(lam, fs)
            info = t.info()
            assert list(info.pi_mode)[:T.nmodes] == [pm] * T.nmodes
            got[pm] = [t.phi(n) for n in range(T.nmodes)]
    for n in range(T.nmodes):
        assert np.array_equal(got[PI_MODES[0]][n], got[PI_MODES[1]][n]), (name, n)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_mu_solve_materialised_pi_equals_fused(use_graph):
    """A whole MU solve (S, B, inner loops with the KKT check, normalisation)
    ends in the same model whether Pi is materialised or fused, and matches
    the oracle."""
    T = case("c3s")
    lam, fs = model_for(T, 13)
    res = {}
    for pm in PI_MODES:
        with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, pi_mode=pm, use_graph=use_graph, tile_nnz=1024) as t:
            t.set_model(lam, fs)
            r = t.mu_solve(tol=1e-4, max_outer=2, max_inner=5)
            res[pm] = (r, t.get_model())
    (r0, (l0, f0)), (r1, (l1, f1)) = res[PI_MODES[0]], res[PI_MODES[1]]
    assert r0["total_inner"] == r1["total_inner"]
    assert np.array_equal(l0, l1)
    for a, b in zip(f0, f1):
        assert np.array_equal(a, b)
    want = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-4, max_outer=2, max_inner=5)
    assert max_rel(l1, want["lambda"]) <= 1e-10
    for A, Ar in zip(f1, want["factors"]):
        np.testing.assert_allclose(A, Ar, rtol=1e-9, atol=1e-14 * Ar.max())


def test_staging_wait_timeout_is_reported(monkeypatch):
    """The tile kernels' one wait (for a tile's bulk copies into shared
    memory) is bounded in time.  With the host-side injection every tile's
    barrier expects 16 bytes more than its copies bring: the wait runs out
    after its limit (about a second), the tile is skipped, the call reports
    CPAPR_E_TIMEOUT (6), and the context stays usable.  Nothing faults."""
    T = synth.random_tensor((60, 50, 40), 3_000, 8, 91)
    lam, fs = model_for(T, 14)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, tile_nnz=4096, pi_mode=cpapr.CPAPR_PI_FUSED) as t:
        t.set_model(lam, fs)
        assert t.info().ntiles[0] == 1
        monkeypatch.setenv("CPAPR_FAULT_STAGE_WAIT", "1")
        with pytest.raises(cpapr.CpaprError) as e:
            t.phi(0)
        assert e.value.status == 6
        monkeypatch.delenv("CPAPR_FAULT_STAGE_WAIT")
        want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[0] * lam[None, :], 0)
        assert max_rel(t.phi(0), want) <= 1e-12


def test_tile_size_limits():
    """A tile's staged streams must fit in shared memory and start on 16-byte
    boundaries: the largest 3-way FP64 tile works, larger or odd sizes are
    argument errors, not faults."""
    T = case("c2s")
    lam, fs = model_for(T, 9)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, tile_nnz=8192) as t:
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[n] * lam[None, :], n)
            assert max_rel(t.phi(n), want) <= 1e-12
    for name, tile in (("c2s", 66), ("c2s", 16384), ("c5s64", 8192)):
        T = case(name)
        with pytest.raises(cpapr.CpaprError) as e:
            cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, tile_nnz=tile)
        assert e.value.status == 1, (name, tile)


def test_invalid_inputs_are_errors_not_faults():
    dims = (4, 3, 3)
    idx = np.array([[0, 1, 3], [0, 2, 1], [1, 1, 2]], dtype=np.int64)
    vals = np.array([1.0, 2.0, 3.0])
    bad = idx.copy()
    bad[1, 2] = 3
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.Tensor(dims, bad, vals, 2)
    assert e.value.status == 2
    bad = idx.copy()
    bad[0, 0] = -1
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.Tensor(dims, bad, vals, 2)
    assert e.value.status == 2
    for v in (-1.0, np.nan, np.inf):
        vv = vals.copy()
        vv[1] = v
        with pytest.raises(cpapr.CpaprError) as e:
            cpapr.Tensor(dims, idx, vv, 2)
        assert e.value.status == 3
    with cpapr.Tensor(dims, idx, vals, 2) as t:
        with pytest.raises(cpapr.CpaprError) as e:
            t.phi(0)
        assert e.value.status == 7
        fs = synth.random_factors(dims, 2, 1)
        fs[1][0, 0] = -0.5
        with pytest.raises(cpapr.CpaprError) as e:
            t.set_model(np.ones(2), fs)
        assert e.value.status == 3
        fs[1][0, 0] = 0.5
        t.set_model(np.ones(2), fs)
        with pytest.raises(cpapr.CpaprError) as e:
            t.phi(3)
        assert e.value.status == 1
        t.phi(2)


@pytest.mark.parametrize("precision", [cpapr.CPAPR_FP64, cpapr.CPAPR_FP32])
@pytest.mark.parametrize("pi_mode", PI_MODES)
def test_l2_persist_window_changes_no_result(precision, pi_mode):
    """The persisting-L2 window over the factor matrices only changes cache
    priorities: Phi, MTTKRP, the log-likelihood and a short MU solve are
    bit-identical with and without it, and the info block reports the window
    (the factors fit the device's window on this workload)."""
    T = case("c2s")
    lam, fs = model_for(T, 15)
    out = {}
    for l2 in (0, 1):
        with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, pi_mode=pi_mode, l2_persist=l2) as t:
            info = t.info()
            if l2:
                factor_bytes = sum(d * info.rank_padded * (8 if precision == cpapr.CPAPR_FP64 else 4) for d in T.dims)
                assert factor_bytes <= info.l2_window_bytes <= factor_bytes + 256 * T.nmodes
            else:
                assert info.l2_window_bytes == 0
            t.set_model(lam, fs)
            phis = [t.phi(n) for n in range(T.nmodes)]
            mtt = [t.mttkrp(n) for n in range(T.nmodes)]
            ll = t.loglik()
            r = t.mu_solve(tol=1e-4, max_outer=2, max_inner=3)
            out[l2] = (phis, mtt, ll, r, t.get_model(), t.loglik())
    a, b = out[0], out[1]
    for x, y in zip(a[0] + a[1], b[0] + b[1]):
        assert np.array_equal(x, y)
    assert a[2] == b[2] and a[5] == b[5]
    assert a[3]["total_inner"] == b[3]["total_inner"]
    assert np.array_equal(a[4][0], b[4][0])
    for x, y in zip(a[4][1], b[4][1]):
        assert np.array_equal(x, y)


def test_torch_device_buffers_and_stream():
    """The boundary tells host from device buffers by their attributes: a
    context on torch's current stream takes its model from CUDA tensors and
    writes Phi, MTTKRP and the model into CUDA tensors, with the same values
    as through host arrays."""
    import ctypes
    import torch
    T = case("c1")
    lam, fs = model_for(T, 24)
    stream = torch.cuda.current_stream()
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as h:
        h.set_model(lam, fs)
        want_phi = [h.phi(n) for n in range(T.nmodes)]
        want_mtt = [h.mttkrp(n) for n in range(T.nmodes)]
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, stream=stream.cuda_stream) as t:
        t.set_model(torch.from_numpy(lam).cuda(), [torch.from_numpy(np.ascontiguousarray(A)).cuda() for A in fs])
        for n in range(T.nmodes):
            out = torch.full((T.dims[n], T.rank), float("nan"), dtype=torch.float64, device="cuda")
            t.phi(n, out=out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), want_phi[n])
            out.fill_(float("nan"))
            t.mttkrp(n, out=out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), want_mtt[n])
        lam_d = torch.zeros(T.rank, dtype=torch.float64, device="cuda")
        fs_d = [torch.zeros((d, T.rank), dtype=torch.float64, device="cuda") for d in T.dims]
        arr = (ctypes.c_void_p * T.nmodes)(*[A.data_ptr() for A in fs_d])
        assert cpapr.load().cpapr_get_model(t.ctx, ctypes.c_void_p(lam_d.data_ptr()), arr) == 0
        torch.cuda.synchronize()
        assert np.array_equal(lam_d.cpu().numpy(), t.get_model()[0])
        for A, Ar in zip(fs_d, t.get_model()[1]):
            assert np.array_equal(A.cpu().numpy(), Ar)


@pytest.mark.parametrize("where", ["pinned", "cuda"])
def test_create_from_pinned_and_device_inputs(where):
    """The index build reads device inputs in place (no staging copy) and
    host ones, pinned or pageable, through a copy: the layouts, and so every
    Phi, are the same; invalid coordinates are reported as E_RANGE on every
    route."""
    import torch
    T = case("c2s")
    lam, fs = model_for(T, 25)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as h:
        h.set_model(lam, fs)
        want = [h.phi(n) for n in range(T.nmodes)]
    idx_t = torch.from_numpy(T.idx)
    val_t = torch.from_numpy(T.vals)
    if where == "pinned":
        idx_t, val_t = idx_t.pin_memory(), val_t.pin_memory()
    else:
        idx_t, val_t = idx_t.cuda(), val_t.cuda()
    with cpapr.Tensor(T.dims, [idx_t[m] for m in range(T.nmodes)], val_t, T.rank) as t:
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            assert np.array_equal(t.phi(n), want[n])
    bad = idx_t.clone()
    bad[1, 7] = T.dims[1]
    if where == "pinned":
        bad = bad.pin_memory()
    with pytest.raises(cpapr.CpaprError) as e:
        cpapr.Tensor(T.dims, [bad[m] for m in range(T.nmodes)], val_t, T.rank)
    assert e.value.status == 2


@pytest.mark.parametrize("precision", [cpapr.CPAPR_FP64, cpapr.CPAPR_FP32])
def test_mu_shift_moves_an_inadmissible_zero(precision):
    """Algorithm 1's B <- (A + S) Lambda with Chi and Kolda's shift: a factor
    entry set to exactly 0 stays 0 under B <- B * Phi; from the second outer
    iteration on, S adds kappa where A < kappa_tol and the previous Phi > 1,
    which moves it.  Same tiny tensor and model as the oracle's dense pin,
    three outer iterations against the oracle (FP64 at the MU-solve
    tolerances of these tests, FP32 at the FP32 ones)."""
    T = synth.random_tensor((5, 4, 3), 35, 3, 101)
    fs = synth.random_factors(T.dims, 3, 108)
    fs[0][1, 0] = 0.0
    lam = np.ones(3)
    kappa = 0.01
    ref = oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-12, max_outer=3, max_inner=4, kappa=kappa)
    assert ref["factors"][0][1, 0] > 0.0
    with cpapr.Tensor(T.dims, T.idx, T.vals, 3, precision=precision, kappa=kappa, tile_nnz=64) as t:
        t.set_model(lam, fs)
        r1 = t.mu_solve(tol=1e-12, max_outer=1, max_inner=4, trace=True, ll_trace=False)
        assert t.get_model()[1][0][1, 0] == 0.0  # no shift in the first outer iteration
        r2 = t.mu_solve(tol=1e-12, max_outer=2, max_inner=4, trace=True, ll_trace=False)
        lg, fg = t.get_model()
    assert fg[0][1, 0] > 0.0
    inner = np.concatenate([r1["inner"], r2["inner"]]).tolist()
    assert inner == ref["inner"].tolist()
    if precision == cpapr.CPAPR_FP64:
        np.testing.assert_allclose(lg, ref["lambda"], rtol=1e-10)
        for A, Ar in zip(fg, ref["factors"]):
            np.testing.assert_allclose(A, Ar, rtol=1e-9, atol=1e-14 * Ar.max())
    else:
        np.testing.assert_allclose(lg, ref["lambda"], rtol=1e-5)
        for A, Ar in zip(fg, ref["factors"]):
            np.testing.assert_allclose(A, Ar, rtol=1e-4, atol=1e-6 * Ar.max())


def _cache_lines(path):
    out = {}
    for line in path.read_text().splitlines():
        f = line.split()
        assert f[0] == "cpapr-tune-1" and len(f) == 7
        out[f[1]] = tuple(int(x) for x in f[2:6])  # the last line of a key wins
    return out


@pytest.mark.parametrize("precision,tol", [(cpapr.CPAPR_FP64, 1e-12), (cpapr.CPAPR_FP32, 1e-5)])
def test_tune_cache_written_then_reused(tmp_path, precision, tol):
    """autotune with a cache file times every mode once and appends one line
    per mode; a second context of the same tensor with autotune off reads the
    cached (lanes, tile, reduction, Pi form) for every mode without timing,
    and its Phi matches the oracle."""
    T = case("c3s")
    lam, fs = model_for(T, 23)
    path = tmp_path / "tune.txt"
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, autotune=1, tune_cache=str(path)) as t:
        first = t.info()
    lines = path.read_text().splitlines()
    assert len(lines) == T.nmodes
    cached = _cache_lines(path)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, precision=precision, tune_cache=str(path)) as t:
        info = t.info()
        got = {(info.rank_lanes[n], info.tile_nnz[n], info.reduction[n],
                int(info.pi_mode[n] == cpapr.CPAPR_PI_MATERIALISED)) for n in range(T.nmodes)}
        assert got <= set(cached.values())
        if len(cached) == T.nmodes:  # every mode its own class: the same choices as the timed context
            for n in range(T.nmodes):
                assert (info.rank_lanes[n], info.tile_nnz[n], info.reduction[n], info.pi_mode[n]) == (
                    first.rank_lanes[n], first.tile_nnz[n], first.reduction[n], first.pi_mode[n])
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[n] * lam[None, :], n)
            assert max_rel(t.phi(n), want) <= tol, n
    assert path.read_text().splitlines() == lines  # a hit times nothing and writes nothing


def test_tune_cache_ignores_lines_that_do_not_fit(tmp_path):
    """A cache line with a choice this tensor cannot run (a lanes count its
    rank does not allow, a tile too large for shared memory) or that does not
    parse is ignored: the context keeps the heuristic and works."""
    T = case("c2s")
    lam, fs = model_for(T, 24)
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank) as t:
        heur = t.info()
    path = tmp_path / "bad.txt"
    # learn this tensor's keys by tuning into a scratch file
    probe = tmp_path / "probe.txt"
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, autotune=1, tune_cache=str(probe)):
        pass
    keys = list(_cache_lines(probe))
    path.write_text("garbage line\n" + "".join(f"cpapr-tune-1 {k} 3 1048576 2 0 1.0\n" for k in keys))
    with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, tune_cache=str(path)) as t:
        info = t.info()
        assert list(info.tile_nnz[:3]) == list(heur.tile_nnz[:3])
        assert list(info.rank_lanes[:3]) == list(heur.rank_lanes[:3])
        t.set_model(lam, fs)
        want = oracle.phi(T.dims, T.idx, T.vals, fs, fs[0] * lam[None, :], 0)
        assert max_rel(t.phi(0), want) <= 1e-12


@pytest.mark.parametrize("pi_mode", PI_MODES)
def test_fp64_dot_fallbacks_match_oracle(pi_mode):
    """The FP64 form takes the dot <B, pi> on the FP32 pipe (operands cut into
    48-bit hi/lo float pairs).  Where an operand is 2^31 or more the group
    redoes its batch with the FP64 dot, and with eps below 2^-43 the FP64 dot
    is used throughout; both paths against the oracle at the FP64 bound, with
    B entries spread from 1e-40 to 1e12."""
    T = case("c3s")
    lam, fs = model_for(T, 31)
    rng = np.random.default_rng(5)
    for n in range(T.nmodes):
        B = fs[n] * 10.0 ** rng.uniform(-30, 12, size=fs[n].shape)
        B[::7, 0] = 2.0 ** 40  # rows whose batches fall back to the FP64 dot
        B[1::11, 1] = 1e-40    # entries below the float range (dropped parts)
        with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, pi_mode=pi_mode, fp64_dot=cpapr.CPAPR_DOT_FP32_PIPE) as t:
            t.set_model(lam, fs)
            want = oracle.phi(T.dims, T.idx, T.vals, fs, B, n)
            assert max_rel(t.phi(n, B=B), want) <= 1e-12, n
        with cpapr.Tensor(T.dims, T.idx, T.vals, T.rank, pi_mode=pi_mode, eps=1e-20,
                          fp64_dot=cpapr.CPAPR_DOT_FP32_PIPE) as t:
            t.set_model(lam, fs)
            want = oracle.phi(T.dims, T.idx, T.vals, fs, B, n, eps=1e-20)
            assert max_rel(t.phi(n, B=B), want) <= 1e-12, n


@pytest.mark.parametrize("pi_mode", PI_MODES)
def test_fp64_division_value_range_matches_oracle(pi_mode):
    """On the FP32 pipe the FP64 form also divides x / max(s, eps); values
    outside {0} and [2^-20, 2^31) make their group redo the batch with the
    FP64 dot and division.  Tensor values from 1e-30 to 4e9 (exact zeros,
    values at both edges of the range) against the oracle at the FP64 bound."""
    T = case("c3s")
    lam, fs = model_for(T, 32)
    rng = np.random.default_rng(6)
    vals = T.vals * 10.0 ** rng.uniform(-8, 6, size=T.vals.shape)
    vals[::13] = 0.0
    vals[1::17] = 1e-30
    vals[2::19] = 2.0 ** -20
    vals[3::23] = 2.0 ** 31
    vals[4::29] = 4e9
    vals[5::31] = 2.0 ** 31 - 2.0 ** 8
    with cpapr.Tensor(T.dims, T.idx, vals, T.rank, pi_mode=pi_mode, fp64_dot=cpapr.CPAPR_DOT_FP32_PIPE) as t:
        t.set_model(lam, fs)
        for n in range(T.nmodes):
            want = oracle.phi(T.dims, T.idx, vals, fs, fs[n] * lam[None, :], n)
            assert max_rel(t.phi(n), want) <= 1e-12, n
