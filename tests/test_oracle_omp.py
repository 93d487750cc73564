"""Pins for the FP64 OMP oracle against facts that do not come from the oracle itself:
hand-worked examples, brute force over all supports, closed forms, a recovery theorem,
statistical recovery, invariants and equivariances (paper Alg. 1, Sec. 2.1, Sec. 2.3, App. A)."""
import itertools

import numpy as np
import pytest
import scipy.linalg

from oracle import omp
from tests import golden_util
from workloads import gen

MODES = ["reference", "batch", "inverse_cholesky"]


def run_mode(mode, A, y, S, eps=0.0, eps_relative=True):
    if mode == "reference":
        return omp.omp_reference(A, y, S, eps, eps_relative)
    if mode == "batch":
        return omp.omp_batch(A, y[None, :], S, eps, eps_relative)
    return omp.omp_inverse_cholesky(A, y, S, eps, eps_relative)[0]


# ---------------------------------------------------------------- hand-worked examples
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", golden_util.FIXTURES)
def test_golden_examples(name, mode):
    d = golden_util.load(name)
    r = run_mode(mode, d["A"], d["y"], d["S"], d["eps"])
    k = d["n_iter"]
    assert r.n_iter[0] == k
    assert list(r.support[0, :k]) == d["support"]
    assert np.all(r.support[0, k:] == -1)
    np.testing.assert_allclose(r.coef[0, :k], d["coef"], atol=1e-12)
    np.testing.assert_allclose(r.resid_trace[0, :k], d["resid_trace"], atol=1e-12)
    if "margin" in d:
        np.testing.assert_allclose(r.margin[0, :k], d["margin"], atol=1e-12)
    if d.get("stop") == "dependent":
        assert r.stop[0] == omp.STOP_DEPENDENT


def test_zero_signal_gives_empty_support():
    A = gen.dictionary(gen.get_config("gaussian_64x256_s8_b16"))
    for mode in MODES:
        r = run_mode(mode, A, np.zeros(64), 8)
        assert r.n_iter[0] == 0 and np.all(r.support == -1) and np.all(r.coef == 0)
        assert r.stop[0] == omp.STOP_ZERO


# ---------------------------------------------------------------- brute force on tiny inputs
def _explicit_pick(A, r):
    """Selection by an explicit loop over atoms, strict '>' so the lowest index keeps a tie."""
    best, best_s = -1, -1.0
    for n in range(A.shape[1]):
        nrm = sum(v * v for v in A[:, n]) ** 0.5
        s = abs(sum(A[m, n] * r[m] for m in range(A.shape[0]))) / nrm
        if s > best_s:
            best, best_s = n, s
    return best


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_steps_tiny(seed):
    """Every step's pick equals an explicit loop over atoms, and x_k equals the normal-equations
    solution on S_k (an independent solve) for all three modes."""
    rng = np.random.default_rng(100 + seed)
    M, N, S = 6, 12, 3
    A = rng.standard_normal((M, N)) * rng.uniform(0.5, 2.0, size=N)
    y = rng.standard_normal(M)
    res = {m: run_mode(m, A, y, S) for m in MODES}
    r = y.copy()
    supp = []
    for k in range(S):
        n = _explicit_pick(A, r)
        supp.append(n)
        As = A[:, supp]
        x = np.linalg.solve(As.T @ As, As.T @ y)
        r = y - As @ x
        for m in MODES:
            assert res[m].support[0, k] == n, (m, k)
    for m in MODES:
        np.testing.assert_allclose(res[m].coef[0], x, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(res[m].resid_norm[0], np.linalg.norm(r), rtol=1e-10)


@pytest.mark.parametrize("seed", range(4))
def test_bruteforce_best_subset_noiseless(seed):
    """On noiseless planted inputs the minimum-residual S-subset (exhaustive over C(N,S)) is the
    planted one; OMP's final residual is 0 exactly when its support equals it."""
    rng = np.random.default_rng(200 + seed)
    M, N, S = 8, 14, 3
    A = rng.standard_normal((M, N))
    A /= np.linalg.norm(A, axis=0)
    planted = sorted(rng.choice(N, S, replace=False))
    y = A[:, planted] @ rng.standard_normal(S)
    best, best_r = None, np.inf
    for sub in itertools.combinations(range(N), S):
        As = A[:, sub]
        x = np.linalg.lstsq(As, y, rcond=None)[0]
        rr = np.linalg.norm(y - As @ x)
        if rr < best_r:
            best, best_r = sub, rr
    assert list(best) == planted
    for m in MODES:
        r = run_mode(m, A, y, S)
        found = sorted(r.support[0])
        if found == planted:
            assert r.resid_norm[0] < 1e-12 * np.linalg.norm(y)
        else:
            assert r.resid_norm[0] > 1e-6 * np.linalg.norm(y)


# ---------------------------------------------------------------- closed form
@pytest.mark.parametrize("mode", MODES)
def test_orthogonal_dictionary_closed_form(mode):
    """A orthogonal (N = M): OMP picks atoms by decreasing |(A^T y)_n| and x is those entries
    of A^T y; the residual norm is sqrt(||y||^2 - sum of their squares)."""
    rng = np.random.default_rng(7)
    M = 16
    Q = np.linalg.qr(rng.standard_normal((M, M)))[0]
    y = rng.standard_normal(M)
    c = Q.T @ y
    order = np.argsort(-np.abs(c), kind="stable")
    S = 6
    r = run_mode(mode, Q, y, S)
    assert list(r.support[0]) == list(order[:S])
    np.testing.assert_allclose(r.coef[0], c[order[:S]], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r.resid_norm[0], np.sqrt(np.sum(c ** 2) - np.sum(c[order[:S]] ** 2)),
                               rtol=1e-10)


# ---------------------------------------------------------------- recovery theorem
def test_hadamard_exact_recovery():
    """A = [I | H/sqrt(M)] has coherence mu = 1/sqrt(M) = 1/8 at M = 64. Tropp's exact recovery
    condition mu < 1/(2S-1) holds for S <= 4, so OMP recovers every such support exactly
    (noiseless), whatever the coefficients."""
    M = 64
    A = np.hstack([np.eye(M), scipy.linalg.hadamard(M) / np.sqrt(M)])
    rng = np.random.default_rng(11)
    for trial in range(200):
        S = 1 + trial % 4
        supp = rng.choice(2 * M, S, replace=False)
        x = rng.standard_normal(S) * rng.choice([1e-3, 1.0, 1e3], size=S)
        y = A[:, supp] @ x
        r = omp.omp_batch(A, y[None], S)
        assert set(r.support[0]) == set(supp)
        got = dict(zip(r.support[0], r.coef[0]))
        np.testing.assert_allclose([got[s] for s in supp], x, rtol=1e-9, atol=1e-12)


def test_statistical_recovery_gaussian_64x256():
    """Gaussian 64 x 256, S = 8, noiseless: recovery >= 99% over 1000 seeded trials, and all 16
    signals of the seed-0 batch are recovered."""
    w = gen.get_config("gaussian_64x256_s8_b16")
    A = gen.dictionary(w)
    Y, sp, sup, coef = gen.signals(w, A)
    r = omp.omp_batch(A, Y, w.S)
    assert all(set(r.support[b]) == set(sup[b]) for b in range(w.B))
    w2 = gen.get_config("gaussian_64x256_s8_b16", B=1000)
    Y2, _, sup2, _ = gen.signals(w2, A, seed=1)
    r2 = omp.omp_batch(A, Y2, w2.S)
    rate = np.mean([set(r2.support[b]) == set(sup2[b]) for b in range(w2.B)])
    assert rate >= 0.99, rate


# ---------------------------------------------------------------- invariants
def test_invariants_noisy():
    """For every k: |A_{S_k}^T r_k|_inf <= 1e-10 ||y|| (orthogonality of the residual, Sec. 4.4 of
    the paper reports ~1e-15), ||r_k|| non-increasing, ||r_k||^2 + ||A_S x_k||^2 = ||y||^2."""
    rng = np.random.default_rng(3)
    M, N = 32, 80
    A = rng.standard_normal((M, N))
    Y = rng.standard_normal((5, M))
    for S in range(1, 11):
        r = omp.omp_batch(A, Y, S)
        for b in range(Y.shape[0]):
            s = r.support[b][r.support[b] >= 0]
            As = A[:, s]
            fit = As @ r.coef[b, : len(s)]
            res = Y[b] - fit
            yn = np.linalg.norm(Y[b])
            assert np.max(np.abs(As.T @ res)) <= 1e-10 * yn
            assert abs(res @ res + fit @ fit - yn ** 2) <= 1e-12 * yn ** 2
            assert abs(np.linalg.norm(res) - r.resid_norm[b]) <= 1e-12 * yn
            tr = r.resid_trace[b, : r.n_iter[b]]
            assert np.all(np.diff(tr) <= 1e-12 * yn)


def test_modes_agree_with_eps_stop():
    """Timed (progressive Cholesky), reference (lstsq) and inverse-Cholesky modes agree on
    supports, iteration counts and coefficients (1e-12 relative), with relative and absolute
    eps stops."""
    w = gen.get_config("gaussian_64x256_s8_b16", B=12, s_min=2, s_max=12, sigma=1e-2)
    A = gen.dictionary(w, seed=5)
    Y, *_ = gen.signals(w, A, seed=5)
    for eps, rel in [(0.05, True), (0.3, False), (0.0, True)]:
        rb = omp.omp_batch(A, Y, 16, eps, rel)
        for b in range(w.B):
            for m in ["reference", "inverse_cholesky"]:
                ro = run_mode(m, A, Y[b], 16, eps, rel)
                assert ro.n_iter[0] == rb.n_iter[b]
                assert np.array_equal(ro.support[0], rb.support[b])
                assert ro.stop[0] == rb.stop[b]
                scale = np.linalg.norm(rb.coef[b]) + 1e-300
                assert np.linalg.norm(ro.coef[0] - rb.coef[b]) <= 1e-12 * scale * 10


def test_inverse_cholesky_factor_identities():
    """F_k = V_k^{-T} with V_k the Cholesky factor of A_k^T A_k (Sec. 2.3), hence
    F_k^T (A_k^T A_k) F_k = I; checked against LAPACK's Cholesky (numpy.linalg.cholesky)."""
    rng = np.random.default_rng(9)
    M, N, S = 40, 120, 12
    A = rng.standard_normal((M, N)) * rng.uniform(0.5, 2, size=N)
    y = rng.standard_normal(M)
    r, F = omp.omp_inverse_cholesky(A, y, S)
    As = A[:, r.support[0]]
    G = As.T @ As
    V = np.linalg.cholesky(G)
    np.testing.assert_allclose(F @ V.T, np.eye(S), atol=1e-12)
    np.testing.assert_allclose(F.T @ G @ F, np.eye(S), atol=1e-12)
    assert np.allclose(F, np.triu(F))


# ---------------------------------------------------------------- equivariances
def test_equivariances():
    """Column permutation permutes the support; flipping a column's sign flips its coefficient;
    scaling column n by d_n leaves the support unchanged and divides its coefficient by d_n
    (App. A: the method is invariant to column norms)."""
    rng = np.random.default_rng(21)
    M, N, S = 30, 90, 8
    A = rng.standard_normal((M, N))
    Y = rng.standard_normal((4, M))
    base = omp.omp_batch(A, Y, S)
    perm = rng.permutation(N)
    inv = np.argsort(perm)
    rp = omp.omp_batch(A[:, perm], Y, S)
    assert np.array_equal(perm[rp.support], base.support)
    np.testing.assert_allclose(rp.coef, base.coef, rtol=1e-10, atol=1e-12)
    sign = rng.choice([-1.0, 1.0], size=N)
    rs = omp.omp_batch(A * sign, Y, S)
    assert np.array_equal(rs.support, base.support)
    np.testing.assert_allclose(rs.coef, base.coef * sign[base.support], rtol=1e-10, atol=1e-12)
    d = rng.uniform(0.5, 2.0, size=N)
    rd = omp.omp_batch(A * d, Y, S)
    assert np.array_equal(rd.support, base.support)
    np.testing.assert_allclose(rd.coef, base.coef / d[base.support], rtol=1e-10, atol=1e-12)
    assert inv.shape == perm.shape


def test_replay_support_matches_run():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((20, 50))
    y = rng.standard_normal(20)
    r = omp.omp_reference(A, y, 6)
    x, rn = omp.replay_support(A, y, r.support[0])
    np.testing.assert_allclose(x, r.coef[0], rtol=1e-12)
    np.testing.assert_allclose(rn, r.resid_trace[0], rtol=1e-12)


def test_generator_planted_model():
    """The generator's y equals A_S x + noise for the planted (support, coef); rows regenerate
    identically in any slice; columns have unit norm."""
    w = gen.get_config("gaussian_64x256_s8_b16", B=600, sigma=1e-3)
    A = gen.dictionary(w)
    np.testing.assert_allclose(np.linalg.norm(A.astype(np.float64), axis=0), 1.0, atol=1e-6)
    Y, sp, sup, coef = gen.signals(w, A)
    Ys, *_ = gen.signals(w, A, rows=slice(250, 530))
    assert np.array_equal(Ys, Y[250:530])
    fit = np.stack([A[:, sup[b]].astype(np.float64) @ coef[b] for b in range(w.B)])
    resid = Y - fit
    assert abs(np.std(resid) - 1e-3) < 1e-4
    wc = gen.get_config("coherent_4096x32768_s64_b16384", M=256, N=512, B=4)
    Ac = gen.dictionary(wc).astype(np.float64)
    G = Ac.T @ Ac
    top = np.sort(np.abs(G - np.eye(512)), axis=1)[:, -1]
    assert abs(np.median(top) - 0.3) < 0.1
