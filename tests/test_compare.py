"""The parity rules themselves (oracle.compare), on CPU: the oracle's own result passes; a pick
that differs at a clear margin, a near-tie pick that scores below (1 - 1e-3) of the best, a bad
pick after a legitimate near-tie, wrong coefficients or residuals, and a wrong stopping step are
each caught; a legitimate near-tie divergence is accepted and checked on its own support."""
import numpy as np
import pytest

from oracle import compare, omp


def _near_tie_problem(seed=3, M=40, N=120, s=5, eps_pert=1e-6):
    """Atom 1 is a 1e-6 perturbation of atom 0 (renormalised); y uses atom 0 with the largest
    coefficient, so the first step is a near-tie between atoms 0 and 1."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, N))
    A[:, 1] = A[:, 0] + eps_pert * rng.standard_normal(M)
    A /= np.linalg.norm(A, axis=0)
    sup = np.concatenate([[0], rng.choice(np.arange(2, N), s - 1, replace=False)])
    x = np.array([5.0, 1.0, -0.9, 0.8, 0.7])[:s]
    y = A[:, sup] @ x + 1e-4 * rng.standard_normal(M)
    return A, y[None, :]


def _next_pick(A, y, picks):
    """Alg. 1's pick after the given prefix (the scores of its least-squares residual)."""
    scores, _ = omp.prefix_scores(A, y, list(picks) + [0])
    return int(np.argmax(scores[len(picks)]))


def _result_from(A, Y, S, support):
    """Coefficients, residual norms and iteration counts of the least squares on given supports."""
    B = Y.shape[0]
    X = np.zeros((B, S))
    sup = np.full((B, S), -1)
    rn = np.zeros(B)
    for b in range(B):
        k = len(support[b])
        x, r = omp.replay_support(A, Y[b], support[b])
        X[b, :k], sup[b, :k] = x, support[b]
        rn[b] = r[-1] if k else np.linalg.norm(Y[b])
    return sup, X, np.array([len(s) for s in support]), rn


def test_oracle_result_passes():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((30, 80))
    Y = rng.standard_normal((6, 30))
    ref = omp.omp_batch(A, Y, 6)
    st = compare.compare(A, Y, ref, ref.support, ref.coef, ref.n_iter, ref.resid_norm)
    assert st["tie_diverged"] == 0 and st["max_coef_rel"] < 1e-10 and not st["violations"]


def test_clear_margin_difference_fails():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((30, 80))
    Y = rng.standard_normal((1, 30))
    ref = omp.omp_batch(A, Y, 4)
    picks = list(ref.support[0])
    assert ref.margin[0, 2] > 1e-3
    scores, _ = omp.prefix_scores(A, Y[0], picks)
    picks[2] = int(np.argsort(scores[2])[-2])      # the runner-up at a clear margin
    sup, X, n, rn = _result_from(A, Y, 4, [picks])
    with pytest.raises(compare.ParityError, match="margin"):
        compare.compare(A, Y, ref, sup, X, n, rn)
    st = compare.compare(A, Y, ref, sup, X, n, rn, strict=False)
    assert st["violations"] and compare.error_report(st)["mismatch_rate_at_margin_gt_1e-3"] == 1.0


def test_near_tie_divergence_is_accepted_and_replayed():
    A, Y = _near_tie_problem()
    ref = omp.omp_batch(A, Y, 5)
    assert ref.margin[0, 0] < 1e-3 and ref.support[0, 0] in (0, 1)
    other = 1 - ref.support[0, 0]
    # the result takes the other atom of the near-tie, then continues greedily on its own support
    picks = [other]
    for t in range(1, 5):
        picks.append(_next_pick(A, Y[0], picks))
    sup, X, n, rn = _result_from(A, Y, 5, [picks])
    st = compare.compare(A, Y, ref, sup, X, n, rn)
    assert st["tie_diverged"] == 1 and st["off_greedy_steps"] == 1
    # a wrong pick later on the diverged support is caught
    scores, _ = omp.prefix_scores(A, Y[0], picks)
    bad = picks[:3] + [int(np.argsort(scores[3])[-2])]
    bad.append(_next_pick(A, Y[0], bad))
    s3 = np.sort(scores[3])
    assert (s3[-1] - s3[-2]) / s3[-1] > 1e-3
    sup, X, n, rn = _result_from(A, Y, 5, [bad])
    with pytest.raises(compare.ParityError, match="step 3"):
        compare.compare(A, Y, ref, sup, X, n, rn)


def test_near_tie_pick_must_score_within_the_margin():
    """At a near-tie step the result's atom must itself be one of the near-tied atoms: a third
    atom that scores far below the best fails even though the oracle's margin is tiny."""
    A, Y = _near_tie_problem(seed=4)
    ref = omp.omp_batch(A, Y, 5)
    assert ref.margin[0, 0] < 1e-3
    s0 = np.abs(A.T @ Y[0]) / np.linalg.norm(A, axis=0)
    third = int(np.argsort(s0)[-3])
    assert s0[third] < 0.999 * s0.max()
    picks = [third]
    for t in range(1, 5):
        picks.append(_next_pick(A, Y[0], picks))
    sup, X, n, rn = _result_from(A, Y, 5, [picks])
    with pytest.raises(compare.ParityError, match="step 0"):
        compare.compare(A, Y, ref, sup, X, n, rn)


def test_coefficient_and_residual_tolerances():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 80))
    Y = rng.standard_normal((2, 30))
    ref = omp.omp_batch(A, Y, 5)
    X = ref.coef.copy()
    X[1, 2] *= 1 + 3e-4
    with pytest.raises(compare.ParityError, match="coefficient"):
        compare.compare(A, Y, ref, ref.support, X, ref.n_iter, ref.resid_norm)
    rn = ref.resid_norm * (1 + 3e-4)
    with pytest.raises(compare.ParityError, match="residual"):
        compare.compare(A, Y, ref, ref.support, ref.coef, ref.n_iter, rn)
    st = compare.compare(A, Y, ref, ref.support, ref.coef, ref.n_iter,
                         ref.resid_norm * (1 + 5e-5))
    assert 0.4 < st["max_resid_over_tol"] < 0.6


def test_stopping_step_on_a_diverged_support():
    """With an eps stop, a diverged signal must stop at the first step where the residual along
    its own support reaches eps: stopping one step late is caught."""
    A, Y = _near_tie_problem(seed=6, eps_pert=1e-7)
    eps = 1e-3
    ref = omp.omp_batch(A, Y, 10, eps)
    assert ref.margin[0, 0] < 1e-3
    picks = [1 - ref.support[0, 0]]
    while True:
        sc, rn = omp.prefix_scores(A, Y[0], picks)
        if rn[-1] <= eps * np.linalg.norm(Y[0]) or len(picks) == 10:
            break
        picks.append(_next_pick(A, Y[0], picks))
    k = len(picks)
    assert k < 10
    sup, X, n, rn = _result_from(A, Y, 10, [picks])
    compare.compare(A, Y, ref, sup, X, n, rn, eps=eps)
    late = picks + [_next_pick(A, Y[0], picks)]
    late_sup, late_X, late_n, late_rn = _result_from(A, Y, 10, [late])
    with pytest.raises(compare.ParityError):
        compare.compare(A, Y, ref, late_sup, late_X, late_n, late_rn, eps=eps)


def test_prefix_scores_match_alg1_residuals():
    """prefix_scores along the oracle's own support reproduces the oracle's residual trace and
    picks the oracle's atom at every step."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((25, 60))
    y = rng.standard_normal(25)
    ref = omp.omp_reference(A, y, 6)
    sc, rn = omp.prefix_scores(A, y, ref.support[0])
    assert list(np.argmax(sc, axis=1)) == list(ref.support[0])
    np.testing.assert_allclose(rn[1:], ref.resid_trace[0], rtol=1e-12)
    assert abs(rn[0] - np.linalg.norm(y)) < 1e-12
