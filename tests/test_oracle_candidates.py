"""Pins for the candidate-restricted OMP reference (oracle.omp.omp_candidates_reference) against
hand-worked examples whose numbers were derived on paper (tests/golden/candidates_*.json): the
residual-drop check is the normalised ENERGY drop (||r_{k-1}||^2 - ||r_k||^2) / ||r_{k-1}||^2
(taus placed between the energy drop and the norm ratio 1 - ||r_k|| / ||r_{k-1}|| tell the two
apart), a rejected step falls back to the full selection of Alg. 1 in the same step, and the
restricted score divides by the atom's norm (a dictionary with unequal column norms where leaving
the division out picks another atom)."""
import numpy as np
import pytest

from oracle import omp
from tests import golden_util


@pytest.mark.parametrize("name", golden_util.CANDIDATE_FIXTURES)
def test_candidate_fixtures(name):
    d = golden_util.load_candidates(name)
    for c in d["cases"]:
        r, fb = omp.omp_candidates_reference(d["A"], d["y"], d["S"], d["cand"], c["tau"], d["eps"])
        k = len(c["support"])
        assert fb == c["fallback"], c["name"]
        assert r.n_iter[0] == k, c["name"]
        assert list(r.support[0, :k]) == c["support"], c["name"]
        np.testing.assert_allclose(r.coef[0, :k], c["coef"], atol=1e-12, err_msg=c["name"])
        np.testing.assert_allclose(r.resid_trace[0, :k], c["resid_trace"], atol=1e-12,
                                   err_msg=c["name"])
        np.testing.assert_allclose(r.margin[0, :k], c["margin"], atol=1e-12, err_msg=c["name"])


def test_fixture_drops_are_energy_drops():
    """The hand-derived drops of the fallback fixture sit on the two sides of the taus exactly as
    the cases say (a check of the fixture itself, independent of the oracle)."""
    d = golden_util.load_candidates("candidates_fallback_3x4.json")
    fb, acc = d["cases"]
    drops = fb["drops"]
    assert drops[0] >= fb["tau"][0] and drops[1] < fb["tau"][1]
    assert drops[0] >= acc["tau"][0] and drops[1] >= acc["tau"][1]
    # the norm ratios would decide differently: 1 - sqrt(8/17) < 0.4 and 1 - 1/sqrt(2) < 0.45
    assert 1 - np.sqrt(8 / 17) < fb["tau"][0] and 1 - 1 / np.sqrt(2) < acc["tau"][1]


def test_mid_run_fallback_on_a_planted_signal():
    """A larger case with a fallback in mid-run: a 32 x 64 Gaussian dictionary, a planted 6-sparse
    noiseless signal, candidates = the planted support minus its atom with the smallest
    coefficient plus 10 decoys. The restricted iteration recovers the five remaining planted atoms
    (each drop is large), then at step 5 its best candidate is a decoy whose drop is small, so
    with tau_5 = 0.5 the step falls back, picks the missing atom among all atoms, and the final
    support equals the planted one with a zero residual -- the same result as Alg. 1."""
    rng = np.random.default_rng(21)
    M, N = 32, 64
    A = rng.standard_normal((M, N))
    A /= np.linalg.norm(A, axis=0)
    sup = rng.choice(N, 6, replace=False)
    x = np.array([3.0, -2.5, 2.0, 1.8, -1.5, 0.05])
    y = A[:, sup] @ x
    decoys = rng.choice(np.setdiff1d(np.arange(N), sup), 10, replace=False)
    cand = np.concatenate([sup[:5], decoys])
    tau = np.zeros(6)
    tau[5] = 0.5
    r, fb = omp.omp_candidates_reference(A, y, 6, cand, tau)
    ref = omp.omp_reference(A, y, 6)
    assert fb == 5
    assert set(r.support[0]) == set(sup)
    assert np.array_equal(r.support, ref.support)
    assert r.resid_norm[0] < 1e-12 * np.linalg.norm(y)
    # the same run without the fallback (tau = 0) keeps a decoy and leaves a residual
    r0, fb0 = omp.omp_candidates_reference(A, y, 6, cand, np.zeros(6))
    assert fb0 == -1 and r0.support[0, 5] in decoys and r0.resid_norm[0] > 1e-3
