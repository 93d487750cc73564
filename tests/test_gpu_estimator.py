"""The scikit-learn-style front end (paper_2407_06434_gb300.estimator) on the GPU, against the
FP64 oracle: orthogonal_mp with a fixed number of atoms (one and several targets) and with
scikit-learn's tol (squared residual norm, absolute), and the estimator's fit / predict with and
without the intercept."""
import numpy as np
import pytest

from oracle import omp as oracle
from workloads import gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_06434_gb300 import build
    build.build()
    from paper_2407_06434_gb300 import omp
    omp.load()
    return omp


def _dense(ref, N):
    C = np.zeros((ref.support.shape[0], N))
    for b in range(C.shape[0]):
        k = int(ref.n_iter[b])
        C[b, ref.support[b, :k]] = ref.coef[b, :k]
    return C


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_orthogonal_mp_fixed_sparsity(prec):
    from paper_2407_06434_gb300 import orthogonal_mp
    w = gen.get_config("gaussian_64x256_s8_b16")
    A = gen.dictionary(w)
    Y, *_ = gen.signals(w, A)
    ref = oracle.omp_batch(A, Y, w.S)
    coef = orthogonal_mp(A, Y.T, n_nonzero_coefs=w.S, precision=prec)
    assert coef.shape == (w.N, w.B)
    want = _dense(ref, w.N)
    np.testing.assert_allclose(coef.T, want, rtol=0, atol=1e-4 * np.abs(want).max())
    assert np.array_equal(coef.T != 0, want != 0)
    one, n = orthogonal_mp(A, Y[3], n_nonzero_coefs=w.S, precision=prec, return_n_iter=True)
    assert one.shape == (w.N,) and n == w.S
    np.testing.assert_allclose(one, coef[:, 3], rtol=0, atol=0)


def test_orthogonal_mp_tol_is_squared_residual():
    """tol bounds ||r||^2 (absolute): the iteration counts and coefficients are the oracle's with
    the absolute stop ||r|| <= sqrt(tol)."""
    from paper_2407_06434_gb300 import orthogonal_mp
    w = gen.get_config("gaussian_64x256_s8_b16", M=128, N=512, B=64, S=64, s_min=3, s_max=12,
                       sigma=1e-5, col_scale=1.0)
    A = gen.dictionary(w, seed=17)
    Y, *_ = gen.signals(w, A, seed=17)
    tol = 1e-4
    coef, n_iter = orthogonal_mp(A, Y.T, tol=tol, precision="fp32", return_n_iter=True)
    ref = oracle.omp_batch(A, Y, min(w.M, w.N), np.sqrt(tol), eps_relative=False)
    assert np.mean(n_iter == ref.n_iter) >= 0.95
    same = n_iter == ref.n_iter
    want = _dense(ref, w.N)
    err = np.linalg.norm(coef.T[same] - want[same], axis=1) / np.linalg.norm(want[same], axis=1)
    assert err.max() <= 1e-4
    r = Y.T - A @ coef
    assert np.all(np.sum(r * r, axis=0)[same] <= tol * (1 + 1e-3))


def test_estimator_fit_predict():
    from paper_2407_06434_gb300 import OrthogonalMatchingPursuit, orthogonal_mp
    w = gen.get_config("gaussian_64x256_s8_b16")
    A = gen.dictionary(w).astype(np.float64)
    Y, *_ = gen.signals(w, A.astype(np.float32))
    y = Y[0].astype(np.float64)
    est = OrthogonalMatchingPursuit(n_nonzero_coefs=8, fit_intercept=False, precision="fp32")
    est.fit(A, y)
    np.testing.assert_allclose(est.coef_, orthogonal_mp(A, y, n_nonzero_coefs=8, precision="fp32"),
                               rtol=0, atol=0)
    assert est.intercept_ == 0.0 and est.n_iter_ == 8
    np.testing.assert_allclose(est.predict(A), A @ est.coef_)
    # with the intercept: the oracle on centred data, intercept = mean(y) - mean(X) coef
    est = OrthogonalMatchingPursuit(n_nonzero_coefs=8, precision="fp32").fit(A, Y[:4].T)
    Ac = A - A.mean(axis=0)
    Yc = Y[:4].astype(np.float64) - Y[:4].mean(axis=1, keepdims=True)
    ref = oracle.omp_batch(Ac.astype(np.float32), Yc.astype(np.float32), 8)
    want = _dense(ref, w.N)
    np.testing.assert_allclose(est.coef_, want, rtol=0, atol=1e-4 * np.abs(want).max())
    y_mean = Y[:4].astype(np.float64).mean(axis=1)
    np.testing.assert_allclose(est.intercept_, y_mean - est.coef_ @ A.mean(axis=0), rtol=1e-6,
                               atol=1e-7 * np.abs(Y[:4]).max())
    pred = est.predict(A)
    assert pred.shape == (w.M, 4)
    assert np.linalg.norm(pred - Y[:4].T) <= 1e-3 * np.linalg.norm(Y[:4])
