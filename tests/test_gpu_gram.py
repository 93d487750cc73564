"""Parity of the Gram-space solve (omp_solve_batch_gram: one FP32 GEMM for c = A^T y, then
per-step updates of c through the Gram matrix, Sec. 2.3's v0 family) with the FP64 oracle, on
the same cases as the dense loop: the hand-worked fixtures, the 64 x 256 planted batch, ragged
shapes, eps-stopped uneven batches (relative and absolute), zero and non-finite signals, and the
paper's three application shapes at full batch on sampled signals."""
import numpy as np
import pytest

from oracle import omp as oracle
from tests import golden_util, parity
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


def solve_gram(A, Y, S, eps=0.0, eps_relative=True, precision="fp32"):
    from paper_2407_06434_gb300 import omp
    M, N = A.shape
    B = Y.shape[0]
    s = omp.OmpSolver(M, N, max_batch=B, max_iters=S, precision=precision,
                      eps_relative=eps_relative)
    Ad = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float32).T)).cuda().t()
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    X, sup, n_iter, resid, stop = s.solve_gram(Ad, Yd, S, eps, diagnostics=True)
    torch.cuda.synchronize()
    out = dict(X=X.cpu().numpy(), sup=sup.cpu().numpy(), n_iter=n_iter.cpu().numpy(),
               resid=resid.cpu().numpy(), stop=stop.cpu().numpy())
    out["status"] = omp.omp_get_error(s.h)
    s.close()
    return out


@pytest.mark.parametrize("name", golden_util.FIXTURES)
def test_golden_fixtures(name):
    d = golden_util.load(name)
    A = d["A"].astype(np.float32)
    r = solve_gram(A, d["y"][None, :].astype(np.float32), d["S"])
    k = d["n_iter"]
    assert r["n_iter"][0] == k
    assert list(r["sup"][0, :k]) == d["support"]
    assert np.all(r["sup"][0, k:] == -1)
    np.testing.assert_allclose(r["X"][0, :k], d["coef"], rtol=1e-5, atol=1e-6)
    if d.get("stop") == "dependent":
        assert r["stop"][0] == oracle.STOP_DEPENDENT


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_planted_64x256_full(precision):
    w = gen.get_config("gaussian_64x256_s8_b16")
    A = gen.dictionary(w)
    Y, sp, sup, coef = gen.signals(w, A)
    ref = oracle.omp_batch(A, Y, w.S)
    r = solve_gram(A, Y, w.S, precision=precision)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"])
    assert st["tie_diverged"] == 0
    assert np.array_equal(r["sup"], ref.support)


def test_ragged_shapes():
    """M = 200 (padded), N = 1000 (not a multiple of the 256 threads), B = 301, S = 24, noisy."""
    w = gen.get_config("gaussian_64x256_s8_b16", M=200, N=1000, B=301, S=24, s_min=5, s_max=24,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=3)
    Y, *_ = gen.signals(w, A, seed=3)
    ref = oracle.omp_batch(A, Y, w.S)
    r = solve_gram(A, Y, w.S)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"])
    assert st["tie_diverged"] <= 3, st


@pytest.mark.parametrize("eps_relative", [True, False])
def test_eps_stop_uneven(eps_relative):
    w = gen.get_config("gaussian_64x256_s8_b16", M=256, N=2048, B=200, S=48, s_min=4, s_max=40,
                       sigma=1e-6, col_scale=1.0)
    A = gen.dictionary(w, seed=4)
    Y, sp, _, _ = gen.signals(w, A, seed=4)
    eps = 1e-3 if eps_relative else 5e-3
    ref = oracle.omp_batch(A, Y, w.S, eps, eps_relative)
    r = solve_gram(A, Y, w.S, eps=eps, eps_relative=eps_relative)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"], eps=eps,
                        eps_relative=eps_relative)
    assert np.mean(r["n_iter"] < w.S) > 0.9
    assert np.mean(r["stop"] == oracle.STOP_EPS) > 0.9
    assert st["tie_diverged"] <= 2, st


def test_zero_and_nonfinite_signals():
    w = gen.get_config("gaussian_64x256_s8_b16", B=20)
    A = gen.dictionary(w)
    Y, *_ = gen.signals(w, A)
    Y[3] = 0.0
    Y[7, 5] = np.nan
    Y[11, 0] = np.inf
    good = [b for b in range(w.B) if b not in (3, 7, 11)]
    ref = oracle.omp_batch(A, Y[good], w.S)
    r = solve_gram(A, Y, w.S)
    for b in (3, 7, 11):
        assert r["n_iter"][b] == 0 and np.all(r["sup"][b] == -1) and np.all(r["X"][b] == 0)
        assert r["stop"][b] == oracle.STOP_ZERO
    parity.compare(A, Y[good], ref, r["sup"][good], r["X"][good], r["n_iter"][good],
                   r["resid"][good])


def test_matches_the_dense_fp32_loop():
    """Both forms pick by the same FP32 scores up to rounding, so their supports agree except
    where a near-tie can go either way."""
    from paper_2407_06434_gb300 import omp
    w = gen.get_config("gaussian_64x256_s8_b16", M=256, N=1024, B=500, S=32, s_min=32, s_max=32,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=9)
    Y, *_ = gen.signals(w, A, seed=9)
    s = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="fp32")
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    Yd = torch.from_numpy(Y).cuda()
    _, sd = s.solve(Ad, Yd, w.S)
    _, sg = s.solve_gram(Ad, Yd, w.S)
    torch.cuda.synchronize()
    s.close()
    same = np.all(sd.cpu().numpy() == sg.cpu().numpy(), axis=1)
    assert np.mean(same) > 0.97


@pytest.mark.parametrize("name", ["patches_256x1024_s32_b5000", "face_8064x1207_s30_b1200",
                                  "audio_512x2048_s64_b5000"])
def test_paper_application_shapes(name):
    w = gen.get_config(name)
    A = gen.dictionary(w)
    Y, *_ = gen.signals(w, A)
    r = solve_gram(A, Y, w.S, eps=w.eps)
    rows = np.linspace(0, w.B - 1, 24).astype(int)
    ref = oracle.omp_batch(A, Y[rows], w.S, w.eps, True)
    st = parity.compare(A, Y[rows], ref, r["sup"][rows], r["X"][rows], r["n_iter"][rows],
                        r["resid"][rows], eps=w.eps, rows=rows)
    assert st["tie_diverged"] <= 3, st


def test_unsupported_size_is_refused():
    """Per-signal shared memory above 227 KB (25000 floats of c plus the S = 256 packed factor)
    is an argument error, returned before any launch."""
    from paper_2407_06434_gb300 import omp
    s = omp.OmpSolver(256, 25000, max_batch=4, max_iters=256, precision="fp32")
    A = torch.zeros((25000, 256), device="cuda").t()
    Y = torch.zeros((4, 256), device="cuda")
    with pytest.raises(omp.OmpError):
        s.solve_gram(A, Y, 8)
    s.close()
