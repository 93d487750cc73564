"""Full-size workloads on the GPU (graph replay, the benchmark's launch configuration), checked
against the FP64 oracle on 1024 seeded signals of each batch (every signal when the batch is
smaller) with the parity rules of oracle/compare.py: identical supports wherever the oracle's
top-two margin exceeds 1e-3, every pick after a near-tie valid along the result's own support,
coefficients and residual norms within 1e-4.

- uneven batching: 2048 x 16384, B = 8192, sparsity 4..128, eps = 1e-3 relative, S = 128, at
  noise sigma = 1e-3 (the eps stop never fires) and sigma = 1e-6 (it fires near k = s);
- coherent dictionary: 4096 x 32768 (pairs at correlation ~0.3), B = 16384, S = 64, FP8 E4M3
  correlation with FP32 rescoring;
- 1024 x 8192, B = 16384, S = 48 (the learned-proposal workload, dense path);
- the paper's three application shapes with synthetic data: 256 x 1024 (S = 32, B = 5000),
  8064 x 1207 (S = 30, B = 1200), 512 x 2048 (S = 64, B = 5000)."""
import numpy as np
import pytest

from oracle import omp as oracle
from tests import parity
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


N_CHECK = 1024


def check_rows(B, n=N_CHECK, seed=0):
    """The seeded sample of signals checked against the oracle (all of them when B <= n)."""
    if B <= n:
        return np.arange(B)
    return np.sort(np.random.default_rng(seed).choice(B, n, replace=False))


def run_config(name, prec, n_check=N_CHECK, solver_kw=None, **overrides):
    from paper_2407_06434_gb300 import omp
    w = gen.get_config(name, **overrides)
    A = gen.dictionary(w)
    Y, sp, sup, coef = gen.signals(w, A)
    s = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision=prec, **(solver_kw or {}))
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    X, S_, n_iter, resid, stop = s.solve(Ad, torch.from_numpy(Y).cuda(), w.S, w.eps, diagnostics=True)
    torch.cuda.synchronize()
    X, S_, n_iter, resid = X.cpu().numpy(), S_.cpu().numpy(), n_iter.cpu().numpy(), resid.cpu().numpy()
    s.close()
    rows = check_rows(w.B, n_check)
    ref = oracle.omp_batch(A, Y[rows], w.S, w.eps, True)
    st = parity.compare(A, Y[rows], ref, S_[rows], X[rows], n_iter[rows], resid[rows], eps=w.eps,
                        rows=rows)
    return w, st, n_iter, S_, sup


def test_uneven_batch_2048x16384_bf16():
    w, st, n_iter, S_, sup = run_config("gaussian_2048x16384_s4to128_b8192", "bf16")
    assert st["tie_diverged"] <= 0.02 * st["signals"], st
    assert np.all(n_iter == w.S)                      # the noise floor stays above eps ||y||


def test_uneven_batch_2048x16384_lownoise_bf16():
    w, st, n_iter, S_, sup = run_config("gaussian_2048x16384_s4to128_b8192_lownoise", "bf16")
    assert st["tie_diverged"] <= 0.02 * st["signals"], st
    sp = np.sum(sup >= 0, axis=1)
    assert np.mean(np.abs(n_iter - sp) <= 2) > 0.9     # the eps stop fires near k = s


def test_coherent_4096x32768_fp8():
    w, st, n_iter, S_, sup = run_config("coherent_4096x32768_s64_b16384", "fp8")
    assert st["tie_diverged"] <= 0.02 * st["signals"], st
    assert np.all(n_iter == w.S)


def test_coherent_4096x32768_fp8_gather24():
    """The same workload with the update's atom-row gather reading the 24-bit copy of A (3 bytes
    per element): the same parity bar against the FP64 oracle."""
    w, st, n_iter, S_, sup = run_config("coherent_4096x32768_s64_b16384", "fp8",
                                        solver_kw=dict(gather24=True))
    assert st["tie_diverged"] <= 0.02 * st["signals"], st
    assert np.all(n_iter == w.S)
    assert st["max_coef_rel"] <= 1e-4


def test_learned_workload_dense_1024x8192_s48():
    w, st, n_iter, S_, sup = run_config("gaussian_1024x8192_s48_b16384", "bf16")
    assert st["tie_diverged"] <= 0.02 * st["signals"], st


@pytest.mark.parametrize("name", ["patches_256x1024_s32_b5000", "face_8064x1207_s30_b1200",
                                  "audio_512x2048_s64_b5000"])
def test_paper_application_shapes(name):
    w, st, n_iter, S_, sup = run_config(name, "bf16")
    assert st["tie_diverged"] <= 0.02 * st["signals"], st
