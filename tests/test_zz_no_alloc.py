"""The allocation-free correlate-and-select entry point, for callers that cannot allocate
device memory (a fixed memory budget, or a framework that owns every device allocation).

It is checked through the C ABI against the handle-based entry point (omp_correlate_topk on an
FP32 handle) on two calls in a row with different inputs, so a second call that reused the
first call's scratch contents would show; both kernel variants (16-byte vector loads, and
scalar loads for unaligned buffers or M not a multiple of 4) are covered. This file is
collected last on purpose."""
import numpy as np
import pytest

from oracle import omp as oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_06434_gb300 import build
    build.build()
    from paper_2407_06434_gb300 import omp
    omp.load()
    return omp


def _handle_top1(omp, A, R):
    M, N = A.shape
    s = omp.OmpSolver(M, N, max_batch=R.shape[0], max_iters=1, precision="fp32")
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    idx = torch.empty((R.shape[0], 1), dtype=torch.int32, device="cuda")
    sc = torch.empty((R.shape[0], 1), dtype=torch.float32, device="cuda")
    omp.omp_correlate_topk(s.h, Ad, torch.from_numpy(R).cuda(), 1, idx, sc)
    out = idx.cpu().numpy()[:, 0], sc.cpu().numpy()[:, 0]
    s.close()
    return out


def test_noalloc_matches_handle_entry_point_on_two_calls(lib):
    omp = lib
    rng = np.random.default_rng(31)
    M, N, B = 200, 1000, 300
    A = rng.standard_normal((M, N)).astype(np.float32) * rng.uniform(0.5, 2.0, N).astype(np.float32)
    A[:, 777] = A[:, 12]                      # exact tie across atom tiles: 12 must win
    A = np.asfortranarray(A)
    R1 = rng.standard_normal((B, M)).astype(np.float32)
    R1[3] = A[:, 12]
    R2 = 0.01 * rng.standard_normal((B, M)).astype(np.float32)   # smaller scores than call 1
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    for R in (R1, R2):
        idx = torch.full((B,), -7, dtype=torch.int32, device="cuda")
        sc = torch.full((B,), -7.0, dtype=torch.float32, device="cuda")
        omp.omp_correlate_argmax_noalloc(Ad, torch.from_numpy(R).cuda(), idx, sc)
        got_i, got_s = idx.cpu().numpy(), sc.cpu().numpy()
        ref_i, ref_s = _handle_top1(omp, A, R)
        S64 = np.stack([oracle.scores(A, R[b]) for b in range(B)])
        top2 = np.sort(S64, axis=1)[:, -2:]
        clear = (top2[:, 1] - top2[:, 0]) > 1e-5 * top2[:, 1]
        assert np.array_equal(got_i[clear], ref_i[clear])
        np.testing.assert_allclose(got_s, ref_s, rtol=1e-5)
        np.testing.assert_allclose(got_s, S64[np.arange(B), got_i], rtol=1e-5)
        if R is R1:
            assert got_i[3] == 12 and ref_i[3] == 12


def test_noalloc_scalar_loads_and_zero_dictionary(lib):
    """The scalar-load variant of the kernel: M = 203 (not a multiple of 4, so the last K chunk
    is partial) and a residual buffer that starts 4 bytes past a 16-byte boundary, on two calls
    in a row, against the handle entry point on aligned copies. Then an all-zero dictionary:
    every atom scores 0 and the lowest index, 0, is returned."""
    omp = lib
    rng = np.random.default_rng(32)
    M, N, B = 203, 700, 150
    A = np.asfortranarray(rng.standard_normal((M, N)).astype(np.float32))
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    for call in range(2):
        R = rng.standard_normal((B, M)).astype(np.float32) * (1.0 + 9.0 * call)
        flat = torch.zeros(B * M + 1, dtype=torch.float32, device="cuda")
        Rv = flat[1:].view(B, M)
        Rv.copy_(torch.from_numpy(R))
        assert Rv.data_ptr() % 16 == 4
        idx = torch.full((B,), -7, dtype=torch.int32, device="cuda")
        sc = torch.full((B,), -7.0, dtype=torch.float32, device="cuda")
        omp.omp_correlate_argmax_noalloc(Ad, Rv, idx, sc)
        got_i, got_s = idx.cpu().numpy(), sc.cpu().numpy()
        ref_i, ref_s = _handle_top1(omp, A, R)
        S64 = np.stack([oracle.scores(A, R[b]) for b in range(B)])
        top2 = np.sort(S64, axis=1)[:, -2:]
        clear = (top2[:, 1] - top2[:, 0]) > 1e-5 * top2[:, 1]
        assert clear.mean() > 0.9
        assert np.array_equal(got_i[clear], ref_i[clear])
        np.testing.assert_allclose(got_s, ref_s, rtol=1e-5)
    Z = torch.zeros((N, M), dtype=torch.float32, device="cuda").t()
    idx = torch.full((B,), -7, dtype=torch.int32, device="cuda")
    sc = torch.full((B,), -7.0, dtype=torch.float32, device="cuda")
    omp.omp_correlate_argmax_noalloc(Z, torch.from_numpy(R).cuda(), idx, sc)
    assert np.all(idx.cpu().numpy() == 0) and np.all(sc.cpu().numpy() == 0)


def test_noalloc_binding_checks_buffers(lib):
    """The binding refuses buffers the kernel would read or write out of bounds (short or
    mistyped outputs, a strided or mistyped R) before calling into C."""
    omp = lib
    M, N, B = 16, 64, 10
    A = torch.zeros((N, M), device="cuda").t()
    R = torch.zeros((B, M), device="cuda")
    idx = torch.zeros(B, dtype=torch.int32, device="cuda")
    sc = torch.zeros(B, dtype=torch.float32, device="cuda")
    bad = [
        (A, R, idx[:B - 1], sc),
        (A, R, idx, sc[:B - 1]),
        (A, R, idx.float(), sc),
        (A, R.double(), idx, sc),
        (A, torch.zeros((B, 2 * M), device="cuda")[:, ::2], idx, sc),
        (A, torch.zeros((B, M + 1), device="cuda"), idx, sc),
        (torch.zeros((M, N), device="cuda"), R, idx, sc),
    ]
    for args in bad:
        with pytest.raises(ValueError):
            omp.omp_correlate_argmax_noalloc(*args)


def test_noalloc_rejects_batches_beyond_its_scratch(lib):
    omp = lib
    M, N = 8, 16
    B = omp.NOALLOC_MAX_SIGNALS + 1
    A = torch.zeros((N, M), device="cuda").t()
    R = torch.zeros((B, M), device="cuda")
    idx = torch.zeros(B, dtype=torch.int32, device="cuda")
    sc = torch.zeros(B, dtype=torch.float32, device="cuda")
    with pytest.raises(omp.OmpError) as e:
        omp.omp_correlate_argmax_noalloc(A, R, idx, sc)
    assert e.value.status == 1
