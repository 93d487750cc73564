"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes: the hand-worked fixtures; the 64 x 256 planted workload in full; ragged shapes that span
several correlation tiles with a partial last tile in M, N and B; eps-stopped uneven batches;
the full-size 1024 x 8192, B = 4096, S = 32 workload checked on sampled signals; edge cases
(zero and non-finite signals, dependent atoms, exact ties across tiles, a single signal, a
128-step support, the largest signal length, scale equivariance over 24 orders of magnitude)."""
import numpy as np
import pytest

from oracle import omp as oracle
from tests import golden_util, parity
from workloads import gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRECS = ["fp32", "bf16", "fp8"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_06434_gb300 import build
    build.build()
    from paper_2407_06434_gb300 import omp
    omp.load()
    return omp


def dev_dict(A):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float32).T)).cuda().t()


def solve(prec, A, Y, S, eps=0.0, eps_relative=True, use_graph=True, max_batch=None, topk=8,
          gather24=False):
    from paper_2407_06434_gb300 import omp
    M, N = A.shape
    B = Y.shape[0]
    s = omp.OmpSolver(M, N, max_batch=max_batch or B, max_iters=S, precision=prec,
                      eps_relative=eps_relative, use_graph=use_graph, rescore_topk=topk,
                      gather24=gather24)
    Ad = dev_dict(A)
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    X, sup, n_iter, resid, stop = s.solve(Ad, Yd, S, eps, diagnostics=True)
    torch.cuda.synchronize()
    out = dict(X=X.cpu().numpy(), sup=sup.cpu().numpy(), n_iter=n_iter.cpu().numpy(),
               resid=resid.cpu().numpy(), stop=stop.cpu().numpy())
    out["status"] = omp.omp_get_error(s.h)
    s.close()
    return out


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", golden_util.FIXTURES)
def test_golden_fixtures(prec, name):
    d = golden_util.load(name)
    A = d["A"].astype(np.float32)
    r = solve(prec, A, d["y"][None, :].astype(np.float32), d["S"])
    k = d["n_iter"]
    assert r["n_iter"][0] == k
    assert list(r["sup"][0, :k]) == d["support"]
    assert np.all(r["sup"][0, k:] == -1)
    np.testing.assert_allclose(r["X"][0, :k], d["coef"], rtol=1e-5, atol=1e-6)
    if d.get("stop") == "dependent":
        assert r["stop"][0] == oracle.STOP_DEPENDENT


@pytest.mark.parametrize("prec", PRECS)
def test_planted_64x256_full(prec):
    w = gen.get_config("gaussian_64x256_s8_b16")
    A = gen.dictionary(w)
    Y, sp, sup, coef = gen.signals(w, A)
    ref = oracle.omp_batch(A, Y, w.S)
    r = solve(prec, A, Y, w.S)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"])
    assert st["tie_diverged"] == 0
    assert np.array_equal(r["sup"], ref.support)
    assert all(set(r["sup"][b]) == set(sup[b]) for b in range(w.B))


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_tiles(prec):
    """M = 200 (padded to 256), N = 1000 (7 full atom tiles + a partial one), B = 300 (two full
    signal tiles + a partial one), S = 24, noisy."""
    w = gen.get_config("gaussian_64x256_s8_b16", M=200, N=1000, B=300, S=24, s_min=5, s_max=24,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=3)
    Y, *_ = gen.signals(w, A, seed=3)
    ref = oracle.omp_batch(A, Y, w.S)
    r = solve(prec, A, Y, w.S)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"])
    assert st["tie_diverged"] <= 3, st


@pytest.mark.parametrize("prec", PRECS)
def test_gather24_signal_level_steps(prec):
    """The 24-bit gather option (q = A_S F[:,k] from A rounded to a 15-bit mantissa, 3 bytes per
    element) against the FP64 oracle where every step picks at signal level: ragged tiles
    (M = 200, N = 1000, B = 300), S = each signal's planted sparsity (5..24) with coefficients of
    magnitude in [0.5, 1] and noise 1e-3, then an eps-stopped uneven batch (eps = 1e-2 relative,
    above the noise floor 1e-3, signals
    retire once their planted atoms are found). Same parity bar as the FP32 rows; results move by
    rounding only (coefficients within 2e-5 of the FP32-gather solve). Past the noise floor the
    option moves picks at margins up to ~2e-3, and a final residual near 1e-5 ||y|| is off by
    about as much (the rounding of q, 2^-16 of ||y||, is then no longer small next to the scores
    and the residual), so it is for solves that stop at signal level above such a residual."""
    w = gen.get_config("gaussian_64x256_s8_b16", M=200, N=1000, B=300, S=24, s_min=5, s_max=24,
                       sigma=1e-3, col_scale=1.0, coef_kind="signed_uniform")
    A = gen.dictionary(w, seed=3)
    Y, sp, sup, coef = gen.signals(w, A, seed=3)
    rows = [np.flatnonzero(sp == s_) for s_ in np.unique(sp)]
    n_div = n_same = 0
    for rr in rows:
        S = int(sp[rr[0]])
        ref = oracle.omp_batch(A, Y[rr], S)
        r = solve(prec, A, Y[rr], S, gather24=True)
        st = parity.compare(A, Y[rr], ref, r["sup"], r["X"], r["n_iter"], r["resid"])
        n_div += st["tie_diverged"]
        r32 = solve(prec, A, Y[rr], S)
        same = np.all(r["sup"] == r32["sup"], axis=1)
        n_same += int(same.sum())
        d = np.linalg.norm(r["X"][same] - r32["X"][same], axis=1) / np.linalg.norm(r32["X"][same], axis=1)
        assert d.size == 0 or d.max() <= 2e-5, d.max()
    assert n_div <= 2 and n_same >= w.B - 2, (n_div, n_same)
    w = gen.get_config("gaussian_64x256_s8_b16", M=256, N=2048, B=200, S=48, s_min=4, s_max=40,
                       sigma=1e-3, col_scale=1.0, coef_kind="signed_uniform")
    A = gen.dictionary(w, seed=4)
    Y, *_ = gen.signals(w, A, seed=4)
    ref = oracle.omp_batch(A, Y, w.S, 1e-2)
    r = solve(prec, A, Y, w.S, eps=1e-2, gather24=True)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"], eps=1e-2)
    assert np.mean(r["stop"] == oracle.STOP_EPS) > 0.9
    assert st["tie_diverged"] <= 2, st


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("eps_relative", [True, False])
def test_eps_stop_uneven(prec, eps_relative):
    """Per-signal sparsity 4..40 with a low noise floor: the eps stop fires near k = s, so the
    live set shrinks unevenly and is compacted every iteration."""
    w = gen.get_config("gaussian_64x256_s8_b16", M=256, N=2048, B=200, S=48, s_min=4, s_max=40,
                       sigma=1e-6, col_scale=1.0)
    A = gen.dictionary(w, seed=4)
    Y, sp, _, _ = gen.signals(w, A, seed=4)
    eps = 1e-3 if eps_relative else 5e-3
    ref = oracle.omp_batch(A, Y, w.S, eps, eps_relative)
    r = solve(prec, A, Y, w.S, eps=eps, eps_relative=eps_relative)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"], eps=eps,
                        eps_relative=eps_relative)
    assert np.mean(r["n_iter"] < w.S) > 0.9
    assert np.mean(r["stop"] == oracle.STOP_EPS) > 0.9
    assert st["tie_diverged"] <= 2, st


@pytest.mark.parametrize("prec", PRECS)
def test_zero_and_nonfinite_signals(prec):
    w = gen.get_config("gaussian_64x256_s8_b16", B=20)
    A = gen.dictionary(w)
    Y, *_ = gen.signals(w, A)
    Y[3] = 0.0
    Y[7, 5] = np.nan
    Y[11, 0] = np.inf
    good = [b for b in range(w.B) if b not in (3, 7, 11)]
    ref = oracle.omp_batch(A, Y[good], w.S)
    r = solve(prec, A, Y, w.S)
    for b in (3, 7, 11):
        assert r["n_iter"][b] == 0 and np.all(r["sup"][b] == -1) and np.all(r["X"][b] == 0)
        assert r["stop"][b] == oracle.STOP_ZERO
    status, flags = r["status"]
    assert status == 6 and flags & 0x2
    parity.compare(A, Y[good], ref, r["sup"][good], r["X"][good], r["n_iter"][good],
                   r["resid"][good])


@pytest.mark.parametrize("prec", PRECS)
def test_graph_replay_and_direct_launches_agree(prec):
    from paper_2407_06434_gb300 import omp
    w = gen.get_config("gaussian_64x256_s8_b16", M=128, N=512, B=100, S=16, s_min=16, s_max=16,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=6)
    Y, *_ = gen.signals(w, A, seed=6)
    Ad = dev_dict(A)
    Yd = torch.from_numpy(Y).cuda()
    outs = []
    for use_graph in (True, False):
        s = omp.OmpSolver(w.M, w.N, max_batch=128, max_iters=16, precision=prec,
                          use_graph=use_graph)
        for _ in range(2):     # second call replays the captured graph
            X, sup = s.solve(Ad, Yd, w.S)
            outs.append((X.cpu().numpy(), sup.cpu().numpy()))
        s.close()
    for X, sup in outs[1:]:
        assert np.array_equal(sup, outs[0][1])
        assert np.array_equal(X.view(np.uint32), outs[0][0].view(np.uint32))


@pytest.mark.parametrize("prec", PRECS)
def test_device_loop_stops_when_no_signal_is_live(prec):
    """With use_graph = 2 the graph runs the iterations as a device-side while loop: with a
    relative eps that every signal reaches after about s iterations it stops after max(n_iter)
    passes, well before S, and gives bit-identical results to direct launches and to the unrolled
    graph; an all-zero batch takes one pass."""
    from paper_2407_06434_gb300 import omp
    w = gen.get_config("gaussian_64x256_s8_b16", M=128, N=512, B=100, S=32, s_min=2, s_max=6,
                       sigma=1e-6, col_scale=1.0)
    A = gen.dictionary(w, seed=8)
    Y, *_ = gen.signals(w, A, seed=8)
    Ad = dev_dict(A)
    Yd = torch.from_numpy(Y).cuda()
    res = {}
    for use_graph in (2, 1, 0):
        s = omp.OmpSolver(w.M, w.N, max_batch=128, max_iters=w.S, precision=prec,
                          use_graph=use_graph)
        for _ in range(2):
            X, sup, n_iter, resid, stop = s.solve(Ad, Yd, w.S, 1e-3, diagnostics=True)
        torch.cuda.synchronize()
        res[use_graph] = (X.cpu().numpy(), sup.cpu().numpy(), n_iter.cpu().numpy(),
                          omp.omp_loop_passes(s.h))
        if use_graph == 2:
            Z = torch.zeros_like(Yd)
            s.solve(Ad, Z, w.S, 1e-3)
            assert omp.omp_loop_passes(s.h) == 1
            assert np.array_equal(s.solve(Ad, Z, w.S, 1e-3)[1].cpu().numpy(), np.full((w.B, w.S), -1))
        s.close()
    Xg, supg, ng, passes = res[2]
    for other in (1, 0):
        Xd, supd, nd, passes_other = res[other]
        assert passes_other == 0
        assert np.array_equal(supg, supd) and np.array_equal(ng, nd)
        assert np.array_equal(Xg.view(np.uint32), Xd.view(np.uint32))
    assert passes == int(ng.max()) and passes < w.S


SHORTCUT_CASES = {
    # many close calls: coherent pairs among the planted atoms, noise-level late steps
    "noisy_256x2048": ("gaussian_64x256_s8_b16",
                       dict(M=256, N=2048, B=512, S=48, s_min=8, s_max=40, sigma=1e-2,
                            col_scale=1.0), 11),
    # the benchmark shape, whole batch
    "bench_1024x8192": ("gaussian_1024x8192_s32_b4096", {}, 0),
    # paired atoms at correlation ~0.3 with unequal column norms: the Gram terms of the
    # threshold bound are large
    "coherent_512x4096": ("coherent_4096x32768_s64_b16384",
                          dict(M=512, N=4096, B=1024, S=40, s_min=40, s_max=40), 5),
    # uneven sparsity with a relative eps stop: signals retire at different steps, so the
    # compaction moves rows, operand rows and thresholds to new positions
    "eps_uneven_512x4096": ("gaussian_2048x16384_s4to128_b8192_lownoise",
                            dict(M=512, N=4096, B=1500, S=48, s_min=4, s_max=44), 7),
    # exact duplicates (equal scores: the lower index must win everywhere) and near-duplicates
    # (scores within the error bounds) of the first 128 atoms, in other atom tiles
    "duplicates_256x2048": ("gaussian_64x256_s8_b16",
                            dict(M=256, N=2048, B=600, S=32, s_min=8, s_max=24, sigma=1e-3,
                                 col_scale=1.0), 13),
}


def _duplicate_columns(A, seed):
    """Columns 1000..1127 copy columns 0..127; columns 1500..1627 are those copies with a
    1e-4 perturbation, renormalised."""
    A = np.array(A, dtype=np.float64)
    A[:, 1000:1128] = A[:, 0:128]
    rng = np.random.default_rng(seed)
    B = A[:, 0:128] + 1e-4 * rng.standard_normal((A.shape[0], 128))
    A[:, 1500:1628] = B / np.linalg.norm(B, axis=0)
    return np.asfortranarray(A.astype(np.float32))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("case", sorted(SHORTCUT_CASES))
def test_rescoring_shortcut_and_pruning_are_exact(monkeypatch, case, prec):
    """The quantised paths skip the FP32 rescoring when the quantised best leads the second by
    more than twice the quantisation error bound, and rescore only the candidates within that
    window otherwise; BF16 also drops, in its correlation, columns below the pruning threshold
    that the previous step's update derived from its runner-up candidates. None of it may change
    a pick: the supports, coefficients and residual norms must be bit-identical to rescoring all
    eight candidates with no pruning (OMP_RESCORE_ALWAYS=1 turns the bound off)."""
    from paper_2407_06434_gb300 import omp
    name, over, seed = SHORTCUT_CASES[case]
    w = gen.get_config(name, **over)
    A = gen.dictionary(w, seed=seed)
    if w.dict_kind == "coherent":
        scale = np.random.default_rng(seed).uniform(0.5, 2.0, w.N).astype(np.float32)
        A = np.asfortranarray(A * scale[None, :])
    if case.startswith("duplicates"):
        A = _duplicate_columns(A, seed)
    Y, *_ = gen.signals(w, A, seed=seed)
    Ad = dev_dict(A)
    Yd = torch.from_numpy(Y).cuda()
    out = {}
    for always in ("0", "1"):
        monkeypatch.setenv("OMP_RESCORE_ALWAYS", always)
        s = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision=prec)
        X, sup, n_iter, resid, stop = s.solve(Ad, Yd, w.S, w.eps, diagnostics=True)
        torch.cuda.synchronize()
        out[always] = (X.cpu().numpy(), sup.cpu().numpy(), resid.cpu().numpy())
        assert omp.omp_get_error(s.h)[1] == 0
        if w.eps > 0:
            n = n_iter.cpu().numpy()
            assert np.mean(n < w.S) > 0.5 and len(np.unique(n)) > 10   # many retirement steps
        s.close()
    assert np.array_equal(out["0"][1], out["1"][1])
    assert np.array_equal(out["0"][0].view(np.uint32), out["1"][0].view(np.uint32))
    assert np.array_equal(out["0"][2].view(np.uint32), out["1"][2].view(np.uint32))


@pytest.mark.parametrize("prec", PRECS)
def test_host_entry_point(prec):
    from paper_2407_06434_gb300 import omp
    w = gen.get_config("gaussian_64x256_s8_b16", B=64)
    A = gen.dictionary(w)
    Y, *_ = gen.signals(w, A)
    s = omp.OmpSolver(w.M, w.N, max_batch=64, max_iters=8, precision=prec)
    Ad = dev_dict(A)
    Xd, supd = s.solve(Ad, torch.from_numpy(Y).cuda(), 8)
    Yh = torch.from_numpy(Y).pin_memory()
    Xh = torch.empty((64, 8), dtype=torch.float32).pin_memory()
    Sh = torch.empty((64, 8), dtype=torch.int32).pin_memory()
    omp.omp_solve_batch_host(s.h, Ad, Yh, 8, 0.0, Xh, Sh)
    assert np.array_equal(Sh.numpy(), supd.cpu().numpy())
    assert np.array_equal(Xh.numpy(), Xd.cpu().numpy())
    s.close()


def test_correlate_top1_fp32_and_ties_across_tiles():
    """FP32 correlation: the top-1 atom equals the FP64 argmax wherever the FP64 top-two margin
    exceeds 1e-5; exact ties made by duplicated columns (in another atom tile and another
    signal tile) resolve to the lower index."""
    from paper_2407_06434_gb300 import omp
    rng = np.random.default_rng(8)
    M, N, B = 96, 700, 260
    A = rng.standard_normal((M, N)).astype(np.float32)
    A[:, 650] = A[:, 37]          # duplicate in another atom tile
    A[:, 300] = A[:, 299]         # duplicate in the same tile
    A = np.asfortranarray(A)
    R = rng.standard_normal((B, M)).astype(np.float32)
    R[5] = A[:, 37] * 2.0         # signal 5's best atoms are 37 and 650 (exact tie)
    R[200] = -A[:, 300]           # signal 200 ties 299 and 300
    s = omp.OmpSolver(M, N, max_batch=B, max_iters=1, precision="fp32")
    idx = torch.empty((B, 1), dtype=torch.int32, device="cuda")
    sc = torch.empty((B, 1), dtype=torch.float32, device="cuda")
    omp.omp_correlate_topk(s.h, dev_dict(A), torch.from_numpy(R).cuda(), 1, idx, sc)
    idx = idx.cpu().numpy()[:, 0]
    sc = sc.cpu().numpy()[:, 0]
    assert idx[5] == 37 and idx[200] == 299
    S64 = np.stack([oracle.scores(A, R[b]) for b in range(B)])
    top2 = np.sort(S64, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 1e-5 * top2[:, 1]
    assert np.array_equal(idx[clear], np.argmax(S64, axis=1)[clear])
    np.testing.assert_allclose(sc, S64[np.arange(B), idx], rtol=1e-5)
    s.close()


_FULL_REF = {}


def _full_size_reference():
    """The 1024 x 8192, B = 4096, S = 32 workload and the oracle's result for every signal
    (computed once for the three precisions)."""
    if not _FULL_REF:
        w = gen.get_config("gaussian_1024x8192_s32_b4096")
        A = gen.dictionary(w)
        Y, *_ = gen.signals(w, A)
        _FULL_REF.update(w=w, A=A, Y=Y, ref=oracle.omp_batch(A, Y, w.S))
    return _FULL_REF["w"], _FULL_REF["A"], _FULL_REF["Y"], _FULL_REF["ref"]


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_1024x8192_whole_batch(prec):
    """The 1024 x 8192, B = 4096, S = 32 workload at full size in the launch configuration the
    benchmark times (graph replay); every signal of the batch is checked against the oracle."""
    w, A, Y, ref = _full_size_reference()
    r = solve(prec, A, Y, w.S)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"])
    assert st["tie_diverged"] <= 0.01 * w.B, st
    assert np.all(r["n_iter"] == w.S)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_correlate_top8_quantised(prec):
    """Tensor-core correlation: the top-8 atoms per signal equal a CPU top-8 of the scores
    computed exactly (FP64) from the same quantised operands (BF16 round-to-nearest-even, or
    E4M3 with per-atom and per-signal scales), wherever the CPU's 8th and 9th scores are apart
    by more than 1e-4 relative; exact ties made by duplicated atoms resolve to the lower index.
    N = 1000 gives a partial last atom tile, B = 300 a partial last signal tile."""
    from oracle import quant
    from paper_2407_06434_gb300 import omp
    rng = np.random.default_rng(12)
    M, N, B = 200, 1000, 300
    A = rng.standard_normal((M, N)).astype(np.float32)
    A[:, 900] = A[:, 10]
    A = np.asfortranarray(A)
    R = rng.standard_normal((B, M)).astype(np.float32)
    R[7] = 3.0 * A[:, 10]
    s = omp.OmpSolver(M, N, max_batch=B, max_iters=1, precision=prec)
    idx = torch.empty((B, 8), dtype=torch.int32, device="cuda")
    sc = torch.empty((B, 8), dtype=torch.float32, device="cuda")
    omp.omp_correlate_topk(s.h, dev_dict(A), torch.from_numpy(R).cuda(), 8, idx, sc)
    idx = idx.cpu().numpy()
    sc = sc.cpu().numpy()
    s.close()
    At = np.ascontiguousarray(A.T)
    inv_norm = (1.0 / np.sqrt(np.sum(At.astype(np.float64) ** 2, axis=1))).astype(np.float32)
    if prec == "bf16":
        Aq = quant.bf16_round(At).astype(np.float64)
        Rq = quant.bf16_round(R).astype(np.float64)
        esc = inv_norm.astype(np.float64)
    else:
        ca, sa = quant.fp8_scale_rows(At)
        cr, _ = quant.fp8_scale_rows(R)
        Aq = quant.e4m3_value(ca)
        Rq = quant.e4m3_value(cr)
        esc = (sa * inv_norm).astype(np.float32).astype(np.float64)
    S = np.abs(Rq @ Aq.T) * esc[None, :]
    assert idx[7, 0] == 10 and 900 in idx[7]          # tie: 10 before 900
    checked = 0
    for b in range(B):
        order = np.lexsort((np.arange(N), -S[b]))
        s8, s9 = S[b, order[7]], S[b, order[8]]
        if s8 - s9 > 1e-4 * s8:
            assert set(idx[b]) == set(order[:8]), b
            np.testing.assert_allclose(np.sort(sc[b])[::-1], S[b, order[:8]], rtol=2e-5)
            checked += 1
    assert checked > 0.9 * B


def _tune_key(w, prec=1):
    name = torch.cuda.get_device_properties(0).name[:64]
    return f"{name} M={w.M} N={w.N} prec={prec} B={w.B} S={w.S}"


def test_autotune_choice_and_cache(tmp_path, monkeypatch):
    """The autotuner picks valid launch shapes (update warps per signal; correlation stages and
    persistent CTAs), results still match the oracle after the switch, and a second handle reads
    the recorded choice from the cache file instead of timing again. Every correlation shape the
    tuner can pick gives bit-identical results."""
    from paper_2407_06434_gb300 import omp
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("OMP_AUTOTUNE_CACHE", str(cache))
    w = gen.get_config("gaussian_64x256_s8_b16", M=1024, N=2048, B=512, S=16, s_min=16, s_max=16,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=13)
    Y, *_ = gen.signals(w, A, seed=13)
    Ad, Yd = dev_dict(A), torch.from_numpy(Y).cuda()
    s = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="bf16")
    X, S_ = s.solve(Ad, Yd, w.S)                     # captures a graph with the default shape
    choice = omp.omp_autotune(s.h, Ad, Yd, w.S, 0.0, repeats=1)
    assert choice in (1, 2, 4, 8)
    tw, tpe, tst, tg, tcl = omp.omp_tuning(s.h)
    _, sms = omp.omp_handle_info(s.h)
    assert tw == choice and tpe in (0, 1) and tst in (2, 3, 4, 6) and tcl in (1, 2)
    assert 1 <= tg <= sms and tg % tcl == 0
    X, S_, n_iter, resid, stop = s.solve(Ad, Yd, w.S, diagnostics=True)
    torch.cuda.synchronize()
    rows = np.arange(0, w.B, 16)
    ref = oracle.omp_batch(A, Y[rows], w.S)
    parity.compare(A, Y[rows], ref, S_.cpu().numpy()[rows], X.cpu().numpy()[rows],
                   n_iter.cpu().numpy()[rows], resid.cpu().numpy()[rows], rows=rows)
    s.close()
    # the cache records the CTAs asked for; a pair launch takes an even count
    cw, cst, cg, cpe, ccl = (int(v) for v in cache.read_text().strip().split("|")[-1].split(","))
    assert (cw, cst, cpe, ccl) == (choice, tst, tpe, tcl) and tg <= cg <= sms
    s2 = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="bf16")
    assert omp.omp_autotune(s2.h, Ad, Yd, w.S, 0.0, repeats=1) == choice
    assert omp.omp_tuning(s2.h) == (tw, tpe, tst, tg, tcl)
    assert len(cache.read_text().strip().splitlines()) == 1
    s2.close()
    # every shape gives the same results (cache lines force each one)
    outs = []
    for st, g, pe, cl in ((4, sms, 0, 1), (3, sms, 0, 1), (2, sms, 0, 1), (4, sms - sms // 8, 0, 1),
                          (4, sms, 1, 1), (4, sms, 0, 2), (6, sms - sms // 8, 0, 2)):
        cache.write_text(f"{_tune_key(w)}|{choice},{st},{g},{pe},{cl}\n")
        s3 = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="bf16")
        omp.omp_autotune(s3.h, Ad, Yd, w.S, 0.0, repeats=1)
        t3 = omp.omp_tuning(s3.h)
        assert t3[:3] == (choice, pe, st) and t3[4] == cl
        assert (t3[3] == g) if cl == 1 else (0 < t3[3] <= g and t3[3] % cl == 0)
        X3, S3 = s3.solve(Ad, Yd, w.S)
        outs.append((X3.cpu().numpy(), S3.cpu().numpy()))
        s3.close()
    for X3, S3 in outs[1:]:
        assert np.array_equal(S3, outs[0][1])
        assert np.array_equal(X3.view(np.uint32), outs[0][0].view(np.uint32))


@pytest.mark.parametrize("prec,pcode", [("bf16", 1), ("fp8", 2)])
def test_cta_pair_ragged(tmp_path, monkeypatch, prec, pcode):
    """Correlation CTA pairs (one 256-row MMA across two SMs, each holding half of the atom
    tile), with 4 and 6 stages: on a batch of 600 signals (5 signal tiles, the last ragged, so the
    last pair has a tile past the batch) with a residual stop that retires signals (the live
    count, and with it the tile count, shrinks from step to step), every shape gives results
    bit-identical to one CTA per tile, and the results match the oracle."""
    from paper_2407_06434_gb300 import omp
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("OMP_AUTOTUNE_CACHE", str(cache))
    w = gen.get_config("gaussian_64x256_s8_b16", M=512, N=2304, B=600, S=24, s_min=4, s_max=24,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=21)
    Y, *_ = gen.signals(w, A, seed=21)
    Ad, Yd = dev_dict(A), torch.from_numpy(Y).cuda()
    eps = 1e-2  # signals stop after 4 to 24 steps
    outs = []
    for st, cl in ((4, 1), (4, 2), (6, 2), (3, 1)):
        s = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision=prec)
        sms = omp.omp_handle_info(s.h)[1]
        cache.write_text(f"{_tune_key(w, pcode)}|1,{st},{sms},0,{cl}\n")
        omp.omp_autotune(s.h, Ad, Yd, w.S, eps, repeats=1)
        assert omp.omp_tuning(s.h)[2] == st and omp.omp_tuning(s.h)[4] == cl
        X, S_, n_iter, resid, _ = s.solve(Ad, Yd, w.S, eps, diagnostics=True)
        torch.cuda.synchronize()
        outs.append((X.cpu().numpy(), S_.cpu().numpy(), n_iter.cpu().numpy(), resid.cpu().numpy()))
        s.close()
    n_it = outs[0][2]
    assert n_it.min() < w.S and n_it.max() > n_it.min()  # signals retire at different steps
    for X, S_, it, r in outs[1:]:
        assert np.array_equal(S_, outs[0][1]) and np.array_equal(it, n_it)
        assert np.array_equal(X.view(np.uint32), outs[0][0].view(np.uint32))
        assert np.array_equal(r.view(np.uint32), outs[0][3].view(np.uint32))
    rows = np.arange(0, w.B, 7)
    X, S_, it, r = outs[2]
    ref = oracle.omp_batch(A, Y[rows], w.S, eps=eps)
    parity.compare(A, Y[rows], ref, S_[rows], X[rows], it[rows], r[rows], eps=eps, rows=rows)


def test_read_bandwidth_probe():
    """The benchmark's L2 read probe reads every word: the per-block sums add up to reps times
    the buffer's sum; its bandwidth over an L2-resident buffer is positive and finite."""
    from paper_2407_06434_gb300 import omp
    buf = torch.arange(1 << 16, dtype=torch.float32, device="cuda") % 7
    out = torch.zeros(64, device="cuda")
    st = omp.load().omp_read_bandwidth_probe(buf.data_ptr(), buf.numel() * 4, 3, out.data_ptr(), 64, None)
    assert st == 0
    torch.cuda.synchronize()
    assert float(out.sum()) == pytest.approx(3 * float(buf.sum()), rel=1e-5)
    assert omp.load().omp_read_bandwidth_probe(buf.data_ptr(), 12, 1, out.data_ptr(), 64, None) != 0
    gbs = omp.read_bandwidth_gbs(32, 10)
    assert np.isfinite(gbs) and gbs > 0


@pytest.mark.parametrize("prec", PRECS)
def test_single_signal_and_long_support(prec):
    """B = 1 (one partial tile everywhere) and a long run, S = 128 on a 256 x 512 dictionary."""
    w = gen.get_config("gaussian_64x256_s8_b16", M=256, N=512, B=1, S=128, s_min=100, s_max=100,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=13)
    Y, *_ = gen.signals(w, A, seed=13)
    ref = oracle.omp_batch(A, Y, w.S)
    r = solve(prec, A, Y, w.S)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"])
    assert st["tie_diverged"] == 0, st


@pytest.mark.parametrize("prec", PRECS)
def test_longest_signal_length(prec):
    """M = 8192, the largest padded length (eight warps per signal in the update, 64 or 128
    tensor-core K stages per unit), with a ragged atom count and batch."""
    w = gen.get_config("gaussian_64x256_s8_b16", M=8192, N=700, B=70, S=12, s_min=4, s_max=12,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=14)
    Y, *_ = gen.signals(w, A, seed=14)
    ref = oracle.omp_batch(A, Y, w.S)
    r = solve(prec, A, Y, w.S)
    st = parity.compare(A, Y, ref, r["sup"], r["X"], r["n_iter"], r["resid"])
    assert st["tie_diverged"] <= 1, st


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("scale", [1e-12, 1e12])
def test_scale_equivariance(prec, scale):
    """OMP is scale-equivariant in y (App. A): scaling the batch by 1e-12 or 1e12 picks the same
    supports, scales the coefficients by the same factor and keeps the relative eps stop."""
    w = gen.get_config("gaussian_64x256_s8_b16", M=128, N=512, B=40, S=16, s_min=4, s_max=12,
                       sigma=1e-6, col_scale=1.0)
    A = gen.dictionary(w, seed=15)
    Y, *_ = gen.signals(w, A, seed=15)
    r1 = solve(prec, A, Y, w.S, eps=1e-3)
    r2 = solve(prec, A, (Y * scale).astype(np.float32), w.S, eps=1e-3)
    assert np.array_equal(r1["sup"], r2["sup"])
    assert np.array_equal(r1["n_iter"], r2["n_iter"])
    np.testing.assert_allclose(r2["X"], r1["X"] * scale, rtol=1e-4, atol=1e-6 * scale)


def test_handles_with_different_layouts_coexist():
    """A kernel's shared-memory limit is one setting of the process: a handle whose layout is
    smaller (FP32, or fewer iterations, or a smaller dictionary for the Gram-space form) must
    not lower the limit under a handle created before it."""
    from paper_2407_06434_gb300 import omp
    w = gen.get_config("gaussian_64x256_s8_b16", M=256, N=2048, B=300, S=48, s_min=8, s_max=40,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=2)
    Y, *_ = gen.signals(w, A, seed=2)
    Ad = dev_dict(A)
    Yd = torch.from_numpy(Y).cuda()
    big = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="bf16")
    X0, S0 = big.solve(Ad, Yd, w.S)
    G0 = big.solve_gram(Ad, Yd, w.S)
    torch.cuda.synchronize()
    small = [omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=8, precision="fp32"),
             omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=8, precision="bf16")]
    for s in small:
        s.solve(Ad, Yd, 8)
    A2 = np.asfortranarray(A[:, :256])
    small_gram = omp.OmpSolver(w.M, 256, max_batch=w.B, max_iters=8, precision="fp32")
    small_gram.solve_gram(dev_dict(A2), Yd, 8)
    torch.cuda.synchronize()
    X1, S1 = big.solve(Ad, Yd, w.S)
    G1 = big.solve_gram(Ad, Yd, w.S)
    torch.cuda.synchronize()
    assert np.array_equal(S0.cpu().numpy(), S1.cpu().numpy())
    assert np.array_equal(X0.cpu().numpy().view(np.uint32), X1.cpu().numpy().view(np.uint32))
    assert np.array_equal(G0[1].cpu().numpy(), G1[1].cpu().numpy())
    for s in small + [small_gram, big]:
        s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_margins_against_the_oracle(prec):
    """margin_out of omp_solve_batch_ex: the top-two score margin (s1 - s2) / s1 of every step,
    against the FP64 oracle's on a noisy ragged batch (several atom and signal tiles). Asking
    for margins changes no result (supports and coefficients bit-identical to the same solve
    without them). FP32: equal to the oracle's within 2e-4 at every step of every signal whose
    support is the oracle's. Quantised paths (margins over the FP32 scores of the rescored
    candidates): never below the oracle's by more than 2e-4 (the runner-up can only be missed,
    which raises the margin), and equal to it at most steps. The tolerance is the FP32 rounding
    of two scores near the noise floor (about 5e-5 was seen), well below a near-tie's 1e-3. -1
    past each signal's last step."""
    from paper_2407_06434_gb300 import omp
    w = gen.get_config("gaussian_64x256_s8_b16", M=200, N=1000, B=300, S=24, s_min=5, s_max=24,
                       sigma=1e-3, col_scale=1.0)
    A = gen.dictionary(w, seed=3)
    Y, *_ = gen.signals(w, A, seed=3)
    ref = oracle.omp_batch(A, Y, w.S)
    s = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision=prec)
    Ad, Yd = dev_dict(A), torch.from_numpy(Y).cuda()
    X0, S0 = s.solve(Ad, Yd, w.S)
    X1, S1, n_iter, resid, stop, mg = s.solve(Ad, Yd, w.S, diagnostics=True, margins=True)
    X2, S2 = s.solve(Ad, Yd, w.S)                    # the plain graph again after the stats one
    torch.cuda.synchronize()
    s.close()
    for Xa, Sa in ((X1, S1), (X2, S2)):
        assert np.array_equal(Sa.cpu().numpy(), S0.cpu().numpy())
        assert np.array_equal(Xa.cpu().numpy().view(np.uint32), X0.cpu().numpy().view(np.uint32))
    sup, mg, n_iter = S1.cpu().numpy(), mg.cpu().numpy(), n_iter.cpu().numpy()
    for b in range(w.B):
        assert np.all(mg[b, n_iter[b]:] == -1.0)
    same = np.all(sup == ref.support, axis=1)
    assert same.mean() > 0.95
    steps = np.arange(w.S)[None, :] < n_iter[:, None]
    sel = same[:, None] & steps
    diff = mg[sel] - ref.margin[sel]
    assert np.all(np.isfinite(diff))
    if prec == "fp32":
        assert np.max(np.abs(diff)) <= 2e-4, np.max(np.abs(diff))
    else:
        assert diff.min() >= -2e-4, diff.min()
        assert np.mean(np.abs(diff) <= 2e-4) >= (0.8 if prec == "bf16" else 0.3)
