"""Pins for the FP64 proposal-network reference and the candidate-restricted OMP reference:
central finite differences, brute-force top-K with ties, and special cases of the restricted
iteration that reduce to plain OMP (Alg. 1)."""
import numpy as np

from oracle import mlp, omp
from workloads import gen


def _instance(seed=0, N=64, H=16, B=6):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, N)) * 0.3
    W1 = rng.standard_normal((H, N)) * 0.2
    b1 = rng.standard_normal(H) * 0.1
    W2 = rng.standard_normal((N, H)) * 0.2
    b2 = rng.standard_normal(N) * 0.1
    sup = np.stack([rng.choice(N, 5, replace=False) for _ in range(B)])
    return X, mlp.labels_matrix(sup, N), W1, b1, W2, b2


def test_gradients_match_central_differences():
    """64 -> 16 -> 64 network in FP64 (no BF16 rounding): every analytic gradient entry checked
    against a central difference of the loss, relative error <= 1e-6."""
    X, Yl, W1, b1, W2, b2 = _instance()
    pw = 7.0
    beta = np.array([3.0])
    loss, dW1, db1, dW2, db2, dbeta = mlp.loss_and_grads(X, Yl, W1, b1, W2, b2, pw, False, beta[0])
    h = 1e-5
    rng = np.random.default_rng(1)
    for name, P, G in [("W1", W1, dW1), ("b1", b1, db1), ("W2", W2, dW2), ("b2", b2, db2),
                       ("beta", beta, np.array([dbeta]))]:
        flat = P.reshape(-1)
        idx = rng.choice(flat.size, size=min(40, flat.size), replace=False)
        fds, gs = [], []
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = mlp.loss_and_grads(X, Yl, W1, b1, W2, b2, pw, False, beta[0])[0]
            flat[i] = old - h
            lm = mlp.loss_and_grads(X, Yl, W1, b1, W2, b2, pw, False, beta[0])[0]
            flat[i] = old
            fds.append((lp - lm) / (2 * h))
            gs.append(G.reshape(-1)[i])
        fds, gs = np.array(fds), np.array(gs)
        assert np.linalg.norm(fds - gs) <= 1e-6 * np.linalg.norm(gs), name


def test_loss_closed_form_at_zero_weights():
    """With all weights zero the logits equal b2, so the loss is the mean of
    pw y softplus(-b2) + (1 - y) softplus(b2) and the gradient w.r.t. b2 is the column mean of
    sigma(b2) (1 - y + pw y) - pw y."""
    X, Yl, W1, b1, W2, b2 = _instance(2)
    Z = np.zeros_like
    pw = 3.0
    loss, dW1, db1, dW2, db2, _ = mlp.loss_and_grads(X, Yl, Z(W1), Z(b1), Z(W2), b2, pw, False)
    sp = lambda v: np.log1p(np.exp(v))
    want = np.mean(pw * Yl * sp(-b2) + (1 - Yl) * sp(b2))
    assert abs(loss - want) < 1e-12
    sg = 1 / (1 + np.exp(-b2))
    B, N = Yl.shape
    np.testing.assert_allclose(db2, np.sum(sg * (1 - Yl + pw * Yl) - pw * Yl, axis=0) / (B * N),
                               rtol=1e-12, atol=1e-15)
    assert np.all(dW1 == 0) and np.all(db1 == 0)


def test_bf16_rounding_points_change_little():
    X, Yl, W1, b1, W2, b2 = _instance(3)
    a = mlp.loss_and_grads(X, Yl, W1, b1, W2, b2, 5.0, round_bf16=False)
    b = mlp.loss_and_grads(X, Yl, W1, b1, W2, b2, 5.0, round_bf16=True)
    for ga, gb in zip(a[1:5], b[1:5]):
        rel = np.linalg.norm(ga - gb) / np.linalg.norm(ga)
        assert 0 < rel < 0.05


def test_topk_lowest_index_brute_force():
    rng = np.random.default_rng(4)
    v = rng.integers(0, 6, size=(20, 30)).astype(float)   # many exact ties
    got = mlp.topk_lowest_index(v, 7)
    for b in range(20):
        # explicit: repeatedly take the max, lowest index first
        rem = list(range(30))
        pick = []
        for _ in range(7):
            best = max(rem, key=lambda i: (v[b, i], -i))
            pick.append(best)
            rem.remove(best)
        assert list(got[b]) == sorted(pick)


def test_candidate_reference_reduces_to_plain_omp():
    """All atoms as candidates with tau = 0: identical to Alg. 1. The planted support as
    candidates (noiseless): the same result with no fallback. Candidates that miss the best atom
    with a high tau: falls back at step 0 and equals Alg. 1."""
    w = gen.get_config("gaussian_64x256_s8_b16")
    A = gen.dictionary(w)
    Y, sp, sup, coef = gen.signals(w, A)
    for b in range(4):
        ref = omp.omp_reference(A, Y[b], 8)
        r, fb = omp.omp_candidates_reference(A, Y[b], 8, np.arange(256), np.zeros(8))
        assert fb == -1 and np.array_equal(r.support, ref.support)
        np.testing.assert_allclose(r.coef, ref.coef, rtol=1e-10, atol=1e-12)
        r, fb = omp.omp_candidates_reference(A, Y[b], 8, sup[b], np.full(8, 1e-6))
        assert fb == -1 and set(r.support[0]) == set(sup[b])
        others = np.setdiff1d(np.arange(256), [ref.support[0, 0]])
        r, fb = omp.omp_candidates_reference(A, Y[b], 8, others[:40], np.full(8, 0.99))
        assert fb == 0 and np.array_equal(r.support, ref.support)


def _orthonormal_dictionary(seed, M=16):
    """Q D: an orthonormal basis with columns rescaled by d_n in [0.5, 2]."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((M, M)))
    d = rng.uniform(0.5, 2.0, M)
    return Q, Q * d[None, :]


def test_features_closed_form_on_an_orthonormal_dictionary():
    """For A = Q D (Q orthonormal, D a positive diagonal) the features x = A^T y / (||a|| ||y||)
    are Q^T y / ||y||: a unit vector whatever the column scales and the signal's scale, from
    which Q x gives back y / ||y||. A zero signal gives zero features."""
    Q, A = _orthonormal_dictionary(5)
    rng = np.random.default_rng(6)
    Y = rng.standard_normal((6, 16)) * np.array([1e-3, 1.0, 1e3, 2.0, 0.5, 7.0])[:, None]
    Y[4] = 0.0
    X = mlp.features(A.astype(np.float32), Y.astype(np.float32), round_bf16=False)
    Y32 = Y.astype(np.float32).astype(np.float64)
    for b in range(6):
        yn = np.linalg.norm(Y32[b])
        if yn == 0:
            assert np.all(X[b] == 0)
            continue
        assert abs(np.linalg.norm(X[b]) - 1.0) < 1e-6
        np.testing.assert_allclose(Q @ X[b], Y32[b] / yn, atol=1e-6)


def test_features_bf16_within_the_rounding_bound():
    """With BF16 rounding on, every feature is a BF16 number, within the bound that rounding y
    and a (unit roundoff u = 2^-8, relative error at most 2u + u^2 per product, and
    sum |a_m y_m| <= ||a|| ||y||) and rounding the result (u |x|) give: 2u + u^2 + u |x|."""
    from oracle import quant
    _, A = _orthonormal_dictionary(7, M=64)
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((8, 64))
    Xb = mlp.features(A.astype(np.float32), Y.astype(np.float32), round_bf16=True)
    Xe = mlp.features(A.astype(np.float32), Y.astype(np.float32), round_bf16=False)
    assert np.array_equal(quant.bf16_round(Xb.astype(np.float32)).astype(np.float64), Xb)
    u = 2.0 ** -8
    assert np.all(np.abs(Xb - Xe) <= (2 * u + u * u) * 1.001 + u * np.abs(Xe))
    assert np.any(Xb != Xe)


def test_logits_closed_form_without_hidden_layer():
    """With W1 = 0 and b1 = 0 the hidden layer is GELU(0) = 0, so the logits are exactly
    b2 + beta |x| (the skip term), with and without BF16 rounding."""
    X, Yl, W1, b1, W2, b2 = _instance(9)
    for rb in (False, True):
        O = mlp.logits(X, np.zeros_like(W1), np.zeros_like(b1), W2, b2, round_bf16=rb, beta=2.5)
        np.testing.assert_allclose(O, b2[None, :] + 2.5 * np.abs(X), rtol=0, atol=1e-15)


def test_logits_match_the_training_forward_pass():
    """logits() and the forward pass inside loss_and_grads() are separate code: the weighted BCE
    evaluated here from logits() (as (1 - y + pw y) log(1 + e^o) - pw y o, an algebraically
    equal form) equals loss_and_grads()'s loss, and a central difference of that loss in beta
    equals loss_and_grads()'s d loss / d beta."""
    X, Yl, W1, b1, W2, b2 = _instance(10)
    pw = 6.0

    def loss_from_logits(beta):
        O = mlp.logits(X, W1, b1, W2, b2, round_bf16=False, beta=beta)
        return np.mean((1 - Yl + pw * Yl) * np.logaddexp(0.0, O) - pw * Yl * O)

    for beta in (0.0, 1.7, -0.8):
        loss, *_, dbeta = mlp.loss_and_grads(X, Yl, W1, b1, W2, b2, pw, False, beta)
        assert abs(loss_from_logits(beta) - loss) <= 1e-12 * abs(loss)
        h = 1e-5
        fd = (loss_from_logits(beta + h) - loss_from_logits(beta - h)) / (2 * h)
        assert abs(fd - dbeta) <= 1e-7 * max(abs(dbeta), 1e-3)
