"""FP64 reference of the learned proposal network (test infrastructure only).

Network (the learned-proposal design; the paper has no learned component):
  x  = features of a signal (the first correlation, normalised)
  Z1 = X W1^T + b1,  H = GELU(Z1) = Z1 Phi(Z1)  (exact, through scipy.special.erf)
  O  = H W2^T + b2 + beta |X|   (per-atom logits; beta a scalar skip-term scale)
Loss: mean over all B x N entries of the weighted BCE with logits
  l = pw y softplus(-o) + (1 - y) softplus(o),   dl/do = sigma(o) (1 - y + pw y) - pw y.

``round_bf16=True`` rounds to BF16 (oracle.quant.bf16_round) at exactly the points where the
CUDA path stores BF16: the features X, both weight matrices, the activations H, the logit
gradient dO and the pre-activation gradient dZ1. Everything else is FP64.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from oracle import quant


def _bf(x, on):
    return quant.bf16_round(np.asarray(x, dtype=np.float32)).astype(np.float64) if on else \
        np.asarray(x, dtype=np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def softplus(x):
    return np.where(x > 0, x + np.log1p(np.exp(-np.abs(x))), np.log1p(np.exp(x)))


def features(A, Y, round_bf16=True):
    """x_n = <y, a_n> / (||a_n|| ||y||) from BF16-rounded y and a (FP64 products), then BF16."""
    A = np.asarray(A, dtype=np.float32)
    Y = np.asarray(Y, dtype=np.float32)
    Aq = _bf(A, round_bf16)
    Yq = _bf(Y, round_bf16)
    an = np.sqrt(np.sum(np.asarray(A, np.float64) ** 2, axis=0))
    yn = np.sqrt(np.sum(np.asarray(Y, np.float64) ** 2, axis=1))
    inv_a = np.where(an > 0, 1.0 / np.where(an > 0, an, 1), 0.0)
    inv_y = np.where(yn > 0, 1.0 / np.where(yn > 0, yn, 1), 0.0)
    X = (Yq @ Aq) * inv_a[None, :] * inv_y[:, None]
    return _bf(X, round_bf16)


def labels_matrix(sup, N):
    Ylab = np.zeros((sup.shape[0], N))
    for b in range(sup.shape[0]):
        s = sup[b][sup[b] >= 0]
        Ylab[b, s] = 1.0
    return Ylab


def loss_and_grads(X, Ylab, W1, b1, W2, b2, pos_weight, round_bf16=True, beta=0.0):
    """Returns (loss, dW1, db1, dW2, db2, dbeta) of the mean weighted BCE."""
    X = np.asarray(X, dtype=np.float64)
    B, N = Ylab.shape
    W1q = _bf(W1, round_bf16)
    W2q = _bf(W2, round_bf16)
    Z1 = X @ W1q.T + b1
    H = _bf(gelu(Z1), round_bf16)
    O = H @ W2q.T + b2 + beta * np.abs(X)
    pw = pos_weight
    inv = 1.0 / (B * N)
    loss = np.sum(pw * Ylab * softplus(-O) + (1 - Ylab) * softplus(O)) * inv
    sig = 1.0 / (1.0 + np.exp(-O))
    dO_exact = (sig * (1 - Ylab + pw * Ylab) - pw * Ylab) * inv
    dbeta = float(np.sum(dO_exact * np.abs(X)))
    dO = _bf(dO_exact, round_bf16)
    dW2 = dO.T @ H
    db2 = dO.sum(axis=0)
    dH = dO @ W2q
    dZ1 = _bf(dH * gelu_grad(Z1), round_bf16)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    return loss, dW1, db1, dW2, db2, dbeta


def logits(X, W1, b1, W2, b2, round_bf16=True, beta=0.0):
    W1q = _bf(W1, round_bf16)
    W2q = _bf(W2, round_bf16)
    X = np.asarray(X, np.float64)
    H = _bf(gelu(X @ W1q.T + b1), round_bf16)
    return H @ W2q.T + b2 + beta * np.abs(X)


def topk_lowest_index(v, K):
    """Indices of the K largest entries of each row, lowest index first among equal values,
    returned in ascending index order."""
    out = np.zeros((v.shape[0], K), dtype=np.int64)
    for b in range(v.shape[0]):
        order = np.lexsort((np.arange(v.shape[1]), -v[b]))
        out[b] = np.sort(order[:K])
    return out
