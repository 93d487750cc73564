"""FP64 Orthogonal Matching Pursuit, written from the paper (test infrastructure only).

Definition followed (Alg. 1): r_0 = y; for k = 1..S pick n* = argmax_n |<r_{k-1}, a_n>| / ||a_n||,
add n* to the support, solve the least-squares problem on the support, set r_k = y - A_S x_k, and
stop when ||r_k|| <= eps.

Readings of points the paper leaves open (each is also listed in the design notes):
  * ties in the argmax: the smallest index wins (scan ascending, replace only on a strict >);
  * stop test: after each update; ``eps_relative`` (default) compares ||r_k|| with eps * ||y||,
    otherwise with the absolute eps of Alg. 1; eps = 0 runs exactly S steps unless r becomes
    exactly 0 or the picked atom is dependent;
  * dependent atom: if the squared distance of a_{n*} to span(A_S) is <= 1e-10 ||a_{n*}||^2 the
    signal stops at k-1 without appending n*; atoms already in the support are not masked from
    the argmax (their score is 0 in exact arithmetic);
  * y = 0: empty support;
  * zero-norm atoms score 0 (0/0 is read as 0).

Three modes, all FP64 on the caller's raw (unnormalised) A:
  ``omp_reference``       one signal, x_k re-solved from scratch with LAPACK least squares (gelsd);
  ``omp_batch``           batched "timed" mode: one dgemm for A^T R over the live signals
                          (Sec. 3.2, eq:bmm) and the progressive Cholesky append V_k of Sec. 2.1;
  ``omp_inverse_cholesky`` one signal with the v0 recurrence F_k of Sec. 2.3 and the projection
                          y_hat = A_k F_k (A_k F_k)^T y; also returns F.
"""
from __future__ import annotations

import dataclasses

import numpy as np

DEPENDENT_RTOL = 1e-10
STOP_ITERS, STOP_EPS, STOP_DEPENDENT, STOP_ZERO = 0, 1, 2, 3


@dataclasses.dataclass
class OmpResult:
    """Batched OMP output. Arrays are (B, S) unless stated; support is in selection order."""

    support: np.ndarray      # int64, -1 padded
    coef: np.ndarray         # float64, aligned with support, 0 padded (raw scale of A)
    n_iter: np.ndarray       # (B,) int64
    resid_norm: np.ndarray   # (B,) final ||r||
    resid_trace: np.ndarray  # ||r_k|| after step k (nan past n_iter)
    margin: np.ndarray       # (s1 - s2) / s1 of the scores at step k (nan past the last pick)
    stop: np.ndarray         # (B,) STOP_* code
    y_norm: np.ndarray       # (B,) ||y||


def atom_norms(A: np.ndarray) -> np.ndarray:
    """||a_n||_2 in FP64."""
    A64 = np.asarray(A, dtype=np.float64)
    return np.sqrt(np.einsum("mn,mn->n", A64, A64))


def _inv_or_zero(norms: np.ndarray) -> np.ndarray:
    out = np.zeros_like(norms)
    nz = norms > 0
    out[nz] = 1.0 / norms[nz]
    return out


def select(A: np.ndarray, inv_norm: np.ndarray, r: np.ndarray):
    """Selection step of Alg. 1 for one residual: (n*, margin).

    n* is the smallest index attaining the maximum of |<r, a_n>| / ||a_n||; the margin is
    (s1 - s2) / s1 with s1 >= s2 the two largest scores (0 when s1 = 0)."""
    s = np.abs(A.T @ r) * inv_norm
    n = int(np.argmax(s))            # first occurrence of the maximum = lowest index
    if s.shape[0] < 2:
        return n, 1.0
    s1 = s[n]
    s2 = np.partition(s, -2)[-2]
    return n, (float((s1 - s2) / s1) if s1 > 0 else 0.0)


def _threshold(y_norm, eps, eps_relative):
    return eps * y_norm if eps_relative else eps


def omp_reference(A, y, S, eps=0.0, eps_relative=True):
    """Alg. 1 for one signal with x_k = argmin ||y - A_{S_k} x|| solved from scratch each step
    (LAPACK gelsd through numpy.linalg.lstsq). Returns an OmpResult with B = 1."""
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    M, N = A.shape
    norms = atom_norms(A)
    inv = _inv_or_zero(norms)
    res = _empty_result(1, S)
    y_norm = float(np.linalg.norm(y))
    res.y_norm[0] = y_norm
    res.resid_norm[0] = y_norm
    thr = _threshold(y_norm, eps, eps_relative)
    if y_norm == 0.0:
        res.stop[0] = STOP_ZERO
        return res
    supp: list[int] = []
    r = y.copy()
    x = np.zeros(0)
    for k in range(S):
        n, margin = select(A, inv, r)
        res.margin[0, k] = margin
        a = A[:, n]
        if supp:
            As = A[:, supp]
            proj = As @ np.linalg.lstsq(As, a, rcond=None)[0]
            dist2 = float(np.dot(a - proj, a - proj))
        else:
            dist2 = float(np.dot(a, a))
        if dist2 <= DEPENDENT_RTOL * norms[n] ** 2:
            res.stop[0] = STOP_DEPENDENT
            break
        supp.append(n)
        As = A[:, supp]
        x = np.linalg.lstsq(As, y, rcond=None)[0]
        r = y - As @ x
        rn = float(np.linalg.norm(r))
        res.resid_trace[0, k] = rn
        res.n_iter[0] = k + 1
        res.resid_norm[0] = rn
        if rn <= thr:
            res.stop[0] = STOP_EPS
            break
    else:
        res.stop[0] = STOP_ITERS
    kk = len(supp)
    res.support[0, :kk] = supp
    res.coef[0, :kk] = x[:kk] if kk else x
    return res


def _empty_result(B, S):
    return OmpResult(
        support=np.full((B, S), -1, dtype=np.int64),
        coef=np.zeros((B, S)),
        n_iter=np.zeros(B, dtype=np.int64),
        resid_norm=np.zeros(B),
        resid_trace=np.full((B, S), np.nan),
        margin=np.full((B, S), np.nan),
        stop=np.full(B, STOP_ITERS, dtype=np.int64),
        y_norm=np.zeros(B),
    )


def omp_batch(A, Y, S, eps=0.0, eps_relative=True, chunk=256) -> OmpResult:
    """Batched timed-mode OMP in FP64 (the CPU baseline).

    Per step, over the live signals of a chunk:
      C = R A (one dgemm, Sec. 3.2 eq:bmm); s = |C| / ||a_n||; n* = first argmax;
      progressive Cholesky append (Sec. 2.1): V_k = [[V_{k-1}, 0], [z^T, sqrt(||a||^2 - ||z||^2)]]
      with V_{k-1} z = A_{k-1}^T a_{n*};
      u = V_k^{-1} A_k^T y grows by one entry (forward substitution is incremental);
      x_k = V_k^{-T} u (back substitution); r_k = y - A_k x_k.
    The selected atoms are kept in a layout-separated (B, S, M) array so a column write is one
    contiguous row (Sec. 3.1).
    """
    A = np.asarray(A, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[None, :]
    B = Y.shape[0]
    out = _empty_result(B, S)
    for c0 in range(0, B, chunk):
        _omp_chunk(A, Y[c0: c0 + chunk], S, eps, eps_relative, out, c0)
    return out


def _omp_chunk(A, Y, S, eps, eps_relative, out, off):
    M, N = A.shape
    L = Y.shape[0]
    At = np.ascontiguousarray(A.T)
    norms = atom_norms(A)
    inv = _inv_or_zero(norms)
    y_norm = np.sqrt(np.einsum("bm,bm->b", Y, Y))
    thr = eps * y_norm if eps_relative else np.full(L, eps)
    out.y_norm[off: off + L] = y_norm
    out.resid_norm[off: off + L] = y_norm
    R = Y.copy()
    As = np.zeros((L, S, M))        # selected atoms, one contiguous row per column of A_k
    V = np.zeros((L, S, S))         # lower-triangular Cholesky factor of A_k^T A_k
    u = np.zeros((L, S))            # V_k^{-1} A_k^T y
    x = np.zeros((L, S))
    sup = np.full((L, S), -1, dtype=np.int64)
    kk = np.zeros(L, dtype=np.int64)
    live = np.flatnonzero(y_norm > 0)
    out.stop[off: off + L][y_norm == 0] = STOP_ZERO
    for k in range(S):
        if live.size == 0:
            break
        Rl = R[live]
        s = np.abs(Rl @ A) * inv                      # (l, N)
        n = np.argmax(s, axis=1)                      # first occurrence: lowest index on ties
        if N >= 2:
            top2 = np.partition(s, N - 2, axis=1)[:, N - 2]
            s1 = s[np.arange(live.size), n]
            out.margin[off + live, k] = np.where(s1 > 0, (s1 - top2) / np.where(s1 > 0, s1, 1), 0)
        a = At[n]                                     # (l, M)
        w = np.einsum("lkm,lm->lk", As[live, :k], a)  # A_{k-1}^T a_{n*}
        Vl = V[live]
        z = np.zeros((live.size, k))
        for i in range(k):                            # forward substitution V_{k-1} z = w
            z[:, i] = (w[:, i] - np.einsum("lj,lj->l", Vl[:, i, :i], z[:, :i])) / Vl[:, i, i]
        nrm2 = norms[n] ** 2
        delta = nrm2 - np.einsum("lk,lk->l", z, z)
        dep = delta <= DEPENDENT_RTOL * nrm2
        if dep.any():
            out.stop[off + live[dep]] = STOP_DEPENDENT
        keep = ~dep
        live = live[keep]
        if live.size == 0:
            break
        n, a, z, delta = n[keep], a[keep], z[keep], delta[keep]
        V[live, k, :k] = z
        V[live, k, k] = np.sqrt(delta)
        As[live, k] = a
        sup[live, k] = n
        kk[live] = k + 1
        aty = np.einsum("lm,lm->l", a, Y[live])
        u[live, k] = (aty - np.einsum("lj,lj->l", z, u[live, :k])) / V[live, k, k]
        Vl = V[live, : k + 1, : k + 1]
        xl = np.zeros((live.size, k + 1))
        for i in range(k, -1, -1):                    # back substitution V_k^T x = u
            xl[:, i] = (u[live, i] - np.einsum("lj,lj->l", Vl[:, i + 1:, i], xl[:, i + 1:])) \
                / Vl[:, i, i]
        x[live, : k + 1] = xl
        R[live] = Y[live] - np.einsum("lkm,lk->lm", As[live, : k + 1], xl)
        rn = np.sqrt(np.einsum("lm,lm->l", R[live], R[live]))
        out.resid_trace[off + live, k] = rn
        out.resid_norm[off + live] = rn
        out.n_iter[off + live] = k + 1
        done = rn <= thr[live]
        out.stop[off + live[done]] = STOP_EPS
        live = live[~done]
    out.support[off: off + L] = sup
    out.coef[off: off + L] = np.where(sup >= 0, x, 0.0)


def inverse_cholesky_append(F, w, nrm2):
    """One step of the v0 recurrence (Sec. 2.3).

    F is F_{k-1} ((k-1) x (k-1) upper triangular, F_{k-1} = V_{k-1}^{-T}), w = A_{k-1}^T a_{n*},
    nrm2 = ||a_{n*}||^2. Returns (F_k, z, gamma, delta) with z = F_{k-1}^T w,
    delta = nrm2 - ||z||^2, gamma = 1 / sqrt(delta) and F_k = [[F_{k-1}, -gamma F_{k-1} z],
    [0, gamma]] (gamma is nan when delta <= 0)."""
    k1 = F.shape[0]
    z = F.T @ w if k1 else np.zeros(0)
    delta = float(nrm2 - np.dot(z, z))
    gamma = 1.0 / np.sqrt(delta) if delta > 0 else np.nan
    Fk = np.zeros((k1 + 1, k1 + 1))
    Fk[:k1, :k1] = F
    Fk[:k1, k1] = -gamma * (F @ z) if k1 else 0.0
    Fk[k1, k1] = gamma
    return Fk, z, gamma, delta


def omp_inverse_cholesky(A, y, S, eps=0.0, eps_relative=True):
    """Alg. 1 for one signal with the v0 inverse-Cholesky recurrence (Sec. 2.3).

    Keeps F_k and b_k = (A_k F_k)^T y; the projection is y_hat = A_k F_k b_k (a matvec, no
    triangular solve) and the coefficients are x_k = F_k b_k. A^T a_{n*} restricted to the
    support is read from the Gram matrix G = A^T A (Sec. 2.2 precompute). Returns
    (OmpResult with B = 1, F_final)."""
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    G = A.T @ A
    norms = atom_norms(A)
    inv = _inv_or_zero(norms)
    res = _empty_result(1, S)
    y_norm = float(np.linalg.norm(y))
    res.y_norm[0] = y_norm
    res.resid_norm[0] = y_norm
    thr = _threshold(y_norm, eps, eps_relative)
    F = np.zeros((0, 0))
    b = np.zeros(0)
    supp: list[int] = []
    if y_norm == 0.0:
        res.stop[0] = STOP_ZERO
        return res, F
    r = y.copy()
    for k in range(S):
        n, margin = select(A, inv, r)
        res.margin[0, k] = margin
        w = G[supp, n]
        Fk, z, gamma, delta = inverse_cholesky_append(F, w, G[n, n])
        if delta <= DEPENDENT_RTOL * norms[n] ** 2:
            res.stop[0] = STOP_DEPENDENT
            break
        F = Fk
        supp.append(n)
        Ak = A[:, supp]
        Q = Ak @ F                      # orthonormal columns
        b = Q.T @ y
        r = y - Q @ b                   # y - y_hat, y_hat = A_k F_k (A_k F_k)^T y
        rn = float(np.linalg.norm(r))
        res.resid_trace[0, k] = rn
        res.n_iter[0] = k + 1
        res.resid_norm[0] = rn
        if rn <= thr:
            res.stop[0] = STOP_EPS
            break
    else:
        res.stop[0] = STOP_ITERS
    kk = len(supp)
    res.support[0, :kk] = supp
    res.coef[0, :kk] = F @ b if kk else b
    return res, F


def replay_support(A, y, support):
    """Least squares on the first k atoms of a given support, for k = 1..len(support).

    Returns (coef of the full support, residual norms after each k). Used to check a signal
    whose support legitimately diverged from the oracle's at a near-tie."""
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    supp = [int(s) for s in support if s >= 0]
    rn = np.zeros(len(supp))
    x = np.zeros(0)
    for k in range(1, len(supp) + 1):
        As = A[:, supp[:k]]
        x = np.linalg.lstsq(As, y, rcond=None)[0]
        rn[k - 1] = np.linalg.norm(y - As @ x)
    return x, rn


def scores(A, r):
    """|<r, a_n>| / ||a_n|| for every atom (FP64), zero-norm atoms scoring 0."""
    A = np.asarray(A, dtype=np.float64)
    return np.abs(A.T @ np.asarray(r, dtype=np.float64)) * _inv_or_zero(atom_norms(A))


def omp_candidates_reference(A, y, S, cand, tau, eps=0.0, eps_relative=True):
    """Alg. 1 with a candidate-restricted start and a residual-drop fallback (FP64, one signal).

    While restricted, step k selects only among the candidate atoms `cand` (lowest atom index on
    ties) and is accepted if its normalised drop (||r_{k-1}||^2 - ||r_k||^2) / ||r_{k-1}||^2 is at
    least tau[k] (and the candidate is not dependent and scores above 0). The first rejected step
    ends the restricted phase: that step and every later one select among all atoms, exactly as
    Alg. 1. Returns (OmpResult with B = 1, fallback step or -1)."""
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    norms = atom_norms(A)
    inv = _inv_or_zero(norms)
    cand = np.asarray(sorted(int(c) for c in cand))
    res = _empty_result(1, S)
    y_norm = float(np.linalg.norm(y))
    res.y_norm[0] = y_norm
    res.resid_norm[0] = y_norm
    thr = _threshold(y_norm, eps, eps_relative)
    if y_norm == 0.0:
        res.stop[0] = STOP_ZERO
        return res, -1
    supp: list[int] = []
    r = y.copy()
    x = np.zeros(0)
    restricted = True
    fb = -1
    for k in range(S):
        while True:
            if restricted:
                s = np.abs(A[:, cand].T @ r) * inv[cand]
                j = int(np.argmax(s))
                n, sc = int(cand[j]), float(s[j])
                s2 = np.partition(s, -2)[-2] if s.size > 1 else 0.0
                margin = (sc - s2) / sc if sc > 0 else 0.0
            else:
                n, margin = select(A, inv, r)
                sc = 1.0
            a = A[:, n]
            if supp:
                As = A[:, supp]
                dist2 = float(np.sum((a - As @ np.linalg.lstsq(As, a, rcond=None)[0]) ** 2))
            else:
                dist2 = float(a @ a)
            dep = dist2 <= DEPENDENT_RTOL * norms[n] ** 2
            if restricted:
                ok = sc > 0 and not dep
                if ok:
                    As = A[:, supp + [n]]
                    xn = np.linalg.lstsq(As, y, rcond=None)[0]
                    rn = y - As @ xn
                    drop = (r @ r - rn @ rn) / (r @ r)
                    ok = drop >= tau[k]
                if not ok:
                    restricted = False
                    fb = k
                    continue
            break
        res.margin[0, k] = margin
        if dep:
            res.stop[0] = STOP_DEPENDENT
            break
        supp.append(n)
        As = A[:, supp]
        x = np.linalg.lstsq(As, y, rcond=None)[0]
        r = y - As @ x
        rnn = float(np.linalg.norm(r))
        res.resid_trace[0, k] = rnn
        res.n_iter[0] = k + 1
        res.resid_norm[0] = rnn
        if rnn <= thr:
            res.stop[0] = STOP_EPS
            break
    kk = len(supp)
    res.support[0, :kk] = supp
    res.coef[0, :kk] = x[:kk] if kk else x
    return res, fb


def prefix_scores(A, y, picks):
    """Alg. 1's selection step evaluated along a given support.

    For t = 0..k (k = len(picks)), r_t = y - P_t y with P_t the orthogonal projector onto the span
    of the first t picked atoms (r_t is the least-squares residual of that prefix, as in Alg. 1).
    Returns (scores, rnorm): scores[t, n] = |<r_t, a_n>| / ||a_n|| for t < k (FP64, zero-norm
    atoms scoring 0) and rnorm[t] = ||r_t|| for t = 0..k. The projectors come from one Householder
    QR of A_S (LAPACK), whose first t columns of Q span the first t picked atoms."""
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    picks = [int(p) for p in picks]
    k = len(picks)
    R = np.zeros((k + 1, y.shape[0]))
    R[0] = y
    if k:
        Q, _ = np.linalg.qr(A[:, picks])
        coef = Q.T @ y
        for t in range(k):
            R[t + 1] = R[t] - coef[t] * Q[:, t]
    inv = _inv_or_zero(atom_norms(A))
    scores = np.abs(R[:k] @ A) * inv[None, :]
    return scores, np.sqrt(np.einsum("tm,tm->t", R, R))
