"""A scikit-learn-style front end for the batched OMP solve (argument marshalling only).

``orthogonal_mp(X, y, ...)`` and ``OrthogonalMatchingPursuit`` take their arguments the way
scikit-learn's functions of the same names do -- X is the (n_samples, n_features) dictionary
(here M x N, one atom per column), y one target (n_samples,) or several (n_samples, n_targets),
one OMP problem per target -- and run every target through one batched solve of the C ABI
(``omp_solve_batch_ex``) on the GPU. Differences from scikit-learn, by design:
  * the selection divides by the column norms (|<r, a_n>| / ||a_n||, Alg. 1 of the paper on a
    dictionary of any scale), which equals scikit-learn's rule on the unit-norm dictionaries it
    asks for; coefficients are in the scale of the given X either way;
  * ``precision`` picks the correlation path ("fp32", "bf16" or "fp8"; the atom picked is the
    FP32 path's wherever the top-two margin exceeds the rescoring bound);
  * at most 256 iterations per target (the library's limit).
``tol`` is scikit-learn's: the maximum squared norm of the residual, so the stop test is
||r||^2 <= tol (absolute; it takes precedence over n_nonzero_coefs). There is no CPU fallback.
"""
from __future__ import annotations

import numpy as np

from . import omp

_MAX_ITERS = 256


def _as_cuda_f32(a, device):
    import torch
    if isinstance(a, torch.Tensor):
        return a.detach().to(device=device, dtype=torch.float32)
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(device)


def _solve(X, Y_rows, S, eps, eps_relative, precision, device):
    """One batched solve: X (M, N) dictionary, Y_rows (B, M) signals. Returns (coef (B, N) dense
    float32 tensor, n_iter (B,) int32 tensor, X_t) on the device."""
    import torch
    M, N = X.shape
    B = Y_rows.shape[0]
    Xd = X.t().contiguous().t()                     # column-major (stride (1, M))
    solver = omp.OmpSolver(M, N, max_batch=B, max_iters=S, precision=precision,
                           eps_relative=eps_relative, device=device.index or 0)
    try:
        Xc, sup, n_iter, _, _ = solver.solve(Xd, Y_rows.contiguous(), S, eps, diagnostics=True)
        coef = torch.zeros((B, N), dtype=torch.float32, device=device)
        valid = sup >= 0
        rows = torch.arange(B, device=device)[:, None].expand_as(sup)
        coef[rows[valid], sup[valid].long()] = Xc[valid]
        torch.cuda.synchronize(device)
    finally:
        solver.close()
    return coef, n_iter


def _iters(n_features, n_samples, n_nonzero_coefs, tol):
    if tol is not None:
        if tol < 0:
            raise ValueError("tol must be >= 0")
        return min(n_samples, n_features, _MAX_ITERS)
    if n_nonzero_coefs is None:
        n_nonzero_coefs = max(int(0.1 * n_features), 1)
    if not 1 <= n_nonzero_coefs <= min(n_samples, n_features, _MAX_ITERS):
        raise ValueError(f"n_nonzero_coefs must be in [1, {min(n_samples, n_features, _MAX_ITERS)}]")
    return int(n_nonzero_coefs)


def orthogonal_mp(X, y, *, n_nonzero_coefs=None, tol=None, precision="bf16",
                  return_n_iter=False, device="cuda"):
    """Sparse codes of y over the dictionary X: coef (n_features,) for one target or
    (n_features, n_targets) for several, as numpy arrays (float32), plus the iteration counts
    when return_n_iter is set."""
    import torch
    dev = torch.device(device)
    Xt = _as_cuda_f32(X, dev)
    if Xt.dim() != 2:
        raise ValueError("X must be (n_samples, n_features)")
    yt = _as_cuda_f32(y, dev)
    single = yt.dim() == 1
    if single:
        yt = yt[:, None]
    if yt.dim() != 2 or yt.shape[0] != Xt.shape[0]:
        raise ValueError("y must be (n_samples,) or (n_samples, n_targets)")
    M, N = Xt.shape
    S = _iters(N, M, n_nonzero_coefs, tol)
    eps = float(np.sqrt(tol)) if tol is not None else 0.0
    coef, n_iter = _solve(Xt, yt.t(), S, eps, tol is None, precision, dev)
    out = coef.cpu().numpy().T
    out = out[:, 0] if single else out
    if return_n_iter:
        n = n_iter.cpu().numpy()
        return out, (int(n[0]) if single else n)
    return out


class OrthogonalMatchingPursuit:
    """Estimator with scikit-learn's interface: fit(X, y) stores coef_ ((n_features,) or
    (n_targets, n_features)), intercept_ and n_iter_; predict(X) = X coef_^T + intercept_.
    With fit_intercept (the default, as in scikit-learn) X and y are centred on the host first."""

    def __init__(self, *, n_nonzero_coefs=None, tol=None, fit_intercept=True, precision="bf16",
                 device="cuda"):
        self.n_nonzero_coefs = n_nonzero_coefs
        self.tol = tol
        self.fit_intercept = fit_intercept
        self.precision = precision
        self.device = device

    def get_params(self, deep=True):
        return {"n_nonzero_coefs": self.n_nonzero_coefs, "tol": self.tol,
                "fit_intercept": self.fit_intercept, "precision": self.precision,
                "device": self.device}

    def set_params(self, **params):
        for k, v in params.items():
            if k not in self.get_params():
                raise ValueError(f"unknown parameter {k}")
            setattr(self, k, v)
        return self

    def fit(self, X, y):
        X = np.asarray(X, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        single = y.ndim == 1
        Y = y[:, None] if single else y
        if self.fit_intercept:
            x_mean, y_mean = X.mean(axis=0), Y.mean(axis=0)
            Xc, Yc = X - x_mean, Y - y_mean
        else:
            x_mean, y_mean = np.zeros(X.shape[1]), np.zeros(Y.shape[1])
            Xc, Yc = X, Y
        coef, n_iter = orthogonal_mp(Xc, Yc, n_nonzero_coefs=self.n_nonzero_coefs, tol=self.tol,
                                     precision=self.precision, return_n_iter=True,
                                     device=self.device)
        coef = coef.T.astype(np.float64)             # (n_targets, n_features)
        intercept = y_mean - coef @ x_mean
        self.coef_ = coef[0] if single else coef
        self.intercept_ = float(intercept[0]) if single else intercept
        self.n_iter_ = int(n_iter[0]) if single else n_iter
        self.n_features_in_ = X.shape[1]
        return self

    def predict(self, X):
        X = np.asarray(X, dtype=np.float64)
        return X @ np.asarray(self.coef_).T + self.intercept_
