"""Comparison of CUDA-path results with the FP64 oracle under the stated tolerances.

Rules (readings of the parity requirements):
  * supports are compared step by step; at the first step where they differ the oracle's
    top-two score margin must be <= 1e-3 (a near-tie) -- any difference at a larger margin fails;
    such a signal is counted as tie-diverged and its coefficients and residual are checked
    against the oracle's least squares on the GPU's own support (forced replay);
  * coefficients: ||x_gpu - x_ref||_2 / ||x_ref||_2 <= 1e-4 per signal;
  * residual norm: | ||r||_gpu - ||r||_ref | <= 1e-4 ||r||_ref + 1e-6 ||y||;
  * iteration counts must match unless the eps stop decided differently with the oracle's
    residual within 1e-4 relative of the threshold (a near-threshold stop).
"""
import numpy as np

from oracle import omp

MARGIN = 1e-3
COEF_RTOL = 1e-4
RESID_RTOL = 1e-4
RESID_YTOL = 1e-6


def compare(A, Y, ref: omp.OmpResult, sup, X, n_iter=None, resid=None, eps=0.0,
            eps_relative=True, rows=None):
    """sup, X: (B, S) GPU outputs (numpy); ref: oracle result for the same rows.
    Returns a dict of statistics; raises AssertionError on a violation."""
    B = sup.shape[0]
    rows = np.arange(B) if rows is None else np.asarray(rows)
    stats = {"signals": B, "tie_diverged": 0, "near_threshold": 0, "max_coef_rel": 0.0,
             "max_resid_err": 0.0}
    for i in range(B):
        y = Y[i].astype(np.float64)
        yn = np.linalg.norm(y)
        kg = int(np.sum(sup[i] >= 0))
        ko = int(ref.n_iter[i])
        if n_iter is not None:
            assert int(n_iter[i]) == kg, (rows[i], n_iter[i], kg)
        gs, os_ = sup[i, :kg], ref.support[i, :ko]
        common = min(kg, ko)
        diff = np.flatnonzero(gs[:common] != os_[:common])
        replay = False
        if diff.size:
            j = int(diff[0])
            m = ref.margin[i, j]
            assert m <= MARGIN, f"signal {rows[i]}: support differs at step {j} with margin {m}"
            stats["tie_diverged"] += 1
            replay = True
        elif kg != ko:
            thr = eps * yn if eps_relative else eps
            kk = min(kg, ko)
            rk = ref.resid_trace[i, kk - 1] if kk > 0 else yn
            assert eps > 0 and abs(rk - thr) <= 1e-4 * thr + RESID_YTOL * yn, \
                f"signal {rows[i]}: {kg} GPU vs {ko} oracle iterations"
            stats["near_threshold"] += 1
            replay = True
        if replay:
            xr, rn = omp.replay_support(A, y, gs)
            r_ref = rn[-1] if kg else yn
        else:
            xr = ref.coef[i, :ko]
            r_ref = ref.resid_norm[i]
        xg = X[i, :kg].astype(np.float64)
        assert np.all(X[i, kg:] == 0) and np.all(sup[i, kg:] == -1)
        den = np.linalg.norm(xr)
        if den > 0:
            rel = np.linalg.norm(xg - xr) / den
            stats["max_coef_rel"] = max(stats["max_coef_rel"], rel)
            assert rel <= COEF_RTOL, f"signal {rows[i]}: coefficient error {rel}"
        if resid is not None:
            err = abs(float(resid[i]) - r_ref)
            stats["max_resid_err"] = max(stats["max_resid_err"], err / (r_ref + yn * 1e-2))
            assert err <= RESID_RTOL * r_ref + RESID_YTOL * yn, \
                f"signal {rows[i]}: residual {resid[i]} vs {r_ref}"
    return stats
