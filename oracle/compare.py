"""Comparison of a batched OMP result with the FP64 oracle under the stated tolerances.

Test infrastructure, like the rest of this package: the tests and the benchmark's CPU leg (its
error report) call it; the product path never does.

Rules (readings of the parity requirements of Alg. 1's outputs):
  * supports are compared step by step; at the first step j where they differ the oracle's
    top-two score margin (s1 - s2) / s1 must be <= MARGIN (a near-tie), and the result's atom
    must score at least (1 - MARGIN) s1 on the oracle's residual there;
  * from step j on the result's own picks are checked as steps of Alg. 1 along its own support
    (the oracle's greedy replayed with the result's prefix forced): at each later step the pick
    is the greedy one, or a near-tie under the same two conditions;
  * such a signal is counted as tie-diverged, and its coefficients and residual norm are checked
    against the least squares on its own support (forced replay); with an eps stop, its stopping
    step is checked against the residuals along that support;
  * coefficients: ||x - x_ref||_2 / ||x_ref||_2 <= COEF_RTOL per signal;
  * residual norm: | ||r|| - ||r||_ref | <= RESID_RTOL ||r||_ref + RESID_YTOL ||y||;
  * iteration counts match, unless the eps stop decided differently with the oracle's residual
    within 1e-4 relative of the threshold (a near-threshold stop).
"""
from __future__ import annotations

import numpy as np

from oracle import omp

MARGIN = 1e-3
COEF_RTOL = 1e-4
RESID_RTOL = 1e-4
RESID_YTOL = 1e-6
THR_RTOL = 1e-4


class ParityError(AssertionError):
    pass


def _top2(s):
    """(lowest index of the maximum, the maximum, the second largest score)."""
    n = int(np.argmax(s))
    s2 = np.partition(s, -2)[-2] if s.shape[0] > 1 else 0.0
    return n, float(s[n]), float(s2)


def _check_picks_along(A, y, picks, start, violations, tag):
    """Steps start..len(picks)-1 of Alg. 1 with the result's own prefix forced. Returns
    (number of non-greedy picks, residual norms along the support)."""
    scores, rn = omp.prefix_scores(A, y, picks)
    off = 0
    for t in range(start, len(picks)):
        s = scores[t]
        n, s1, s2 = _top2(s)
        g = int(picks[t])
        if g == n:
            continue
        margin = (s1 - s2) / s1 if s1 > 0 else 0.0
        rel = s[g] / s1 if s1 > 0 else 1.0
        off += 1
        if margin > MARGIN or rel < 1.0 - MARGIN:
            violations.append(f"{tag}: step {t} picks {g} (score {rel:.6f} of the best, "
                              f"margin {margin:.3g}) where Alg. 1 picks {n}")
    return off, rn


def compare(A, Y, ref: omp.OmpResult, sup, X, n_iter=None, resid=None, eps=0.0,
            eps_relative=True, rows=None, strict=True):
    """sup, X: (B, S) results (numpy); ref: the oracle's result for the same signals.

    Returns a dict of statistics: counts (signals, tie_diverged, off_greedy_steps,
    near_threshold, pick_mismatch_signals: signals with a pick that is neither the greedy one nor
    a near-tie, violations) and per-signal errors (coef_rel, resid_abs, resid_rel,
    resid_over_tol: the residual error over its tolerance, <= 1 passes). strict=True raises
    ParityError at the first violation; strict=False records every violation (for reports)."""
    A = np.asarray(A, dtype=np.float64)
    B = sup.shape[0]
    rows = np.arange(B) if rows is None else np.asarray(rows)
    violations: list[str] = []
    coef_rel = np.zeros(B)
    resid_abs = np.full(B, np.nan)
    resid_rel = np.full(B, np.nan)
    resid_over = np.full(B, np.nan)
    st = {"signals": B, "tie_diverged": 0, "off_greedy_steps": 0, "near_threshold": 0,
          "pick_mismatch_signals": 0}

    def fail(msg):
        if strict:
            raise ParityError(msg)
        violations.append(msg)

    for i in range(B):
        tag = f"signal {rows[i]}"
        y = np.asarray(Y[i], dtype=np.float64)
        yn = float(np.linalg.norm(y))
        kg = int(np.sum(sup[i] >= 0))
        ko = int(ref.n_iter[i])
        if n_iter is not None and int(n_iter[i]) != kg:
            fail(f"{tag}: n_iter {n_iter[i]} but {kg} support entries")
        if not (np.all(sup[i, :kg] >= 0) and np.all(sup[i, kg:] == -1) and np.all(X[i, kg:] == 0)):
            fail(f"{tag}: support or coefficients not padded with -1 / 0 after {kg} entries")
        gs, os_ = sup[i, :kg], ref.support[i, :ko]
        common = min(kg, ko)
        diff = np.flatnonzero(gs[:common] != os_[:common])
        thr = eps * yn if eps_relative else eps
        replay = False
        if diff.size:
            j = int(diff[0])
            m = float(ref.margin[i, j])
            local: list[str] = []
            if m > MARGIN:
                local.append(f"{tag}: support differs at step {j} with oracle margin {m}")
            off, rn = _check_picks_along(A, y, gs, j, local, tag)
            if local:
                st["pick_mismatch_signals"] += 1
            for v in local:
                fail(v)
            st["off_greedy_steps"] += off
            if eps > 0 and kg > 0:
                # stopped when (and only when) the residual along its own support reached eps
                tol = THR_RTOL * thr + RESID_YTOL * yn
                if kg < sup.shape[1] and rn[kg] > thr + tol:
                    fail(f"{tag}: stopped at {kg} with residual {rn[kg]} above eps {thr}")
                late = np.flatnonzero(rn[1:kg] < thr - tol)
                if late.size:
                    fail(f"{tag}: continued past step {late[0] + 1} with residual below eps")
            st["tie_diverged"] += 1
            replay = True
        elif kg != ko:
            kk = min(kg, ko)
            rk = ref.resid_trace[i, kk - 1] if kk > 0 else yn
            if not (eps > 0 and abs(rk - thr) <= THR_RTOL * thr + RESID_YTOL * yn):
                fail(f"{tag}: {kg} iterations against the oracle's {ko}")
            st["near_threshold"] += 1
            replay = True
        if replay:
            xr, rn_r = omp.replay_support(A, y, gs)
            r_ref = float(rn_r[-1]) if kg else yn
        else:
            xr = ref.coef[i, :ko]
            r_ref = float(ref.resid_norm[i])
        xg = np.asarray(X[i, :kg], dtype=np.float64)
        den = float(np.linalg.norm(xr))
        if den > 0:
            coef_rel[i] = float(np.linalg.norm(xg - xr)) / den
            if coef_rel[i] > COEF_RTOL:
                fail(f"{tag}: coefficient error {coef_rel[i]}")
        if resid is not None:
            err = abs(float(resid[i]) - r_ref)
            tol = RESID_RTOL * r_ref + RESID_YTOL * yn
            resid_abs[i] = err
            resid_rel[i] = err / r_ref if r_ref > 0 else (0.0 if err == 0 else np.inf)
            resid_over[i] = err / tol if tol > 0 else (0.0 if err == 0 else np.inf)
            if err > tol:
                fail(f"{tag}: residual {resid[i]} against {r_ref}")
    st.update(violations=violations, coef_rel=coef_rel, resid_abs=resid_abs, resid_rel=resid_rel,
              resid_over_tol=resid_over,
              max_coef_rel=float(coef_rel.max()) if B else 0.0,
              median_coef_rel=float(np.median(coef_rel)) if B else 0.0,
              max_resid_over_tol=float(np.nanmax(resid_over)) if B and resid is not None else None)
    return st


def error_report(st):
    """The error figures of a non-strict comparison, as plain numbers for a report line."""
    B = st["signals"]
    out = {"signals": B,
           "max_coef_rel_err": st["max_coef_rel"],
           "median_coef_rel_err": st["median_coef_rel"],
           "tie_diverged": st["tie_diverged"],
           "off_greedy_steps": st["off_greedy_steps"],
           "near_threshold_stops": st["near_threshold"],
           "violations": len(st["violations"]),
           "mismatch_rate_at_margin_gt_1e-3": st["pick_mismatch_signals"] / max(B, 1)}
    if st["max_resid_over_tol"] is not None:
        out["max_resid_rel_err"] = float(np.nanmax(st["resid_rel"])) if B else 0.0
        out["max_resid_err_over_tol"] = st["max_resid_over_tol"]
    return out
