"""Comparison helpers for the GPU-vs-reference parity tests.

Tolerances (FP64 steps): |gpu - ref| <= REL * |ref| + ABS with REL = 1e-9 and ABS = 1e-11
(log-speedup predictions are O(0.1..1); the absolute floor covers values near zero, where a
relative bound is meaningless).  Standardized features and Gram entries: 1e-12 relative
to the row scale.  Rankings must be identical except in rows where the reference itself is
within TOL of a decision: two candidates closer than TOL, a candidate within TOL of the
threshold, or (for the sign counters) a prediction within TOL of zero.
"""
import numpy as np

REL = 1e-9
ABS = 1e-11


def close(gpu, ref, rel=REL, abs_=ABS):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nan_g, nan_r = np.isnan(gpu), np.isnan(ref)
    assert np.array_equal(nan_g, nan_r), f"NaN pattern differs at {np.argwhere(nan_g != nan_r)[:5]}"
    d = np.abs(gpu[~nan_r] - ref[~nan_r])
    lim = rel * np.abs(ref[~nan_r]) + abs_
    bad = d > lim
    assert not bad.any(), (
        f"{bad.sum()} of {bad.size} values out of tolerance; worst abs err {d.max():.3e}; "
        f"worst ratio {(d / lim).max():.3g}")
    return float(d.max()) if d.size else 0.0


def near_decision(pred_row, log_tau, tol):
    """True if this reference row has a near-tie, a near-threshold or a near-zero value."""
    v = pred_row[~np.isnan(pred_row)]
    if v.size == 0:
        return False
    s = np.sort(v)
    if s.size > 1 and np.min(np.diff(s)) < tol:
        return True
    if np.any(np.abs(v - log_tau) < tol) or np.any(np.abs(v) < tol):
        return True
    return False


def compare_rankings(gpu_code, ref_code, ref_pred_all, log_tau, tol=1e-8):
    gpu_code = np.asarray(gpu_code, dtype=np.uint32)
    ref_code = np.asarray(ref_code, dtype=np.uint32)
    diff = np.nonzero(gpu_code != ref_code)[0]
    for r in diff:
        assert near_decision(ref_pred_all[r], log_tau, tol), (
            f"row {r}: gpu code {gpu_code[r]:#x} != ref {ref_code[r]:#x} with no near decision; "
            f"ref preds {ref_pred_all[r]}")
    n_near = sum(near_decision(ref_pred_all[r], log_tau, tol) for r in range(len(ref_code)))
    return len(diff), n_near


def compare_counters(gpu_cnt, ref_cnt, slack=0):
    g = np.asarray(gpu_cnt, dtype=np.int64)[:14]
    r = np.asarray(ref_cnt, dtype=np.int64)[:14]
    assert np.all(np.abs(g - r) <= slack), f"counters differ: gpu {g.tolist()} ref {r.tolist()}"
