"""The identities behind the closed-form leave-one-version-out fits (RS_LOO_CLOSED), in plain
numpy FP64 on the CPU, against the reference's direct ridge fits (primal normal equations) of
the same leave-one-out training sets.  With M = K_PP + lambda I over a program's pairs for one
optimization, u = row i of M^-1, w_y = M^-1 y and w_1 = M^-1 1, deleting pair i gives:
  the reduced solutions (w - u w[i] / u_i) without entry i;
  the intercept from the downdated sums (1^T w_y - w_1[i] w_y[i] / u_i) / (1^T w_1 - w_1[i]^2 / u_i);
  the prediction at pair i's before version y_i - (w_y[i] - b w_1[i]) / u_i;
and none of them depends on the label at position i."""
import numpy as np
import pytest

import oracle
from paper_1910_07776_gb300 import synth

LAM = 1e-3


def _program(seed, feat):
    batch = synth.make_batch(1, versions=64, feat=feat, dtype=np.float64, seed=seed)
    X = batch.X.reshape(64, feat)
    Z, _, _ = oracle.standardize(X)
    return Z, batch.masks.astype(np.uint8), batch.log_time.copy()


@pytest.mark.parametrize("seed,feat", [(3, 24), (4, 48), (5, 80)])
def test_deleting_one_pair_equals_the_direct_fit(seed, feat):
    Z, masks, lt = _program(seed, feat)
    K = Z @ Z.T
    checked = 0
    for j in range(6):
        vb, va = oracle.pairs(masks, j)
        n = len(vb)
        y = lt[vb] - lt[va]
        M = K[np.ix_(vb, vb)] + LAM * np.eye(n)
        Mi = np.linalg.inv(M)
        Mi = 0.5 * (Mi + Mi.T)
        wy, w1 = Mi @ y, Mi @ np.ones(n)
        for i in range(n):
            keep = np.arange(n) != i
            st, beta, b_ref = oracle.ridge_fit(Z[vb[keep]], y[keep], LAM)
            assert st == oracle.FIT_OK
            ui = Mi[i, i]
            # intercept from the downdated sums
            b = (wy.sum() - w1[i] * wy[i] / ui) / (w1.sum() - w1[i] ** 2 / ui)
            assert abs(b - b_ref) <= 1e-9 * abs(b_ref) + 1e-11
            # the held-out before version: the leave-one-out residual
            e = (wy[i] - b * w1[i]) / ui
            pred_ref = b_ref + Z[vb[i]] @ beta
            assert abs((y[i] - e) - pred_ref) <= 1e-9 * abs(pred_ref) + 1e-11
            # the held-out after version: the sum over the reduced fit's pairs
            alpha = (wy - b * w1) - Mi[i] * e
            assert abs(alpha[i]) <= 1e-9 * np.abs(alpha).max()
            pred_a = b + K[va[i], vb[keep]] @ alpha[keep]
            pred_a_ref = b_ref + Z[va[i]] @ beta
            assert abs(pred_a - pred_a_ref) <= 1e-9 * abs(pred_a_ref) + 1e-11
            checked += 1
    assert checked >= 6 * 32


def test_the_label_at_the_deleted_position_does_not_matter():
    # a non-finite label enters the inverse's right-hand side as 0: the fits that leave its
    # pair out are the same as with any other value there
    Z, masks, lt = _program(7, 32)
    K = Z @ Z.T
    vb, va = oracle.pairs(masks, 2)
    n = len(vb)
    y = lt[vb] - lt[va]
    M = K[np.ix_(vb, vb)] + LAM * np.eye(n)
    Mi = np.linalg.inv(M)
    Mi = 0.5 * (Mi + Mi.T)
    i = 5
    out = []
    for yi in (y[i], 0.0, 1e3, -7.5):
        yt = y.copy()
        yt[i] = yi
        wy, w1 = Mi @ yt, Mi @ np.ones(n)
        ui = Mi[i, i]
        b = (wy.sum() - w1[i] * wy[i] / ui) / (w1.sum() - w1[i] ** 2 / ui)
        e = (wy[i] - b * w1[i]) / ui
        out.append((b, yi - e))
    ref_b, ref_p = out[0]
    for b, p in out[1:]:
        assert abs(b - ref_b) <= 1e-10 * abs(ref_b) + 1e-12
        assert abs(p - ref_p) <= 1e-10 * abs(ref_p) + 1e-12
