"""Pooled ridge fits in primal form (rs_fit_pooled: the Gram X^T W X of every optimization's
pairs over many programs as one tcgen05 GEMM of the BF16 hi/lo split, FP64 Cholesky, one FP64
refinement step) against the FP64 reference: the oracle's primal ridge on the same pooled pairs
(Sec. 3.3 pairs of each program, Sec. 3.4 ridge with an unpenalised intercept), and the
predictions, rankings and scores of held-out programs (Sec. 2 tier 3, Sec. 5)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1910_07776_gb300 import synth
from parity import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1910_07776_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    yield rs, ctx
    ctx.close()


def _pooled_reference(batch, Z, train, lam):
    """The oracle's primal fit on the pairs of the training programs, in program order and
    ascending before slot; returns per optimization (status, b, beta, n, kappa of G)."""
    out = []
    for j in range(6):
        zs, ys = [], []
        for p in train:
            V, F = batch.versions(p), int(batch.feat_width[p])
            Zp = Z[int(batch.x_offsets[p]):int(batch.x_offsets[p]) + V * F].reshape(V, F)
            m = batch.masks[batch.program_rows(p)].astype(int)
            lt = batch.log_time[batch.program_rows(p)]
            slot = {int(x): i for i, x in enumerate(m)}
            for v in range(V):
                if not (m[v] >> j) & 1 and (m[v] | 1 << j) in slot:
                    zs.append(Zp[v])
                    ys.append(lt[v] - lt[slot[m[v] | 1 << j]])
        st, beta, b = oracle.ridge_fit(np.array(zs), np.array(ys), lam)
        Zc = np.array(zs) - np.mean(zs, axis=0)
        kappa = np.linalg.cond(Zc.T @ Zc + lam * np.eye(Zc.shape[1]))
        out.append((st, b, beta, len(ys), kappa))
    return out


@pytest.mark.parametrize("feat", [64, 96, 128])
def test_pooled_fit_matches_the_reference(env, feat):
    rs, ctx = env
    batch = synth.make_batch(24, versions=(40, 64), feat=feat, dtype=np.float64, seed=100 + feat)
    r = oracle.cv_batch(batch, synth.make_splits(batch, "all"))
    use = np.zeros(batch.n_programs, dtype=np.uint8)
    use[:16] = 1
    ref = _pooled_reference(batch, r.Z, range(16), 1e-3)
    db = rs.DeviceBatch.from_host(batch)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    out = {}
    for name, flags in (("raw", 0), ("refined", rs.RS_REFINE_X)):
        coef, st = ctx.fit_pooled(zb, torch.from_numpy(use).cuda(), lam=1e-3, flags=flags)
        torch.cuda.synchronize()
        ctx.check_device_status()
        out[name] = (coef.cpu().numpy(), st.cpu().numpy())
    # the BF16 x 3 Gram carries G to delta ~ 2^-17 (hi + lo keeps 17 bits of every value) plus
    # its FP32 accumulation; a solve with it is off by at most about kappa delta, and one
    # refinement step with the exact FP64 residual multiplies that error by at most about
    # kappa delta again (above the FP64 solves' own kappa eps)
    delta = 2.0 ** -17
    eps = np.finfo(float).eps
    for j, (s_ref, b_ref, beta_ref, n, kappa) in enumerate(ref):
        assert s_ref == oracle.FIT_OK and n > feat
        scale = np.abs(beta_ref).max()
        err = {}
        for name, (coef, st) in out.items():
            assert st[j] == oracle.FIT_OK
            err[name] = np.abs(coef[j, 1:] - beta_ref).max() / scale
        assert err["raw"] <= 10 * kappa * delta, (j, err, kappa)
        assert err["refined"] <= 10 * kappa * delta * err["raw"] + 100 * kappa * eps, (j, err, kappa)
        assert err["refined"] <= 1e-6
        b_err = abs(out["refined"][0][j, 0] - b_ref) / (abs(b_ref) + scale)
        assert b_err <= 10 * kappa * delta * err["raw"] + 100 * kappa * eps, (j, b_err)


def test_pooled_predictions_rank_held_out_programs_like_the_reference(env):
    rs, ctx = env
    batch = synth.make_batch(20, versions=(30, 64), feat=64, dtype=np.float64, seed=111)
    r = oracle.cv_batch(batch, synth.make_splits(batch, "all"))
    use = np.zeros(batch.n_programs, dtype=np.uint8)
    use[:12] = 1
    ref = _pooled_reference(batch, r.Z, range(12), 1e-3)
    bound = 1e-6           # the refined pooled fit's bound (test above), on predictions of O(1)
    db = rs.DeviceBatch.from_host(batch)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    coef, st = ctx.fit_pooled(zb, torch.from_numpy(use).cuda(), lam=1e-3, flags=rs.RS_REFINE_X)
    n = batch.n_rows
    code = torch.empty(n, dtype=torch.int32, device="cuda")
    rp = torch.empty(n * 3, dtype=torch.float64, device="cuda")
    pa = torch.empty(n * 6, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(16, dtype=torch.int64, device="cuda")
    ctx.predict_pooled(zb, coef, st, code, rec_pred=rp, pred_all=pa, counters=cnt)
    torch.cuda.synchronize()
    ctx.check_device_status()
    pa = pa.cpu().numpy().reshape(n, 6)
    code = code.cpu().numpy().view(np.uint32)
    log_tau = math.log(1.05)
    checked = 0
    for p in range(batch.n_programs):
        V, F = batch.versions(p), int(batch.feat_width[p])
        Zp = r.Z[int(batch.x_offsets[p]):int(batch.x_offsets[p]) + V * F].reshape(V, F)
        m = batch.masks[batch.program_rows(p)].astype(int)
        for t in range(V):
            row = int(batch.row_offsets[p]) + t
            want = np.full(6, np.nan)
            for j in range(6):
                if not (m[t] >> j) & 1:
                    want[j] = ref[j][1] + Zp[t] @ ref[j][2]
            close(pa[row], want, rel=bound, abs_=bound)
            valid = ~np.isnan(want)
            idx = list(oracle.rank(np.nan_to_num(want), valid.astype(np.int32), 3, log_tau))
            s = np.sort(want[valid])
            tol = max(1e-8, 10 * bound)
            near = (s.size > 1 and np.min(np.diff(s)) < tol) or np.any(np.abs(want[valid] - log_tau) < tol)
            if not near:
                got = [(int(code[row]) >> (4 + 4 * i)) & 0xF for i in range(int(code[row]) & 0xF)]
                assert got == idx, (row, got, idx)
                checked += 1
    assert checked > 500
    assert int(cnt.cpu()[0]) == n
