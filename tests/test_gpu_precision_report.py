"""Error of the precision form against the FP64 reference at the precision workload's shape
(64 versions x 1024 FP64 features, leave-one-version-out), for condition numbers 1e2 .. 1e8 of
the random counter mixing: every coefficient (the dual alpha and b of each fit, and the primal
beta = sum_a alpha_a z_a that the dual form implies), every prediction (elementwise relative
error) and the rankings.  Three GPU forms are measured: the FP64 Gram, the BF16 hi/lo-split
tensor-core Gram, and that Gram followed by one refinement step through Z.  The reference solves
each fit's primal normal equations (Sec. 3.4 ridge) by Cholesky; its dual coefficients follow
from the stationarity of the intercepted ridge problem, lambda alpha = y - b - Z beta.

The stated tolerance of the refined form, 2e-5 relative (+1e-6 absolute) on predictions and on
beta, is asserted for kappa <= 1e4; at larger kappa one refinement step stops converging once
kappa * 2^-16 approaches 1, and the errors are recorded, not bounded.  With RS_REPORT_DIR set,
the table is written there as precision_report.json."""
import json
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_1910_07776_gb300 import synth

pytestmark = pytest.mark.gpu

F = 1024
N_SPLITS = 24          # leave-one-out splits of the sampled program (versions 0..23 left out)
LAM = 1e-3


@pytest.fixture(scope="module")
def env():
    from paper_1910_07776_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    yield rs, ctx
    ctx.close()


@pytest.fixture(scope="module")
def report():
    rep = {}
    yield rep
    d = os.environ.get("RS_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "precision_report.json"), "w") as f:
            json.dump(rep, f, indent=1)


def _fit_pairs(masks, T, j):
    slot = {int(x): i for i, x in enumerate(masks)}
    return [(v, slot[masks[v] | 1 << j]) for v in range(len(masks))
            if not (masks[v] >> j) & 1 and (masks[v] | 1 << j) in slot
            and (T >> v) & 1 and (T >> slot[masks[v] | 1 << j]) & 1]


def _rel(d, ref):
    d, ref = np.abs(np.ravel(d)), np.abs(np.ravel(ref))
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.where(ref > 0, d / ref, np.where(d > 0, np.inf, 0.0))
    return {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)), "max": float(e.max()),
            "normwise_max": float(d.max() / max(ref.max(), 1e-300))}


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6, 1e8])
def test_precision_form_error_against_the_reference(env, report, kappa):
    rs, ctx = env
    base = synth.make_batch(1, versions=64, feat=F, dtype=np.float64, seed=93)
    batch = synth.apply_mixing(base, kappa, seed=93)
    full = (1 << 64) - 1
    tm = np.array([full & ~(1 << t) for t in range(N_SPLITS)], dtype=np.uint64)
    splits = synth.Splits(split_offsets=np.array([0, N_SPLITS], dtype=np.int64), train_masks=tm)
    r = oracle.cv_batch(batch, splits, lam=LAM, nthreads=oracle.threads_available())
    m = batch.masks.astype(int)
    lt = batch.log_time
    Zr = r.Z.reshape(64, F)
    # the reference's coefficients of every fit, from its primal solve
    fits = [(s, j, _fit_pairs(m, int(tm[s]), j)) for s in range(N_SPLITS) for j in range(6)]

    def ref_fit(fit):
        s, j, pairs = fit
        Zt = Zr[[v for v, _ in pairs]]
        y = np.array([lt[v] - lt[w] for v, w in pairs])
        st, beta, b = oracle.ridge_fit(Zt, y, LAM)
        assert st == oracle.FIT_OK
        return beta, b, (y - b - Zt @ beta) / LAM

    with ThreadPoolExecutor(max(1, oracle.threads_available())) as ex:
        ref = list(ex.map(ref_fit, fits))

    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    Zg = Z.cpu().numpy().reshape(64, F)
    out = {"achieved_cond_first_fit": None}
    s0, j0, p0 = fits[0]
    Kt = Zr[[v for v, _ in p0]] @ Zr[[v for v, _ in p0]].T + LAM * np.eye(len(p0))
    out["achieved_cond_first_fit"] = float(np.linalg.cond(Kt))
    for name, prec, flags in (("f64", rs.RS_GRAM_F64, 0), ("bf16x3", rs.RS_GRAM_BF16X3, 0),
                              ("bf16x3_refined", rs.RS_GRAM_BF16X3, rs.RS_REFINE_X)):
        K = ctx.gram(zb, prec)
        coef = torch.full((N_SPLITS * 6 * 33,), 7.0, dtype=torch.float64, device="cuda")
        ctx.fit_batched(zb, K, ds, LAM, rs.RS_FORM_BATCHED | flags, coef)
        g = rs.cv_run(ctx, db, ds, lam=LAM, precision=prec, flags=flags)
        cf = coef.cpu().numpy().reshape(N_SPLITS, 6, 33)
        dbeta, rbeta, dal, ral, db_, rb_ = [], [], [], [], [], []
        for (s, j, pairs), (beta, b, alpha) in zip(fits, ref):
            n = len(pairs)
            al = cf[s, j, 1:1 + n]
            bg = al @ Zg[[v for v, _ in pairs]]
            dbeta.append(bg - beta)
            rbeta.append(beta)
            dal.append(al - alpha)
            ral.append(alpha)
            db_.append(cf[s, j, 0] - b)
            rb_.append(b)
        ok = ~np.isnan(r.pred_all)
        dp = g["pred_all"][ok] - r.pred_all[ok]
        ent = {"beta": _rel(np.concatenate(dbeta), np.concatenate(rbeta)),
               "alpha": _rel(np.concatenate(dal), np.concatenate(ral)),
               "b": _rel(np.array(db_), np.array(rb_)),
               "pred": _rel(dp, r.pred_all[ok]),
               "pred_max_abs": float(np.abs(dp).max()),
               "ranking_rows_changed": int(np.sum(g["rec_code"] != r.rec_code)),
               "rows": int(r.rec_code.size), "predictions": int(ok.sum())}
        out[name] = ent
        if name == "f64":
            # the FP64 path is the parity path: 1e-9 relative on predictions while kappa <= 1e6
            if kappa <= 1e6:
                assert np.all(np.abs(dp) <= 1e-9 * np.abs(r.pred_all[ok]) + 1e-11)
        if name == "bf16x3_refined" and kappa <= 1e4:
            assert np.all(np.abs(dp) <= 2e-5 * np.abs(r.pred_all[ok]) + 1e-6), ent["pred"]
            assert ent["beta"]["normwise_max"] <= 2e-5, ent["beta"]
    report[f"{kappa:.0e}"] = out
