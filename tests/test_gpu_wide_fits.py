"""GPU parity of the fits of 17..32 pairs (solve_wide_kernel: several lanes per fit, the
factorisation's trailing updates spread over them) against the FP64 reference: splits that
leave out a few versions of all-64-mask programs give every size from 17 to 32 within one
batch, so warps hold fits of different sizes at the bucket boundaries; leave-one-version-out
(31 pairs, Sec. 5) at a wide feature width; and the coefficients of the fits against the
reference's primal solution mapped through the dual identity beta = sum_a alpha_a z_a."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1910_07776_gb300 import synth
from parity import close, compare_counters, compare_rankings

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    from paper_1910_07776_gb300 import build
    build.build()
    from paper_1910_07776_gb300 import rs as _rs
    return _rs


@pytest.fixture(scope="module")
def ctx(rs):
    c = rs.Context(0)
    yield c
    c.close()


def _drop_few_splits(batch, per_program, seed):
    """Train masks that keep each version with a probability drawn per split from [0.75, 1]
    (at least 40 kept): the pair counts of the fits spread over 12..32."""
    rng = np.random.default_rng(seed)
    offs, tm = [0], []
    for p in range(batch.n_programs):
        V = batch.versions(p)
        for s in range(per_program):
            keep = rng.random(V) < (1.0 if s == 0 else rng.uniform(0.75, 1.0))
            if keep.sum() < 40:
                keep[:40] = True
            tm.append(sum(1 << int(v) for v in np.nonzero(keep)[0]))
        offs.append(len(tm))
    return synth.Splits(split_offsets=np.array(offs, dtype=np.int64), train_masks=np.array(tm, dtype=np.uint64))


def _check(rs, ctx, batch, splits):
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    g = rs.cv_run(ctx, db, ds, want_Z=True)
    r = oracle.cv_batch(batch, splits)
    np.testing.assert_array_equal(g["rec_offsets"], r.rec_offsets)
    close(g["pred_all"], r.pred_all)
    _, nnear = compare_rankings(g["rec_code"], r.rec_code, r.pred_all, math.log(1.05))
    compare_counters(g["counters"], r.counters, slack=nnear)
    return r


@pytest.mark.parametrize("feat,dtype", [(40, np.float64), (96, np.float32)])
def test_fits_of_17_to_32_pairs_match_the_reference(rs, ctx, feat, dtype):
    batch = synth.make_batch(6, versions=64, feat=feat, dtype=dtype, seed=61 + feat)
    splits = _drop_few_splits(batch, 30, seed=feat)
    r = _check(rs, ctx, batch, splits)
    assert r.counter("fit_ok") == splits.n_splits * 6


def test_leave_one_out_at_a_wide_feature_width(rs, ctx):
    batch = synth.make_batch(3, versions=64, feat=512, dtype=np.float64, seed=67)
    splits = synth.make_splits(batch, "lovo")
    _check(rs, ctx, batch, splits)


def test_wide_fit_coefficients_give_the_reference_primal_solution(rs, ctx):
    # dual alpha, b from the GPU; beta = sum_a alpha_a z_{v_a} must equal the reference's
    # primal ridge coefficients of the same fit (push-through identity)
    batch = synth.make_batch(2, versions=64, feat=24, dtype=np.float64, seed=71)
    splits = _drop_few_splits(batch, 8, seed=71)
    db, ds = rs.DeviceBatch.from_host(batch), rs.DeviceSplits.from_host(splits)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    K = ctx.gram(zb)
    S = ds.n_splits
    coef = torch.full((S * 6 * 33,), 7.0, dtype=torch.float64, device="cuda")
    st = torch.full((S * 6,), 9, dtype=torch.uint8, device="cuda")
    ctx.fit_batched(zb, K, ds, 1e-3, 0, coef, st)
    torch.cuda.synchronize()
    cf = coef.cpu().numpy().reshape(S, 6, 33)
    Zh = Z.cpu().numpy()
    checked = 0
    for p in range(batch.n_programs):
        V, F = batch.versions(p), int(batch.feat_width[p])
        Zp = Zh[int(batch.x_offsets[p]):int(batch.x_offsets[p]) + V * F].reshape(V, F)
        m = batch.masks[batch.program_rows(p)].astype(int)
        lt = batch.log_time[batch.program_rows(p)]
        slot = {int(x): i for i, x in enumerate(m)}
        for s in range(int(splits.split_offsets[p]), int(splits.split_offsets[p + 1])):
            T = int(splits.train_masks[s])
            for j in range(6):
                pairs = [(v, slot[m[v] | 1 << j]) for v in range(V) if not (m[v] >> j) & 1
                         and (m[v] | 1 << j) in slot and (T >> v) & 1 and (T >> slot[m[v] | 1 << j]) & 1]
                n = len(pairs)
                if n <= 16:
                    continue
                Zr = np.array([Zp[v] for v, _ in pairs])
                y = np.array([lt[v] - lt[w] for v, w in pairs])
                st, beta_ref, b_ref = oracle.ridge_fit(Zr, y, 1e-3)
                assert st == oracle.FIT_OK
                alpha = cf[s, j, 1:1 + n]
                close(alpha @ Zr, beta_ref, rel=1e-8, abs_=1e-9)
                close(cf[s, j, 0], b_ref, rel=1e-8, abs_=1e-9)
                checked += 1
    assert checked > 50
