"""GPU parity of the closed-form leave-one-version-out fits (RS_LOO_CLOSED): one inverse of
each program's full system per optimization, every fit from it by deleting the held-out
version's pair, against the FP64 reference's direct solve of every fit (Sec. 5's protocol:
each split holds out one version).  Predictions within the FP64 parity bound, rankings and
counters equal outside near-decisions, statuses equal (a non-finite label fails exactly the
fits that train on its pair); the one-call step gives the individual calls' outputs bit for
bit; splits that hold out more than one pair's worth are refused with RS_EDATA."""
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


def _case(name):
    if name == "tiny":              # 2 programs x 64 versions (all masks) x 96 FP64 features
        b = synth.make_batch(2, versions=64, feat=96, dtype=np.float64, seed=0)
        return b, synth.make_splits(b, "lovo")
    if name == "ragged":            # 1..64 versions, feature widths 8, 33, 64, FP32 counters
        b = synth.make_batch(9, versions=(1, 64), feat_choices=[8, 33, 64], dtype=np.float32, seed=34)
        return b, synth.make_splits(b, "lovo")
    if name == "wide":              # 512 FP64 features
        b = synth.make_batch(3, versions=64, feat=512, dtype=np.float64, seed=67)
        return b, synth.make_splits(b, "lovo")
    if name == "degenerate":        # train on nothing, on everything, all but the first / last
        b = synth.make_batch(3, versions=(30, 64), feat=16, seed=41)
        tm = []
        for p in range(3):
            V = b.versions(p)
            full = (1 << V) - 1 if V < 64 else (1 << 64) - 1
            tm += [0, full, full & ~1, full & ~(1 << (V - 1))]
        return b, synth.Splits(split_offsets=np.arange(4, dtype=np.int64) * 4,
                               train_masks=np.array(tm, dtype=np.uint64))
    if name == "inf_label":         # an infinite log time in programs 1 and 4
        b = synth.make_batch(6, versions=(24, 64), feat=24, dtype=np.float64, seed=77)
        lt = b.log_time.copy()
        for p in (1, 4):
            lt[int(b.row_offsets[p]) + 3] = np.inf
        b.log_time = lt
        return b, synth.make_splits(b, "lovo")
    raise ValueError(name)


@pytest.mark.parametrize("name", ["tiny", "ragged", "wide", "degenerate", "inf_label"])
def test_closed_form_matches_the_reference(rs, ctx, name):
    batch, splits = _case(name)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    g = rs.cv_run(ctx, db, ds, flags=rs.RS_LOO_CLOSED)
    ctx.check_device_status()
    r = oracle.cv_batch(batch, splits)
    np.testing.assert_array_equal(g["rec_offsets"], r.rec_offsets)
    close(g["pred_all"], r.pred_all)
    _, nnear = compare_rankings(g["rec_code"], r.rec_code, r.pred_all, math.log(1.05))
    same = g["rec_code"] == r.rec_code
    close(g["rec_pred"][same], r.rec_pred[same])
    compare_counters(g["counters"], r.counters, slack=nnear)
    if name == "inf_label":
        assert r.counter("fit_nonfinite") > 0


def test_one_call_step_equals_the_individual_calls(rs, ctx):
    batch, splits = _case("ragged")
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    g = rs.cv_run(ctx, db, ds, flags=rs.RS_LOO_CLOSED)
    R = ds.n_test_rows
    out = rs.alloc_outputs(R, ds.n_splits, 3, "cuda")
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    ctx.cv_step(db, ds, ws, out.rec_offsets, out.rec_code, flags=rs.RS_LOO_CLOSED, rec_pred=out.rec_pred,
                pred_all=out.pred_all, counters=out.counters)
    torch.cuda.synchronize()
    ctx.check_device_status()
    np.testing.assert_array_equal(out.rec_code.cpu().numpy().view(np.uint32), g["rec_code"])
    np.testing.assert_array_equal(out.rec_pred.cpu().numpy().reshape(g["rec_pred"].shape), g["rec_pred"])
    np.testing.assert_array_equal(out.pred_all.cpu().numpy().reshape(g["pred_all"].shape), g["pred_all"])


def test_splits_without_the_closed_form_are_refused(rs, ctx):
    # half splits leave out many pairs per fit: RS_EDATA, and those fits count as failed
    batch = synth.make_batch(3, versions=64, feat=16, seed=71)
    splits = synth.make_splits(batch, "half", 9, seed=71)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    R = ds.n_test_rows
    out = rs.alloc_outputs(R, ds.n_splits, 3, "cuda")
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    ctx.cv_step(db, ds, ws, out.rec_offsets, out.rec_code, flags=rs.RS_LOO_CLOSED, counters=out.counters)
    torch.cuda.synchronize()
    with pytest.raises(rs.RsError) as e:
        ctx.check_device_status()
    assert e.value.status == rs.RS_EDATA
    cnt = out.counters.cpu().numpy()
    assert cnt[11] > 0 and cnt[9] + cnt[10] + cnt[11] + cnt[12] == 6 * ds.n_splits


def test_closed_form_argument_errors(rs, ctx):
    batch = synth.make_batch(1, versions=8, feat=8, seed=62)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(synth.make_splits(batch, "lovo"))
    zb = db.with_X(ctx.standardize(db))
    K = ctx.gram(zb)
    ro = ctx.rec_offsets(zb, ds)
    code = torch.empty(int(ro[-1]), dtype=torch.int32, device="cuda")
    for kw in (dict(form=1), dict(flags=rs.RS_LOO_CLOSED | rs.RS_REFINE_X),
               dict(flags=rs.RS_LOO_CLOSED | rs.RS_MODEL_IBK)):
        kw.setdefault("flags", rs.RS_LOO_CLOSED)
        with pytest.raises(rs.RsError) as e:
            ctx.predict_rank(zb, K, ds, ro, code, **kw)
        assert e.value.status == rs.RS_EINVAL


def test_leave_one_out_at_the_precision_form_shape_sampled(rs, ctx):
    # 256 programs x 64 versions (all masks) x 1024 FP64 features, every leave-one-version-out
    # split (16,384 splits, 98,304 fits of 31 pairs) through rs_cv_step with the closed form,
    # as the benchmark times it; 4 splits of each of 12 sampled programs recomputed by the
    # reference row by row
    batch = synth.make_batch_fast(256, versions=64, feat=1024, dtype=np.float64, seed=43)
    splits = synth.make_splits(batch, "lovo")
    db, ds = rs.DeviceBatch.from_host(batch), rs.DeviceSplits.from_host(splits, batch=batch)
    R = ds.n_test_rows
    out = rs.alloc_outputs(R, ds.n_splits, 3, "cuda")
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    ctx.cv_step(db, ds, ws, out.rec_offsets, out.rec_code, flags=rs.RS_LOO_CLOSED, rec_pred=out.rec_pred,
                pred_all=out.pred_all, counters=out.counters)
    torch.cuda.synchronize()
    ctx.check_device_status()
    gro = out.rec_offsets.cpu().numpy()
    cnt = out.counters.cpu().numpy()
    assert cnt[9] == 6 * ds.n_splits                 # every fit solved
    rng = np.random.default_rng(43)
    progs = np.sort(rng.choice(batch.n_programs, size=12, replace=False))
    pick = np.concatenate([int(splits.split_offsets[p]) + np.sort(rng.choice(64, size=4, replace=False))
                           for p in progs])
    sub_batch = synth.take_programs(batch, progs)
    sub = synth.Splits(split_offsets=np.arange(13, dtype=np.int64) * 4, train_masks=splits.train_masks[pick])
    r = oracle.cv_batch(sub_batch, sub)
    rows = np.concatenate([np.arange(gro[i], gro[i + 1]) for i in pick])
    pa = out.pred_all.cpu().numpy().reshape(R, 6)[rows]
    code = out.rec_code.cpu().numpy().view(np.uint32)[rows]
    close(pa, r.pred_all)
    compare_rankings(code, r.rec_code, r.pred_all, math.log(1.05))


@pytest.mark.parametrize("name", ["ragged", "inf_label"])
def test_closed_form_coefficients_equal_the_direct_fits(rs, ctx, name):
    # rs_fit_batched with RS_LOO_CLOSED: b and alpha (ascending pair order) and the statuses
    # of every fit against the direct solves of the same call without the flag
    batch, splits = _case(name)
    db, ds = rs.DeviceBatch.from_host(batch), rs.DeviceSplits.from_host(splits, batch=batch)
    zb = db.with_X(ctx.standardize(db))
    K = ctx.gram(zb)
    S = ds.n_splits
    res = []
    for form in (rs.RS_FORM_BATCHED, rs.RS_FORM_BATCHED | rs.RS_LOO_CLOSED):
        coef = torch.full((S * 6 * 33,), 7.0, dtype=torch.float64, device="cuda")
        st = torch.full((S * 6,), 9, dtype=torch.uint8, device="cuda")
        ctx.fit_batched(zb, K, ds, 1e-3, form, coef, st)
        torch.cuda.synchronize()
        ctx.check_device_status()
        res.append((coef.cpu().numpy().reshape(S * 6, 33), st.cpu().numpy()))
    (cd, sd), (cc, sc) = res
    np.testing.assert_array_equal(sc, sd)
    ok = sd == 0
    assert ok.any()
    # normwise per fit: two backward-stable solutions of one system differ by O(cond * u) of
    # the solution's norm (cond(M) stays below 1e5 on these inputs)
    scale = np.abs(cd[ok]).max(axis=1, keepdims=True)
    assert np.all(np.abs(cc[ok] - cd[ok]) <= 1e-9 * scale + 1e-11)
    np.testing.assert_array_equal(np.isnan(cc[~ok, 0]), np.isnan(cd[~ok, 0]))


def test_rank_all_predicts_the_after_versions_too(rs, ctx):
    # RS_RANK_ALL: the held-out version is also the after side of its pair for the
    # optimizations it has; those predictions take the sum over the fit's pairs
    batch, splits = _case("tiny")
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    g = rs.cv_run(ctx, db, ds, flags=rs.RS_LOO_CLOSED | rs.RS_RANK_ALL)
    r = oracle.cv_batch(batch, splits, flags=oracle.RANK_ALL)
    close(g["pred_all"], r.pred_all)
    _, nnear = compare_rankings(g["rec_code"], r.rec_code, r.pred_all, math.log(1.05))
    compare_counters(g["counters"], r.counters, slack=nnear)


def test_graph_of_the_closed_form_step_equals_the_call(rs, ctx):
    # rs_cv_graph_create captures the step with RS_LOO_CLOSED; two launches give the one-call
    # step's outputs bit for bit (the counters accumulate over launches)
    batch, splits = _case("tiny")
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    R = ds.n_test_rows
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    a = rs.alloc_outputs(R, ds.n_splits, 3, "cuda")
    ctx.cv_step(db, ds, ws, a.rec_offsets, a.rec_code, flags=rs.RS_LOO_CLOSED, rec_pred=a.rec_pred,
                pred_all=a.pred_all, counters=a.counters)
    b = rs.alloc_outputs(R, ds.n_splits, 3, "cuda")
    g = ctx.cv_graph(db, ds, ws, b.rec_offsets, b.rec_code, flags=rs.RS_LOO_CLOSED, rec_pred=b.rec_pred,
                     pred_all=b.pred_all, counters=b.counters)
    b.counters.zero_()
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    g.close()
    ctx.check_device_status()
    assert torch.equal(a.rec_code, b.rec_code)
    np.testing.assert_array_equal(a.pred_all.cpu().numpy(), b.pred_all.cpu().numpy())
    np.testing.assert_array_equal(a.rec_pred.cpu().numpy(), b.rec_pred.cpu().numpy())
    assert torch.equal(2 * a.counters, b.counters)


def test_closed_form_on_the_tensor_core_gram(rs, ctx):
    # the precision form's BF16 hi/lo tensor-core Gram with the fits in closed form: the same
    # system as the direct solves on that Gram, so the two agree to FP64 rounding
    batch = synth.make_batch(4, versions=64, feat=256, dtype=np.float64, seed=82, mixing_kappa=1e4)
    splits = synth.make_splits(batch, "lovo")
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    d = rs.cv_run(ctx, db, ds, precision=rs.RS_GRAM_BF16X3)
    c = rs.cv_run(ctx, db, ds, precision=rs.RS_GRAM_BF16X3, flags=rs.RS_LOO_CLOSED)
    close(c["pred_all"], d["pred_all"])
    _, nnear = compare_rankings(c["rec_code"], d["rec_code"], d["pred_all"], math.log(1.05))
    compare_counters(c["counters"], d["counters"], slack=nnear)
