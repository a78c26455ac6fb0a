"""GPU parity of the instance-based learner (Sec. 3.4, IBK k = 10): the squared-distance
block and the batched IBK predictions, ranking and counters through the C ABI against the
FP64 CPU reference.  The device forms every distance with the plain definition's arithmetic
and sums the neighbours' labels in the reference's order, so the comparison is exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_1910_07776_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1910_07776_gb300 import build
    build.build()
    from paper_1910_07776_gb300 import rs as _rs
    return _rs


@pytest.fixture(scope="module")
def ctx(rs):
    c = rs.Context(0)
    yield c
    c.close()


def _ibk_both(rs, ctx, batch, splits, k=3, tau=1.05):
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    g = rs.cv_run(ctx, db, ds, k=k, tau=tau, flags=rs.RS_MODEL_IBK, want_Z=True)
    r = oracle.cv_batch(batch, splits, k=k, tau=tau, model="ibk")
    return g, r


def _assert_same(g, r):
    np.testing.assert_array_equal(g["rec_offsets"], r.rec_offsets)
    np.testing.assert_array_equal(g["pred_all"], r.pred_all)
    np.testing.assert_array_equal(g["rec_code"], r.rec_code)
    np.testing.assert_array_equal(g["rec_pred"], r.rec_pred)
    np.testing.assert_array_equal(g["counters"], r.counters)


def test_distance_block_is_the_plain_definition(rs, ctx):
    batch = synth.make_batch(6, versions=(1, 64), feat_choices=[1, 33, 96, 200], dtype=np.float64, seed=61)
    db = rs.DeviceBatch.from_host(batch)
    Z = ctx.standardize(db)
    D = ctx.gram(db.with_X(Z), rs.RS_GRAM_DIST2).cpu().numpy().reshape(-1, 64, 64)
    Zh = Z.cpu().numpy()
    for p in range(batch.n_programs):
        V, F = batch.versions(p), int(batch.feat_width[p])
        o = int(batch.x_offsets[p])
        Zp = Zh[o:o + V * F].reshape(V, F)
        e = Zp[:, None, :] - Zp[None, :, :]
        ref = np.cumsum(e * e, axis=2)[:, :, -1]          # ascending f, one rounding per step
        np.testing.assert_array_equal(D[p, :V, :V], ref)


def test_ibk_lovo_all_masks_exact(rs, ctx):
    # 31 training pairs per fit: the 10-nearest selection decides every prediction
    batch = synth.make_batch(2, versions=64, feat=96, dtype=np.float64, seed=0)
    splits = synth.make_splits(batch, "lovo")
    g, r = _ibk_both(rs, ctx, batch, splits)
    _assert_same(g, r)
    assert r.counter("fit_ok") == 128 * 6


def test_ibk_ragged_half_splits_exact(rs, ctx):
    batch = synth.make_batch(9, versions=(1, 64), feat_choices=[8, 40, 130], dtype=np.float32,
                             seed=62, with_cycles=True)
    splits = synth.make_splits(batch, "half", 40, seed=62)
    g, r = _ibk_both(rs, ctx, batch, splits, k=2, tau=1.01)
    _assert_same(g, r)


def test_ibk_ties_from_repeated_feature_rows(rs, ctx):
    # versions with identical counters: equal distances, broken by the lower pair
    batch = synth.make_batch(3, versions=64, feat=20, dtype=np.float64, seed=63)
    X = batch.X.copy()
    for p in range(batch.n_programs):
        o, F = int(batch.x_offsets[p]), int(batch.feat_width[p])
        Xp = X[o:o + 64 * F].reshape(64, F)
        Xp[1::4] = Xp[0::4]
    batch.X = X
    splits = synth.make_splits(batch, "lovo")
    g, r = _ibk_both(rs, ctx, batch, splits, k=6, tau=0.5)
    _assert_same(g, r)


def test_ibk_one_call_step_equals_the_entry_points(rs, ctx):
    batch = synth.make_batch(5, versions=(20, 64), feat=64, dtype=np.float32, seed=64)
    splits = synth.make_splits(batch, "half", 64, seed=64)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    g = rs.cv_run(ctx, db, ds, flags=rs.RS_MODEL_IBK)
    R = int(g["rec_offsets"][-1])
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    ro = torch.empty(ds.n_splits + 1, dtype=torch.int64, device="cuda")
    out = rs.alloc_outputs(R, ds.n_splits, 3, "cuda")
    ctx.cv_step(db, ds, ws, ro, out.rec_code, flags=rs.RS_MODEL_IBK, rec_pred=out.rec_pred,
                counters=out.counters)
    torch.cuda.synchronize()
    ctx.check_device_status()
    np.testing.assert_array_equal(ro.cpu().numpy(), g["rec_offsets"])
    np.testing.assert_array_equal(out.rec_code.cpu().numpy().view(np.uint32), g["rec_code"])
    np.testing.assert_array_equal(out.counters.cpu().numpy().view(np.uint64), g["counters"])


def test_ibk_argument_errors(rs, ctx):
    batch = synth.make_batch(2, versions=16, feat=8, seed=65)
    splits = synth.make_splits(batch, "half", 4, seed=65)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    D = ctx.gram(zb, rs.RS_GRAM_DIST2)
    ro = ctx.rec_offsets(zb, ds)
    out = rs.alloc_outputs(int(ro[-1].item()), ds.n_splits, 3, "cuda")
    for kw in (dict(form=rs.RS_FORM_PLAIN), dict(flags=rs.RS_MODEL_IBK | rs.RS_REFINE_X)):
        flags = kw.pop("flags", rs.RS_MODEL_IBK)
        with pytest.raises(rs.RsError):
            ctx.predict_rank(zb, D, ds, ro, out.rec_code, flags=flags, **kw)
