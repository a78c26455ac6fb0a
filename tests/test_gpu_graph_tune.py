"""One CUDA-graph launch per step on an uneven batch, and the autotuner, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_1910_07776_gb300 import synth
from parity import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1910_07776_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    yield rs, ctx
    ctx.close()


def _uneven(rs):
    batch = synth.make_batch_fast(40, versions=(8, 64), feat_choices=[64, 128, 256, 512], seed=95)
    splits = synth.make_half_splits_fast(batch, 64, seed=95)
    return batch, splits, rs.DeviceBatch.from_host(batch), rs.DeviceSplits.from_host(splits, batch=batch)


def _outs(rs, ds):
    return rs.alloc_outputs(ds.n_test_rows, ds.n_splits, 3)


def test_graph_launch_equals_eager_step(env):
    rs, ctx = env
    batch, splits, db, ds = _uneven(rs)
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    a, b = _outs(rs, ds), _outs(rs, ds)
    ctx.cv_step(db, ds, ws, a.rec_offsets, a.rec_code, rec_pred=a.rec_pred, pred_all=a.pred_all, counters=a.counters)
    g = ctx.cv_graph(db, ds, ws, b.rec_offsets, b.rec_code, rec_pred=b.rec_pred, pred_all=b.pred_all,
                     counters=b.counters)     # creation runs one eager pass
    b.rec_code.fill_(-1)
    b.pred_all.fill_(7.0)
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    ctx.check_device_status()
    assert torch.equal(a.rec_code, b.rec_code)
    assert torch.equal(torch.nan_to_num(a.pred_all, nan=-9.0), torch.nan_to_num(b.pred_all, nan=-9.0))
    assert torch.equal(3 * a.counters, b.counters)      # eager pass + two launches
    g.close()


def test_autotune_keeps_the_results(env):
    rs, ctx = env
    batch, splits, db, ds = _uneven(rs)
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    a, b = _outs(rs, ds), _outs(rs, ds)
    ctx.cv_step(db, ds, ws, a.rec_offsets, a.rec_code, rec_pred=a.rec_pred, pred_all=a.pred_all)
    t = ctx.autotune(db, ds, ws, b.rec_offsets, b.rec_code, rec_pred=b.rec_pred)
    assert len(t["times_ms"]) == 30 and t["solve_split"] in (4, 5, 6, 7, 8) and t["rank_waves"] in (8, 16, 32)
    assert t["solve_order"] in (0, 1)
    ctx.cv_step(db, ds, ws, b.rec_offsets, b.rec_code, rec_pred=b.rec_pred, pred_all=b.pred_all)
    torch.cuda.synchronize()
    close(b.pred_all.cpu().numpy(), a.pred_all.cpu().numpy(), rel=1e-12, abs_=1e-14)
    assert torch.equal(a.rec_code, b.rec_code)


def test_work_order_and_tuning_setter_change_no_result(env):
    # the launch parameters only redistribute work: every configuration gives the same bits
    rs, ctx = env
    batch, splits, db, ds = _uneven(rs)
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    ref = None
    for cfg in ((6, 32, 0), (6, 32, 1), (4, 8, 1), (8, 16, 0)):
        ctx.set_tuning(*cfg)
        assert tuple(ctx.get_tuning().values()) == cfg
        o = _outs(rs, ds)
        ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, rec_pred=o.rec_pred, pred_all=o.pred_all)
        torch.cuda.synchronize()
        got = (o.pred_all.cpu().numpy(), o.rec_code.cpu().numpy())
        if ref is None:
            ref = got
        else:
            np.testing.assert_array_equal(got[0], ref[0])
            np.testing.assert_array_equal(got[1], ref[1])
    for bad in ((3, 32, 0), (6, 12, 0), (6, 32, 2)):
        with pytest.raises(rs.RsError):
            ctx.set_tuning(*bad)
    ctx.set_tuning(6, 32, 1)


def test_gram_tile_shapes_agree_and_the_autotuner_keeps_one(env):
    # every tile shape of the tensor-core Gram (32- or 64-column tiles, K whole or split into
    # its three BF16 products) gives the FP64 Gram within the BF16 x 3 bound, on a batch of mixed
    # widths and version counts; the autotuner keeps one of them for the batch's width
    rs, ctx = env
    batch, splits, db, ds = _uneven(rs)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    K64 = ctx.gram(zb, rs.RS_GRAM_F64).cpu().numpy().reshape(-1, 64, 64)
    Zh = Z.cpu().numpy()
    for tile_n in (64, 32):
        for ksplit in (1, 3):
            ctx.set_gram_tuning(db.max_feat, tile_n, ksplit)
            assert ctx.get_gram_tuning(db.max_feat) == {"tile_n": tile_n, "ksplit": ksplit}
            K = ctx.gram(zb, rs.RS_GRAM_BF16X3).cpu().numpy().reshape(-1, 64, 64)
            for p in range(batch.n_programs):
                V, F = batch.versions(p), int(batch.feat_width[p])
                o = int(batch.x_offsets[p])
                Zp = np.abs(Zh[o:o + V * F].reshape(V, F))
                err = np.abs(K[p, :V, :V] - K64[p, :V, :V]) / (Zp @ Zp.T + 1e-300)
                assert err.max() < 6e-5, (tile_n, ksplit, p, err.max())
                np.testing.assert_array_equal(K[p, :V, :V], K[p, :V, :V].T)
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    got = ctx.autotune_gram(db, ws)
    assert (got["tile_n"], got["ksplit"]) in {(64, 1), (32, 1), (64, 3), (32, 3)}
    assert all(t > 0 for t in got["times_ms"].values())
    assert ctx.get_gram_tuning(db.max_feat) == {"tile_n": got["tile_n"], "ksplit": got["ksplit"]}
    ctx.set_gram_tuning(db.max_feat, 64, 1)
