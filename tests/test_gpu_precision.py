"""Precision form: the BF16 hi/lo-split Gram on the tensor cores, the FP64 factorisation of the
dual systems, and one step of iterative refinement through Z, against the FP64 path and the
FP64 CPU reference."""
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1910_07776_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    yield rs, ctx
    ctx.close()


def test_tensor_core_gram_against_fp64_gram(env):
    rs, ctx = env
    batch = synth.make_batch(7, versions=(1, 64), feat_choices=[40, 96, 300], dtype=np.float64, seed=81)
    db = rs.DeviceBatch.from_host(batch)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    K64 = ctx.gram(zb, rs.RS_GRAM_F64).cpu().numpy().reshape(-1, 64, 64)
    Ktc = ctx.gram(zb, rs.RS_GRAM_BF16X3).cpu().numpy().reshape(-1, 64, 64)
    Zh = Z.cpu().numpy()
    for p in range(batch.n_programs):
        V, F = batch.versions(p), int(batch.feat_width[p])
        o = int(batch.x_offsets[p])
        Zp = np.abs(Zh[o:o + V * F].reshape(V, F))
        scale = Zp @ Zp.T
        err = np.abs(Ktc[p, :V, :V] - K64[p, :V, :V]) / (scale + 1e-300)
        assert err.max() < 6e-5, (p, err.max())
        np.testing.assert_array_equal(Ktc[p, :V, :V], Ktc[p, :V, :V].T)


def _pred(rs, ctx, batch, splits, precision, flags):
    g = rs.cv_run(ctx, rs.DeviceBatch.from_host(batch), rs.DeviceSplits.from_host(splits, batch=batch),
                  precision=precision, flags=flags)
    return g["pred_all"], g


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_refinement_through_z_recovers_fp64_accuracy(env, kappa):
    rs, ctx = env
    batch = synth.make_batch(4, versions=64, feat=256, dtype=np.float64, seed=82, mixing_kappa=kappa)
    splits = synth.make_splits(batch, "lovo")
    ref, _ = _pred(rs, ctx, batch, splits, rs.RS_GRAM_F64, 0)
    raw, _ = _pred(rs, ctx, batch, splits, rs.RS_GRAM_BF16X3, 0)
    ref_d, _ = _pred(rs, ctx, batch, splits, rs.RS_GRAM_F64, rs.RS_REFINE_X)
    fix, _ = _pred(rs, ctx, batch, splits, rs.RS_GRAM_BF16X3, rs.RS_REFINE_X)
    ok = ~np.isnan(ref)
    scale = np.abs(ref[ok]).max()
    e_raw = np.abs(raw[ok] - ref[ok]).max() / scale
    e_fix = np.abs(fix[ok] - ref[ok]).max() / scale
    # refining an exact system changes nothing beyond rounding
    assert np.abs(ref_d[ok] - ref[ok]).max() / scale < 1e-11
    assert e_fix < max(e_raw / 20, 1e-10), (kappa, e_raw, e_fix)


def test_refined_precision_form_against_the_reference(env):
    rs, ctx = env
    batch = synth.make_batch(2, versions=64, feat=128, dtype=np.float64, seed=83, mixing_kappa=1e3)
    splits = synth.make_splits(batch, "lovo")
    fix, g = _pred(rs, ctx, batch, splits, rs.RS_GRAM_BF16X3, rs.RS_REFINE_X)
    r = oracle.cv_batch(batch, splits)
    # one refinement step leaves about (kappa * 2^-16)^2 relative error: the stated tolerance
    # of the precision form is 2e-5 relative (+1e-6 absolute)
    close(fix, r.pred_all, rel=2e-5, abs_=1e-6)
    np.testing.assert_array_equal(g["rec_offsets"], r.rec_offsets)


@pytest.mark.parametrize("precision,flags", [("f64", 0), ("bf16x3", 0), ("bf16x3", "refine"), ("f64", "ibk")])
def test_one_call_step_equals_the_separate_calls(env, precision, flags):
    # rs_cv_step orders its launches itself (the planning beside the Gram on a second stream,
    # or after the tensor-core Gram, whose scratch is the fit workspace): its outputs equal
    # those of the individual entry points, bit for bit
    rs, ctx = env
    prec = {"f64": rs.RS_GRAM_F64, "bf16x3": rs.RS_GRAM_BF16X3}[precision]
    fl = {0: 0, "refine": rs.RS_REFINE_X, "ibk": rs.RS_MODEL_IBK}[flags]
    batch = synth.make_batch(5, versions=(20, 64), feat=160, dtype=np.float64, seed=84, mixing_kappa=1e3)
    for kind in ("lovo", "half"):
        splits = synth.make_splits(batch, kind, 40, seed=84)
        db, ds = rs.DeviceBatch.from_host(batch), rs.DeviceSplits.from_host(splits, batch=batch)
        ref = rs.cv_run(ctx, db, ds, precision=prec, flags=fl)
        R = int(ref["rec_offsets"][-1])
        out = rs.alloc_outputs(R, ds.n_splits, 3)
        ws = torch.empty(ctx.cv_workspace_bytes(db, ds), dtype=torch.uint8, device="cuda")
        for _ in range(2):                       # twice: the second call reuses the workspace
            out.counters.zero_()
            ctx.cv_step(db, ds, ws, out.rec_offsets, out.rec_code, flags=fl, precision=prec,
                        rec_pred=out.rec_pred, pred_all=out.pred_all, counters=out.counters)
            torch.cuda.synchronize()
            ctx.check_device_status()
            np.testing.assert_array_equal(out.rec_offsets.cpu().numpy(), ref["rec_offsets"])
            np.testing.assert_array_equal(out.rec_code.cpu().numpy().view(np.uint32), ref["rec_code"])
            np.testing.assert_array_equal(out.pred_all.cpu().numpy().reshape(R, 6), ref["pred_all"])
            np.testing.assert_array_equal(out.counters.cpu().numpy().view(np.uint64), ref["counters"])
