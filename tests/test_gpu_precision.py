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
