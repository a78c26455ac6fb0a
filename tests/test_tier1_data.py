"""The measured tier-1 data set (tier1/nb_gb300.npz: the 64 versions of the n-body code NB with
the six optimizations of Sec. 3.3, profiled on a GB300): its layout, and the GPU pass against
the FP64 reference on it (leave-one-version-out, ridge and IBK; Table 2 experiments with NB in
the place of BH).  Skipped where the file has not been recorded."""
import math

import numpy as np
import pytest

import oracle
from paper_1910_07776_gb300 import synth, tier1
from parity import close, compare_counters, compare_rankings

pytestmark = pytest.mark.skipif(not tier1.available(), reason="no recorded tier-1 data")


def test_layout_of_the_recorded_data():
    b = tier1.load_nb()
    n_in, runs = len(b.meta["inputs"]), b.meta["runs"]
    assert b.n_programs == n_in * runs
    assert np.all(np.diff(b.row_offsets) == 64)
    for p in range(b.n_programs):
        assert sorted(b.masks[b.program_rows(p)].tolist()) == list(range(64))
    assert np.isfinite(b.log_time).all() and np.isfinite(b.X).all() and (b.X >= 0).all()
    assert b.meta["index"][0] == ("NB", 0, 0)
    # every version was timed: speedups of the 6 optimizations are defined for all 32 pairs
    r = oracle.cv_batch(b, synth.make_splits(b, "lovo"))
    assert r.counter("fit_ok") > 0


@pytest.mark.gpu
@pytest.mark.parametrize("model", ["ridge", "ibk"])
def test_gpu_lovo_on_measured_data_matches_the_reference(model):
    from paper_1910_07776_gb300 import build, rs
    build.build()
    b = tier1.load_nb()
    sp = synth.make_splits(b, "lovo")
    ctx = rs.Context(0)
    flags = rs.RS_MODEL_IBK if model == "ibk" else 0
    g = rs.cv_run(ctx, rs.DeviceBatch.from_host(b), rs.DeviceSplits.from_host(sp, batch=b), flags=flags)
    r = oracle.cv_batch(b, sp, model=model)
    ctx.close()
    np.testing.assert_array_equal(g["rec_offsets"], r.rec_offsets)
    if model == "ibk":
        np.testing.assert_array_equal(g["pred_all"], r.pred_all)
        np.testing.assert_array_equal(g["rec_code"], r.rec_code)
        np.testing.assert_array_equal(g["counters"][:14], r.counters[:14])
    else:
        # two FP64 solvers of one system agree to about kappa * eps; the z-scores of a
        # program's 64 versions have trace(Z Z^T) = 64 F, which bounds the largest eigenvalue of
        # K + lambda I, so kappa <= 1 + 64 F / lambda
        kappa = 1 + 64 * int(b.feat_width[0]) / 1e-3
        scale = np.nanmax(np.abs(r.pred_all))
        close(g["pred_all"], r.pred_all, rel=1e-9, abs_=kappa * np.finfo(float).eps * max(1.0, scale))
        _, nnear = compare_rankings(g["rec_code"], r.rec_code, r.pred_all, math.log(1.05))
        compare_counters(g["counters"], r.counters, slack=nnear)
