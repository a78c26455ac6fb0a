"""The C ABI library builds for sm_103a, loads without a GPU, and exports every entry point
that include/rs.h declares (no compute calls: this runs on CPU-only machines)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rs_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1910_07776_gb300 import build, rs
    so = build.build()
    lib = ctypes.CDLL(so)
    decl = declared_symbols()
    assert len(decl) >= 12
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(set(rs.EXPORTS)) == [n for n in decl if n in rs.EXPORTS]
    assert set(decl) <= set(rs.EXPORTS) | set(getattr(rs, "EXTRA_EXPORTS", []))


def test_workspace_query_needs_no_gpu():
    import numpy as np
    from paper_1910_07776_gb300 import rs, synth
    lib = rs.load()
    b = synth.make_batch(3, versions=(5, 64), feat=20, seed=0)
    cb = rs._Batch(b.n_programs, 0, b.n_rows, 64, 20, b.X.shape[0], int(b.feat_width.sum()),
                   None, None, None, None, None, None, None, None)
    S = 100
    cs = rs._Splits(S, 0, 32, 0, None, None)
    fit = lib.rs_fit_workspace_bytes(ctypes.byref(cb), ctypes.byref(cs))
    # per fit: pair mask, size, 16-byte record in bucket order, offset, status, and up to 17
    # coefficient doubles;
    # per test row (bound: S x max_versions when no row count is given): six predictions
    # and the row's scoring record; per (program, optimization) the pairs' slot sets with their
    # move masks (14 words), and a flag and a 32-bit label mask of the closed-form
    # leave-one-out fits, whose tables (a 32 x 32 inverse, two 32-vectors and their sums) share
    # the coefficient records' region; per program a flag
    coef_region = max(S * 6 * 17 * 8, b.n_programs * 6 * (32 * 32 + 68) * 8)
    need_fit = (S * 6 * (4 + 1 + 16 + 8 + 1) + coef_region + S * 64 * (6 * 8 + 8)
                + b.n_programs * 6 * (1 + 4 + 14 * 8) + b.n_programs)
    assert need_fit <= fit <= need_fit + 64 * 1024
    cs.n_test_rows = 1000
    fit2 = lib.rs_fit_workspace_bytes(ctypes.byref(cb), ctypes.byref(cs))
    assert abs(fit2 - fit - (1000 - S * 64) * 56) < 1024
    cs.n_test_rows = 0
    nbytes = lib.rs_cv_workspace_bytes(ctypes.byref(cb), ctypes.byref(cs))
    need = b.X.shape[0] * 8 + 3 * 64 * 64 * 8 + fit
    assert need <= nbytes <= need + 1024
    assert lib.rs_cv_workspace_bytes(None, None) == 0
    assert lib.rs_fit_workspace_bytes(None, None) == 0


def test_invalid_arguments_are_rejected_before_any_launch():
    from paper_1910_07776_gb300 import rs
    lib = rs.load()
    assert lib.rs_create(None, 0, None) == rs.RS_EINVAL
    assert lib.rs_destroy(None) == rs.RS_EINVAL
    assert lib.rs_standardize(None, None, None, None, None) == rs.RS_EINVAL
    assert lib.rs_last_error(None) == b"context is NULL"
