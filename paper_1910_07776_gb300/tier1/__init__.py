"""Measured tier-1 data (Sec. 2): the 64 versions of a direct n-body code (NB, Sec. 3.2-3.3),
profiled on this GPU by ``capture.py``; ``load_nb`` turns the recorded file into the program
batch the speedup-prediction path takes (one program per input and run, all 64 versions)."""
from __future__ import annotations

import os

import numpy as np

from .. import synth

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "nb_gb300.npz")


def available(path: str = DATA) -> bool:
    return os.path.exists(path)


def load_nb(path: str = DATA) -> synth.ProgramBatch:
    """One program per (input, run), in that nesting order (``meta["index"]`` lists
    ("NB", input, run)), 64 versions each (version = optimization mask, bit order of
    nbody.cu); X = the counters divided by the kernel's cycles (cycles = None: already
    normalised), log_time = log of the version's run time of that input."""
    d = np.load(path, allow_pickle=False)
    feats, times = d["features"], d["time_ms"]          # [run][input][mask][F], [run][input][mask]
    runs, n_in, _, F = feats.shape
    X, lt, masks, index = [], [], [], []
    for i in range(n_in):
        for r in range(runs):
            X.append(np.maximum(feats[r, i], 0.0).reshape(-1))
            lt.append(np.log(times[r, i]))
            masks.append(np.arange(64, dtype=np.uint8))
            index.append(("NB", i, r))
    P = len(index)
    return synth.ProgramBatch(
        X=np.concatenate(X).astype(np.float64), x_offsets=np.arange(P, dtype=np.int64) * 64 * F,
        row_offsets=np.arange(P + 1, dtype=np.int64) * 64, feat_width=np.full(P, F, dtype=np.int32),
        masks=np.concatenate(masks), log_time=np.concatenate(lt).astype(np.float64), cycles=None,
        meta={"index": index, "runs": runs, "codes": [("NB", n_in)], "counters": list(d["counters"]),
              "inputs": d["inputs"].tolist(), "gpu": str(d["gpu"]), "command": str(d["command"])})
