"""FP64 CPU reference for the recommendation path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library never loads it and shares no code with it.

``build()`` compiles ``rs_oracle.c`` and ``rs_m5p.c`` (plain C, double precision, ``-ffp-contract=off``
so every operation rounds once, in source order) into ``oracle/_build``.  The C library's
``log`` may still differ in the last ulp between machines (x86-64 and AArch64 do), so the
reference is always run on the machine whose results it is compared with.  The Python
functions below only marshal numpy arrays into the C functions; the MLP reference used
for the surrogate lives in ``mlp.py`` (numpy, float64).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "librs_oracle.so")
_SO_ASAN = os.path.join(_HERE, "_build", "librs_oracle_asan.so")
_lib = None

N_OPT = 6
N_COUNTERS = 16
EPS = 1e-30
COUNTER_NAMES = [
    "n_rows", "n_pred", "n_scored", "sign_hits", "n_rec", "rec_known", "rec_hits",
    "top1_rows", "top1_hits", "fit_ok", "fit_empty", "fit_notpd", "fit_nonfinite",
    "unscored_invalid", "reserved14", "reserved15",
]
FIT_OK, FIT_EMPTY, FIT_NOTPD, FIT_NONFINITE = 0, 1, 2, 3
RANK_ALL = 1
MODEL_IBK = 4
MODEL_M5P = 8
IBK_NEIGHBORS = 10          # k of the instance-based learner (Sec. 3.4: k = 10)


def build(force: bool = False, sanitize: bool = False) -> str:
    """Compile the C reference with gcc (OpenMP over splits, IEEE double, no FP contraction).
    sanitize=True builds a separate AddressSanitizer copy (``librs_oracle_asan.so``, same
    arithmetic) that a test loads in a child process to check the oracle's memory accesses."""
    srcs = [os.path.join(_HERE, f) for f in ("rs_oracle.c", "rs_m5p.c")]
    so = _SO_ASAN if sanitize else _SO
    os.makedirs(os.path.dirname(so), exist_ok=True)
    if force or not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(f) for f in srcs):
        tmp = so + f".tmp{os.getpid()}"
        extra = ["-g", "-fsanitize=address", "-fno-omit-frame-pointer"] if sanitize else []
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", *extra, "-o", tmp, *srcs, "-lm"])
        os.replace(tmp, so)
    return so


def lib():
    """The oracle's C library; ``RS_ORACLE_SO`` names another build of it (the sanitized one)."""
    global _lib
    if _lib is None:
        so = os.environ.get("RS_ORACLE_SO") or build()
        L = C.CDLL(so)
        P = C.c_void_p
        L.orc_standardize.argtypes = [C.c_int, C.c_int, P, P, C.c_double, P, P, P]
        L.orc_pairs.argtypes = [C.c_int, P, C.c_int, P, P]
        L.orc_pairs.restype = C.c_int
        L.orc_cholesky.argtypes = [C.c_int, P]
        L.orc_cholesky.restype = C.c_int
        L.orc_cholesky_solve.argtypes = [C.c_int, P, P]
        L.orc_ridge_fit.argtypes = [C.c_int, C.c_int, P, P, C.c_double, P, P, P]
        L.orc_ridge_fit.restype = C.c_int
        L.orc_rank.argtypes = [P, P, C.c_int, C.c_double, P]
        L.orc_rank.restype = C.c_int
        L.orc_rec_offsets.argtypes = [C.c_int, P, P, P, P]
        L.orc_cv_batch.argtypes = [C.c_int, P, P, P, P, P, C.c_int, P, P, P, P, P, C.c_double,
                                   C.c_int, C.c_double, C.c_int, C.c_double, P, P, P, P, P, P,
                                   P, P, P, C.c_int, C.c_int]
        L.orc_ibk_predict.argtypes = [C.c_int, C.c_int, P, P, P, C.c_int]
        L.orc_transfer.argtypes = [C.c_int, P, P, P, P, P, P, P, P, P, P, P, P, P, P, C.c_double,
                                   C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_double, P, P, P, P,
                                   P]
        L.orc_ibk_predict.restype = C.c_double
        L.orc_m5p_fit_predict.argtypes = [C.c_int, C.c_int, P, P, C.c_int, P, P, P, P]
        L.orc_m5p_fit_predict.restype = C.c_int
        L.orc_num_threads_available.restype = C.c_int
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def standardize(X: np.ndarray, cycles: Optional[np.ndarray] = None, eps: float = EPS):
    """Sec. 2 feature vectors (counters / cycles), log, per-feature z-score over the rows."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    V, F = X.shape
    cyc = None if cycles is None else np.ascontiguousarray(cycles, dtype=np.float64)
    Z = np.empty_like(X)
    mu = np.empty(F)
    sg = np.empty(F)
    lib().orc_standardize(V, F, _p(X), _p(cyc), eps, _p(Z), _p(mu), _p(sg))
    return Z, mu, sg


def pairs(masks: np.ndarray, j: int):
    """Sec. 3.3 before/after version pairs of optimization j (brute force)."""
    m = np.ascontiguousarray(masks, dtype=np.uint8)
    b = np.zeros(64, dtype=np.int32)
    a = np.zeros(64, dtype=np.int32)
    n = lib().orc_pairs(int(m.shape[0]), _p(m), int(j), _p(b), _p(a))
    return b[:n].copy(), a[:n].copy()


def cholesky(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64).copy()
    st = lib().orc_cholesky(A.shape[0], _p(A))
    return st, np.tril(A)


def ridge_fit(Z: np.ndarray, y: np.ndarray, lam: float):
    """Ridge with unpenalised intercept by the primal normal equations (Sec. 3.4 family)."""
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n, F = Z.shape if Z.ndim == 2 else (0, Z.shape[-1])
    beta = np.zeros(F)
    b = C.c_double(0.0)
    work = np.zeros(F * F + 2 * F)
    st = lib().orc_ridge_fit(n, F, _p(Z), _p(y), lam, _p(beta), C.byref(b), _p(work))
    return st, beta, b.value


def rank(pred: np.ndarray, valid: np.ndarray, k: int, log_tau: float):
    """Sec. 2 Tier 3: sort descending (ties: lower index), threshold, top k."""
    p = np.ascontiguousarray(pred, dtype=np.float64)
    v = np.ascontiguousarray(valid, dtype=np.int32)
    idx = np.zeros(N_OPT, dtype=np.int32)
    c = lib().orc_rank(_p(p), _p(v), int(k), float(log_tau), _p(idx))
    return idx[:c].copy()


@dataclass
class CVResult:
    Z: np.ndarray
    mu: np.ndarray
    sigma: np.ndarray
    fit_status: np.ndarray
    rec_offsets: np.ndarray
    rec_code: np.ndarray
    rec_pred: np.ndarray
    pred_all: np.ndarray
    counters: np.ndarray

    def counter(self, name: str) -> int:
        return int(self.counters[COUNTER_NAMES.index(name)])


def _check_versions(batch):
    """A program (or run) holds at most 64 versions, one per 6-bit mask (Sec. 3.3); the C
    code keeps per-program tables of that size."""
    v = np.diff(np.asarray(batch.row_offsets))
    if v.size and (v.min() < 0 or v.max() > 64):
        raise ValueError("every program needs 0..64 versions")
    if batch.masks.size and int(np.max(batch.masks)) > 63:
        raise ValueError("optimization masks are 6-bit")


def rec_offsets(batch, splits) -> np.ndarray:
    out = np.zeros(splits.n_splits + 1, dtype=np.int64)
    lib().orc_rec_offsets(batch.n_programs, _p(np.ascontiguousarray(batch.row_offsets)),
                          _p(np.ascontiguousarray(splits.split_offsets)),
                          _p(np.ascontiguousarray(splits.train_masks)), _p(out))
    return out


def cv_batch(batch, splits, lam: float = 1e-3, k: int = 3, tau: float = 1.05, flags: int = 0,
             nthreads: int = 1, want_Z: bool = True, model: str = "ridge",
             ibk_k: int = IBK_NEIGHBORS) -> CVResult:
    """Whole pass (standardize, pairs, fits, predictions, ranking, counters) for a batch.
    model "ridge" (Sec. 3.4 regression) or "ibk" (Sec. 3.4 instance-based, ibk_k nearest)."""
    if model not in ("ridge", "ibk"):
        raise ValueError("model must be 'ridge' or 'ibk'")
    if model == "ibk":
        flags |= MODEL_IBK
    _check_versions(batch)
    L = lib()
    P = batch.n_programs
    fo = np.zeros(P + 1, dtype=np.int64)
    fo[1:] = np.cumsum(batch.feat_width.astype(np.int64))
    x_is_f32 = 1 if batch.X.dtype == np.float32 else 0
    X = np.ascontiguousarray(batch.X)
    S = splits.n_splits
    ro = rec_offsets(batch, splits)
    R = int(ro[-1])
    Z = np.empty(X.shape[0], dtype=np.float64) if want_Z else None
    mu = np.empty(int(fo[-1]))
    sg = np.empty(int(fo[-1]))
    fs = np.zeros(S * N_OPT, dtype=np.uint8)
    code = np.zeros(R, dtype=np.uint32)
    rp = np.zeros(R * k, dtype=np.float64)
    pa = np.zeros(R * N_OPT, dtype=np.float64)
    cnt = np.zeros(N_COUNTERS, dtype=np.uint64)
    cyc = None if batch.cycles is None else np.ascontiguousarray(batch.cycles, dtype=np.float64)
    L.orc_cv_batch(P, _p(np.ascontiguousarray(batch.row_offsets)),
                   _p(np.ascontiguousarray(batch.feat_width, dtype=np.int32)),
                   _p(np.ascontiguousarray(batch.x_offsets)), _p(fo), _p(X), x_is_f32,
                   _p(np.ascontiguousarray(batch.masks)),
                   _p(np.ascontiguousarray(batch.log_time)), _p(cyc),
                   _p(np.ascontiguousarray(splits.split_offsets)),
                   _p(np.ascontiguousarray(splits.train_masks)), float(lam), int(k),
                   float(np.log(tau)), int(flags), EPS, _p(Z), _p(mu), _p(sg), _p(fs), _p(ro),
                   _p(code), _p(rp), _p(pa), _p(cnt), int(nthreads), int(ibk_k))
    return CVResult(Z=Z, mu=mu, sigma=sg, fit_status=fs.reshape(S, N_OPT), rec_offsets=ro,
                    rec_code=code, rec_pred=rp.reshape(R, k), pred_all=pa.reshape(R, N_OPT),
                    counters=cnt)


@dataclass
class TransferResult:
    fit_status: np.ndarray       # [Q][6]
    rec_offsets: np.ndarray      # [Q + 1]: test rows of problem q start at rec_offsets[q]
    rec_code: np.ndarray
    rec_pred: np.ndarray
    pred_all: np.ndarray
    counters: np.ndarray

    def counter(self, name: str) -> int:
        return int(self.counters[COUNTER_NAMES.index(name)])


def transfer(train, test, groups=None, lam: float = 1e-3, k: int = 3, tau: float = 1.05, flags: int = 0,
             opt_mask: int = 0x3F, model: str = "ridge", ibk_k: int = IBK_NEIGHBORS) -> TransferResult:
    """Sec. 5 / Table 2: for every problem q, a model trained on all pairs of the runs
    groups[q] .. groups[q+1]-1 of ``train`` (standardized together) predicts, ranks and scores
    every version of ``test``'s program q (standardized with the training runs' statistics).
    groups defaults to one run per problem.  opt_mask limits the candidate optimizations."""
    if model not in ("ridge", "ibk", "m5p"):
        raise ValueError("model must be 'ridge', 'ibk' or 'm5p'")
    if model == "ibk":
        flags |= MODEL_IBK
    if model == "m5p":
        flags |= MODEL_M5P
    _check_versions(train)
    _check_versions(test)
    L = lib()
    Q = test.n_programs
    g = np.arange(Q + 1, dtype=np.int64) if groups is None else np.ascontiguousarray(groups, dtype=np.int64)
    assert g.shape == (Q + 1,) and g[0] == 0 and g[-1] <= train.n_programs and np.all(np.diff(g) >= 1)
    for q in range(Q):
        assert np.all(train.feat_width[g[q]:g[q + 1]] == test.feat_width[q])
    ro = np.zeros(Q + 1, dtype=np.int64)
    ro[1:] = np.cumsum(np.diff(test.row_offsets))
    R = int(ro[-1])
    fs = np.zeros(Q * N_OPT, dtype=np.uint8)
    code = np.zeros(R, dtype=np.uint32)
    rp = np.zeros(R * k, dtype=np.float64)
    pa = np.zeros(R * N_OPT, dtype=np.float64)
    cnt = np.zeros(N_COUNTERS, dtype=np.uint64)
    c64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    cy = lambda b: None if b.cycles is None else c64(b.cycles)
    L.orc_transfer(Q, _p(g), _p(np.ascontiguousarray(train.feat_width, dtype=np.int32)),
                   _p(np.ascontiguousarray(train.row_offsets)), _p(np.ascontiguousarray(train.x_offsets)),
                   _p(c64(train.X)), _p(np.ascontiguousarray(train.masks)), _p(c64(train.log_time)),
                   _p(cy(train)), _p(np.ascontiguousarray(test.row_offsets)),
                   _p(np.ascontiguousarray(test.x_offsets)), _p(c64(test.X)),
                   _p(np.ascontiguousarray(test.masks)), _p(c64(test.log_time)), _p(cy(test)),
                   float(lam), int(k), float(np.log(tau)), int(flags), int(opt_mask), int(ibk_k), EPS,
                   _p(fs), _p(code), _p(rp), _p(pa), _p(cnt))
    return TransferResult(fit_status=fs.reshape(Q, N_OPT), rec_offsets=ro, rec_code=code,
                          rec_pred=rp.reshape(R, k), pred_all=pa.reshape(R, N_OPT), counters=cnt)


def m5p_fit_predict(Zrows, y, Zt):
    """The M5P model tree (rs_m5p.c) fitted on (Zrows, y), predicting the rows of Zt; returns
    (predictions, leaves, nodes after pruning)."""
    Zrows = np.ascontiguousarray(Zrows, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    Zt = np.ascontiguousarray(np.atleast_2d(Zt), dtype=np.float64)
    n, F = Zrows.shape
    out = np.zeros(Zt.shape[0])
    lv, nd = C.c_int(0), C.c_int(0)
    st = lib().orc_m5p_fit_predict(n, F, _p(Zrows), _p(y), Zt.shape[0], _p(Zt), _p(out), C.byref(lv), C.byref(nd))
    if st:
        raise ValueError("m5p: 1 <= n <= 128 instances")
    return out, lv.value, nd.value


def ibk_predict(Zrows, y, zt, k: int = IBK_NEIGHBORS) -> float:
    """Sec. 3.4 IBK for one test vector: mean label of the k nearest training rows."""
    Zrows = np.ascontiguousarray(Zrows, dtype=np.float64)
    n, F = Zrows.shape
    if n < 1 or not 1 <= k <= 64:
        raise ValueError("IBK needs n >= 1 training rows and 1 <= k <= 64")
    return float(lib().orc_ibk_predict(n, F, _p(Zrows), _p(np.ascontiguousarray(y, dtype=np.float64)),
                                       _p(np.ascontiguousarray(zt, dtype=np.float64)), int(k)))


def decode_rec(code: np.ndarray):
    """Unpack rec_code words into (count, [idx...]) lists."""
    out = []
    for c in np.asarray(code, dtype=np.uint64):
        c = int(c)
        n = c & 0xF
        out.append([(c >> (4 + 4 * a)) & 0xF for a in range(n)])
    return out


def threads_available() -> int:
    return int(lib().orc_num_threads_available())
