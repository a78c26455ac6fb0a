"""Python binding of the C ABI in ``include/rs.h`` (ctypes; argument marshalling only).

Every step of the method runs in the CUDA library ``_build/librs.so``.  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library is missing or the
device is not a GB300 (sm_103), the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_build", "librs.so")

RS_OK, RS_EINVAL, RS_ENOMEM, RS_ECUDA, RS_ETIMEOUT, RS_EUNSUPPORTED, RS_EDATA = range(7)
RS_F32, RS_F64 = 0, 1
RS_GRAM_F64, RS_GRAM_BF16X3, RS_GRAM_DIST2 = 0, 1, 2
RS_FORM_BATCHED, RS_FORM_PLAIN = 0, 1
RS_RANK_ALL, RS_REFINE_X, RS_MODEL_IBK, RS_MODEL_M5P, RS_PACK_PRED, RS_LOO_CLOSED = 1, 2, 4, 8, 16, 32
IBK_NEIGHBORS = 10
NOPT = 6
COEF_STRIDE = 33
GRAM_LD = 64
NCOUNTERS = 16

# every symbol include/rs.h declares (tests check that the library exports all of them)
EXPORTS = [
    "rs_create", "rs_destroy", "rs_set_stream", "rs_last_error", "rs_check_device_status",
    "rs_standardize", "rs_gram", "rs_gram_workspace_bytes", "rs_rec_offsets", "rs_fit_batched", "rs_predict_rank",
    "rs_cv_workspace_bytes", "rs_cv_step", "rs_measure_fma_peak", "rs_fit_workspace_bytes",
    "rs_profile_enable", "rs_profile_read", "rs_cv_step_static", "rs_gemm_bf16",
    "rs_surrogate_blob_bytes", "rs_surrogate_offset", "rs_surrogate_workspace_bytes",
    "rs_surrogate_train", "rs_surrogate_infer", "rs_cv_graph_create", "rs_cv_graph_launch",
    "rs_cv_graph_destroy", "rs_autotune", "rs_get_tuning", "rs_set_tuning", "rs_transfer", "rs_transfer_workspace_bytes",
    "rs_check_reciprocals", "rs_check_wait_timeout", "rs_fallback_workspace_bytes", "rs_surrogate_fallback",
    "rs_pooled_workspace_bytes", "rs_fit_pooled", "rs_predict_pooled",
    "rs_autotune_gram", "rs_get_gram_tuning", "rs_set_gram_tuning",
    "rs_surrogate_checkpoint_bytes", "rs_surrogate_save", "rs_surrogate_restore",
]


class RsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rs status {status}: {msg}")
        self.status = status


class _Batch(C.Structure):
    _fields_ = [
        ("n_programs", C.c_int32), ("dtype", C.c_int32), ("n_rows", C.c_int64),
        ("max_versions", C.c_int32), ("max_feat", C.c_int32), ("x_elems", C.c_int64),
        ("feat_total", C.c_int64), ("row_offsets", C.c_void_p), ("feat_width", C.c_void_p),
        ("x_offsets", C.c_void_p), ("feat_offsets", C.c_void_p), ("X", C.c_void_p),
        ("masks", C.c_void_p), ("log_time", C.c_void_p), ("cycles", C.c_void_p),
    ]


class _MlpCfg(C.Structure):
    _fields_ = [("batch_rows", C.c_int32), ("use_graph", C.c_int32), ("steps", C.c_int64),
                ("lr", C.c_float), ("weight_decay", C.c_float)]


class _Groups(C.Structure):
    _fields_ = [("n_groups", C.c_int64), ("max_runs", C.c_int32), ("reserved", C.c_int32),
                ("group_offsets", C.c_void_p)]


class _Splits(C.Structure):
    _fields_ = [
        ("n_splits", C.c_int64), ("n_test_rows", C.c_int64), ("max_train", C.c_int32),
        ("reserved", C.c_int32),
        ("split_offsets", C.c_void_p), ("train_masks", C.c_void_p),
    ]


_lib = None


def load(path: str = SO):
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    P = C.c_void_p
    i, d, i64 = C.c_int, C.c_double, C.c_int64
    L.rs_create.argtypes = [C.POINTER(P), i, P]
    L.rs_destroy.argtypes = [P]
    L.rs_set_stream.argtypes = [P, P]
    L.rs_last_error.argtypes = [P]
    L.rs_last_error.restype = C.c_char_p
    L.rs_check_device_status.argtypes = [P]
    L.rs_standardize.argtypes = [P, P, P, P, P]
    L.rs_gram.argtypes = [P, P, i, P, P, C.c_size_t]
    L.rs_gram_workspace_bytes.argtypes = [P, i]
    L.rs_gram_workspace_bytes.restype = C.c_size_t
    L.rs_rec_offsets.argtypes = [P, P, P, P]
    L.rs_fit_batched.argtypes = [P, P, P, P, d, i, P, C.c_size_t, P, P]
    L.rs_predict_rank.argtypes = [P, P, P, P, d, P, i, d, i, i, P, C.c_size_t, P, P, P, P, P]
    L.rs_fit_workspace_bytes.argtypes = [P, P]
    L.rs_fit_workspace_bytes.restype = C.c_size_t
    L.rs_cv_workspace_bytes.argtypes = [P, P]
    L.rs_cv_workspace_bytes.restype = C.c_size_t
    L.rs_cv_step.argtypes = [P, P, P, d, i, d, i, i, P, C.c_size_t, P, P, P, P, P]
    L.rs_measure_fma_peak.argtypes = [i, i, C.POINTER(d)]
    L.rs_check_reciprocals.argtypes = [P, i64, P, P]
    L.rs_check_wait_timeout.argtypes = [P, P, i64, P]
    L.rs_autotune_gram.argtypes = [P, P, P, C.c_size_t, C.POINTER(C.c_float), C.POINTER(C.c_int)]
    L.rs_get_gram_tuning.argtypes = [P, i, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.rs_set_gram_tuning.argtypes = [P, i, i, i]
    L.rs_pooled_workspace_bytes.argtypes = [P]
    L.rs_pooled_workspace_bytes.restype = C.c_size_t
    L.rs_fit_pooled.argtypes = [P, P, P, d, i, P, C.c_size_t, P, P]
    L.rs_predict_pooled.argtypes = [P, P, P, P, i, d, i, P, P, P, P]
    L.rs_fallback_workspace_bytes.argtypes = [P, P]
    L.rs_fallback_workspace_bytes.restype = C.c_size_t
    L.rs_surrogate_fallback.argtypes = [P, P, P, P, d, i, d, i, P, C.c_size_t, P, P, C.POINTER(i64)]
    L.rs_cv_step_static.argtypes = [P, P, P, d, i, d, i, P, P, P, P, P, P, C.c_char_p, C.c_size_t]
    L.rs_gemm_bf16.argtypes = [P, P, i64, P, i64, P, i64, i, i, i]
    L.rs_cv_graph_create.argtypes = [P, P, P, d, i, d, i, i, P, C.c_size_t, P, P, P, P, P, C.POINTER(P)]
    L.rs_cv_graph_launch.argtypes = [P]
    L.rs_cv_graph_destroy.argtypes = [P]
    L.rs_autotune.argtypes = [P, P, P, d, i, d, i, i, P, C.c_size_t, P, P, P, C.POINTER(C.c_float),
                              C.POINTER(C.c_int)]
    L.rs_get_tuning.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.rs_set_tuning.argtypes = [P, i, i, i]
    L.rs_surrogate_blob_bytes.argtypes = []
    L.rs_surrogate_blob_bytes.restype = C.c_size_t
    L.rs_surrogate_offset.argtypes = [i]
    L.rs_surrogate_offset.restype = C.c_int64
    L.rs_surrogate_workspace_bytes.argtypes = [i]
    L.rs_surrogate_workspace_bytes.restype = C.c_size_t
    L.rs_surrogate_train.argtypes = [P, P, P, P, i64, P, P, P, C.c_size_t]
    L.rs_surrogate_infer.argtypes = [P, P, P, i64, C.c_float, P, P, P, P, i, d, i, P, P, P, C.c_size_t, i]
    L.rs_surrogate_checkpoint_bytes.argtypes = []
    L.rs_surrogate_checkpoint_bytes.restype = C.c_size_t
    L.rs_surrogate_save.argtypes = [P, P, P, C.c_size_t]
    L.rs_surrogate_restore.argtypes = [P, P, P, C.c_size_t]
    L.rs_profile_enable.argtypes = [P, i]
    L.rs_profile_read.argtypes = [P, C.POINTER(C.c_float), i, C.POINTER(C.c_int)]
    L.rs_transfer_workspace_bytes.argtypes = [P, P, P, i]
    L.rs_transfer_workspace_bytes.restype = C.c_size_t
    L.rs_transfer.argtypes = [P, P, P, P, d, i, d, i, i, P, C.c_size_t, P, P, P, P, P]
    for name in EXPORTS:
        if name not in ("rs_last_error", "rs_cv_workspace_bytes", "rs_fit_workspace_bytes", "rs_gram_workspace_bytes",
                        "rs_fallback_workspace_bytes", "rs_pooled_workspace_bytes",
                        "rs_transfer_workspace_bytes", "rs_surrogate_blob_bytes", "rs_surrogate_offset", "rs_surrogate_workspace_bytes",
                        "rs_surrogate_checkpoint_bytes"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


@dataclass
class DeviceBatch:
    """Device-resident copy of a ``synth.ProgramBatch`` (or of its standardized Z)."""
    n_programs: int
    dtype: int
    n_rows: int
    max_versions: int
    max_feat: int
    x_elems: int
    feat_total: int
    row_offsets: torch.Tensor
    feat_width: torch.Tensor
    x_offsets: torch.Tensor
    feat_offsets: torch.Tensor
    X: torch.Tensor
    masks: torch.Tensor
    log_time: torch.Tensor
    cycles: Optional[torch.Tensor]

    @staticmethod
    def from_host(b, device="cuda") -> "DeviceBatch":
        fo = np.zeros(b.n_programs + 1, dtype=np.int64)
        fo[1:] = np.cumsum(b.feat_width.astype(np.int64))
        dt = RS_F32 if b.X.dtype == np.float32 else RS_F64
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return DeviceBatch(
            n_programs=b.n_programs, dtype=dt, n_rows=b.n_rows,
            max_versions=int(np.diff(b.row_offsets).max()), max_feat=int(b.feat_width.max()),
            x_elems=int(b.X.shape[0]), feat_total=int(fo[-1]),
            row_offsets=t(b.row_offsets.astype(np.int64)), feat_width=t(b.feat_width.astype(np.int32)),
            x_offsets=t(b.x_offsets.astype(np.int64)), feat_offsets=t(fo), X=t(b.X),
            masks=t(b.masks.astype(np.uint8)), log_time=t(b.log_time.astype(np.float64)),
            cycles=None if b.cycles is None else t(b.cycles.astype(np.float64)))

    def with_X(self, Z: torch.Tensor) -> "DeviceBatch":
        """The same batch with X replaced by a standardized Z (double)."""
        d = dict(self.__dict__)
        d["X"] = Z
        d["dtype"] = RS_F64
        return DeviceBatch(**d)

    def c(self) -> _Batch:
        return _Batch(self.n_programs, self.dtype, self.n_rows, self.max_versions, self.max_feat,
                      self.x_elems, self.feat_total, _ptr(self.row_offsets), _ptr(self.feat_width),
                      _ptr(self.x_offsets), _ptr(self.feat_offsets), _ptr(self.X),
                      _ptr(self.masks), _ptr(self.log_time), _ptr(self.cycles))


@dataclass
class DeviceSplits:
    n_splits: int
    max_train: int
    split_offsets: torch.Tensor
    train_masks: torch.Tensor
    n_test_rows: int = 0

    @staticmethod
    def from_host(s, device="cuda", batch=None) -> "DeviceSplits":
        """Host hints: the largest train-set size and, when the batch is given, the exact
        number of test rows (otherwise the library sizes buffers by an upper bound)."""
        tm = np.ascontiguousarray(s.train_masks, dtype=np.uint64)
        pc = np.zeros(tm.shape, dtype=np.int64)
        x = tm.copy()
        for _ in range(64):
            pc += (x & np.uint64(1)).astype(np.int64)
            x >>= np.uint64(1)
        rows = 0
        if batch is not None and tm.size:
            V = np.diff(batch.row_offsets).astype(np.int64)
            per = np.repeat(V, np.diff(s.split_offsets))
            full = np.where(per >= 64, np.uint64(0xFFFFFFFFFFFFFFFF),
                            (np.uint64(1) << np.minimum(per, 63).astype(np.uint64)) - np.uint64(1))
            y = tm & full
            pin = np.zeros(tm.shape, dtype=np.int64)
            for _ in range(64):
                pin += (y & np.uint64(1)).astype(np.int64)
                y >>= np.uint64(1)
            rows = int((per - pin).sum())
        return DeviceSplits(
            n_splits=int(tm.shape[0]), max_train=int(pc.max()) if tm.size else 0,
            split_offsets=torch.from_numpy(np.ascontiguousarray(s.split_offsets, dtype=np.int64)).to(device),
            train_masks=torch.from_numpy(tm.view(np.int64)).to(device), n_test_rows=rows)

    def c(self) -> _Splits:
        return _Splits(self.n_splits, self.n_test_rows, self.max_train, 0, _ptr(self.split_offsets),
                       _ptr(self.train_masks))


class Context:
    """An ``rs_ctx`` bound to one device and one CUDA stream (torch's current one by default)."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        self.L = load()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        st = self.L.rs_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream))
        if st != RS_OK:
            raise RsError(st, "rs_create failed (is this an sm_103 GPU?)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.rs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != RS_OK:
            raise RsError(st, self.L.rs_last_error(self.h).decode())

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self.L.rs_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    STAGES = ["pairs", "plan_fits", "bucket_fits", "solve", "solve_join", "rank"]

    def profile_enable(self, on: bool = True):
        self._check(self.L.rs_profile_enable(self.h, 1 if on else 0))

    def profile_read(self) -> dict:
        ms = (C.c_float * 8)()
        n = C.c_int(0)
        self._check(self.L.rs_profile_read(self.h, ms, 8, C.byref(n)))
        return {self.STAGES[i]: float(ms[i]) for i in range(n.value)}

    def gemm_bf16(self, A: torch.Tensor, B: torch.Tensor, D: Optional[torch.Tensor] = None):
        """D = A @ B^T on the tensor cores (A [M,K], B [N,K] bfloat16 row-major; D float32)."""
        M, K = A.shape
        N = B.shape[0]
        if D is None:
            D = torch.empty(M, N, dtype=torch.float32, device=A.device)
        self._check(self.L.rs_gemm_bf16(self.h, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(D),
                                        D.stride(0), M, N, K))
        return D

    def cv_graph(self, b: DeviceBatch, s: DeviceSplits, workspace, rec_offsets, rec_code, lam=1e-3, k=3,
                 tau=1.05, flags=0, precision=RS_GRAM_F64, rec_pred=None, pred_all=None, counters=None):
        """Capture the whole step as a CUDA graph; returns a handle with launch() / close()."""
        bc, sc = b.c(), s.c()
        h = C.c_void_p()
        self._check(self.L.rs_cv_graph_create(
            self.h, C.byref(bc), C.byref(sc), float(lam), int(k), float(tau), int(flags), int(precision),
            _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(rec_offsets), _ptr(rec_code),
            _ptr(rec_pred), _ptr(pred_all), _ptr(counters), C.byref(h)))
        ctx = self

        class _G:
            def launch(self_):
                ctx._check(ctx.L.rs_cv_graph_launch(h))

            def close(self_):
                ctx.L.rs_cv_graph_destroy(h)
        return _G()

    def autotune(self, b: DeviceBatch, s: DeviceSplits, workspace, rec_offsets, rec_code, lam=1e-3, k=3,
                 tau=1.05, flags=0, precision=RS_GRAM_F64, rec_pred=None):
        bc, sc = b.c(), s.c()
        times = (C.c_float * 64)()
        n = C.c_int(64)
        self._check(self.L.rs_autotune(
            self.h, C.byref(bc), C.byref(sc), float(lam), int(k), float(tau), int(flags), int(precision),
            _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(rec_offsets), _ptr(rec_code),
            _ptr(rec_pred), times, C.byref(n)))
        return {**self.get_tuning(), "times_ms": [times[i] for i in range(n.value)]}

    def autotune_gram(self, b: DeviceBatch, workspace) -> dict:
        """rs_autotune_gram: the tensor-core Gram's tile shape for this batch's width."""
        bc = b.c()
        times = (C.c_float * 4)()
        choice = C.c_int(0)
        self._check(self.L.rs_autotune_gram(self.h, C.byref(bc), _ptr(workspace),
                                            workspace.numel() * workspace.element_size(), times, C.byref(choice)))
        shapes = [(64, 1), (32, 1), (64, 3), (32, 3)]
        return {"tile_n": shapes[choice.value][0], "ksplit": shapes[choice.value][1],
                "times_ms": {f"{n}x{k}": float(t) for (n, k), t in zip(shapes, times)}}

    def get_gram_tuning(self, feat_width: int) -> dict:
        tn, ks = C.c_int(0), C.c_int(0)
        self._check(self.L.rs_get_gram_tuning(self.h, int(feat_width), C.byref(tn), C.byref(ks)))
        return {"tile_n": tn.value, "ksplit": ks.value}

    def set_gram_tuning(self, feat_width: int, tile_n: int, ksplit: int):
        self._check(self.L.rs_set_gram_tuning(self.h, int(feat_width), int(tile_n), int(ksplit)))

    def get_tuning(self) -> dict:
        sp_, rw, so = C.c_int(), C.c_int(), C.c_int()
        self._check(self.L.rs_get_tuning(self.h, C.byref(sp_), C.byref(rw), C.byref(so)))
        return {"solve_split": sp_.value, "rank_waves": rw.value, "solve_order": so.value}

    def set_tuning(self, solve_split: int = 6, rank_waves: int = 32, solve_order: int = 0):
        self._check(self.L.rs_set_tuning(self.h, int(solve_split), int(rank_waves), int(solve_order)))

    def check_device_status(self):
        self._check(self.L.rs_check_device_status(self.h))

    # ---- entry points (same names as the C ABI) ------------------------------------------
    def standardize(self, b: DeviceBatch, Z=None, mu=None, sigma=None):
        if Z is None:
            Z = torch.empty(b.x_elems, dtype=torch.float64, device=b.X.device)
        bc = b.c()
        self._check(self.L.rs_standardize(self.h, C.byref(bc), _ptr(Z), _ptr(mu), _ptr(sigma)))
        return Z

    def gram(self, zb: DeviceBatch, precision: int = RS_GRAM_F64, K=None, workspace=None):
        if K is None:
            K = torch.zeros(zb.n_programs * GRAM_LD * GRAM_LD, dtype=torch.float64, device=zb.X.device)
        bc = zb.c()
        need = int(self.L.rs_gram_workspace_bytes(C.byref(bc), precision))
        if workspace is None and need:
            workspace = self.workspace(need)
        wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
        self._check(self.L.rs_gram(self.h, C.byref(bc), precision, _ptr(K), _ptr(workspace), wsb))
        return K

    def rec_offsets(self, b: DeviceBatch, s: DeviceSplits, out=None):
        if out is None:
            out = torch.empty(s.n_splits + 1, dtype=torch.int64, device=b.X.device)
        bc, sc = b.c(), s.c()
        self._check(self.L.rs_rec_offsets(self.h, C.byref(bc), C.byref(sc), _ptr(out)))
        return out

    def fit_workspace_bytes(self, b: DeviceBatch, s: DeviceSplits) -> int:
        bc, sc = b.c(), s.c()
        return int(self.L.rs_fit_workspace_bytes(C.byref(bc), C.byref(sc)))

    def workspace(self, nbytes: int) -> torch.Tensor:
        """A device scratch buffer (256-byte aligned by the caching allocator)."""
        return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=f"cuda:{self.device}")

    def fit_batched(self, zb: DeviceBatch, K, s: DeviceSplits, lam: float = 1e-3,
                    form: int = RS_FORM_BATCHED, coef=None, fit_status=None, workspace=None):
        """form: RS_FORM_BATCHED or RS_FORM_PLAIN; RS_FORM_BATCHED | RS_REFINE_X refines each fit
        once through the standardized features of zb; RS_FORM_BATCHED | RS_LOO_CLOSED takes the
        fits of leave-one-version-out splits in closed form."""
        if workspace is None and (form & ~(RS_REFINE_X | RS_LOO_CLOSED)) == RS_FORM_BATCHED:
            workspace = self.workspace(self.fit_workspace_bytes(zb, s))
        bc, sc = zb.c(), s.c()
        wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
        self._check(self.L.rs_fit_batched(self.h, C.byref(bc), _ptr(K), C.byref(sc), float(lam),
                                          int(form), _ptr(workspace), wsb, _ptr(coef),
                                          _ptr(fit_status)))
        return coef, fit_status

    def predict_rank(self, zb: DeviceBatch, K, s: DeviceSplits, rec_offsets, rec_code,
                     lam: float = 1e-3, coef=None, k: int = 3, tau: float = 1.05, flags: int = 0,
                     form: int = RS_FORM_BATCHED, rec_pred=None, pred_all=None, counters=None,
                     workspace=None):
        if workspace is None and form == RS_FORM_BATCHED and coef is None:
            workspace = self.workspace(self.fit_workspace_bytes(zb, s))
        bc, sc = zb.c(), s.c()
        wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
        self._check(self.L.rs_predict_rank(
            self.h, C.byref(bc), _ptr(K), C.byref(sc), float(lam), _ptr(coef), int(k), float(tau),
            int(flags), int(form), _ptr(workspace), wsb, _ptr(rec_offsets), _ptr(rec_code),
            _ptr(rec_pred), _ptr(pred_all), _ptr(counters)))

    def cv_workspace_bytes(self, b: DeviceBatch, s: DeviceSplits) -> int:
        bc, sc = b.c(), s.c()
        return int(self.L.rs_cv_workspace_bytes(C.byref(bc), C.byref(sc)))

    def cv_step(self, b: DeviceBatch, s: DeviceSplits, workspace, rec_offsets, rec_code,
                lam: float = 1e-3, k: int = 3, tau: float = 1.05, flags: int = 0,
                precision: int = RS_GRAM_F64, rec_pred=None, pred_all=None, counters=None):
        bc, sc = b.c(), s.c()
        self._check(self.L.rs_cv_step(
            self.h, C.byref(bc), C.byref(sc), float(lam), int(k), float(tau), int(flags),
            int(precision), _ptr(workspace), workspace.numel() * workspace.element_size(),
            _ptr(rec_offsets), _ptr(rec_code), _ptr(rec_pred), _ptr(pred_all), _ptr(counters)))

    def pooled_workspace_bytes(self, zb: DeviceBatch) -> int:
        bc = zb.c()
        return int(self.L.rs_pooled_workspace_bytes(C.byref(bc)))

    def fit_pooled(self, zb: DeviceBatch, use_program=None, lam: float = 1e-3, flags: int = 0, workspace=None):
        """rs_fit_pooled: one primal ridge model per optimization over the pairs of the selected
        programs of a standardized batch; returns (coef [6][F+1], fit_status [6])."""
        bc = zb.c()
        if workspace is None:
            workspace = self.workspace(self.pooled_workspace_bytes(zb))
        F = zb.max_feat
        coef = torch.empty(NOPT * (F + 1), dtype=torch.float64, device=zb.X.device)
        st = torch.empty(NOPT, dtype=torch.uint8, device=zb.X.device)
        self._check(self.L.rs_fit_pooled(self.h, C.byref(bc), _ptr(use_program), float(lam), int(flags),
                                         _ptr(workspace), workspace.numel() * workspace.element_size(),
                                         _ptr(coef), _ptr(st)))
        return coef.view(NOPT, F + 1), st

    def predict_pooled(self, zb: DeviceBatch, coef, fit_status, rec_code, k: int = 3, tau: float = 1.05,
                       flags: int = 0, rec_pred=None, pred_all=None, counters=None):
        bc = zb.c()
        self._check(self.L.rs_predict_pooled(self.h, C.byref(bc), _ptr(coef.contiguous()), _ptr(fit_status), int(k),
                                             float(tau), int(flags), _ptr(rec_code), _ptr(rec_pred), _ptr(pred_all),
                                             _ptr(counters)))

    def fallback_workspace_bytes(self, b: DeviceBatch, s: DeviceSplits) -> int:
        bc, sc = b.c(), s.c()
        return int(self.L.rs_fallback_workspace_bytes(C.byref(bc), C.byref(sc)))

    def surrogate_fallback(self, b: DeviceBatch, s: DeviceSplits, used_fallback, rec_code, rec_pred=None,
                           lam: float = 1e-3, k: int = 3, tau: float = 1.05, flags: int = 0, workspace=None):
        """rs_surrogate_fallback: the flagged rows of b re-ranked by the plain pass over their
        programs' splits; returns (programs refitted, versions refitted)."""
        if workspace is None:
            workspace = self.workspace(self.fallback_workspace_bytes(b, s))
        bc, sc = b.c(), s.c()
        refit = (C.c_int64 * 2)()
        self._check(self.L.rs_surrogate_fallback(
            self.h, C.byref(bc), C.byref(sc), _ptr(used_fallback), float(lam), int(k), float(tau), int(flags),
            _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(rec_code), _ptr(rec_pred), refit))
        return int(refit[0]), int(refit[1])

    def transfer_workspace_bytes(self, train: DeviceBatch, test: DeviceBatch, groups=None, flags: int = 0) -> int:
        ac, bc = train.c(), test.c()
        g = _groups_c(groups, test)
        return int(self.L.rs_transfer_workspace_bytes(C.byref(ac), C.byref(bc), None if g is None else C.byref(g),
                                                      int(flags)))

    def transfer(self, train: DeviceBatch, test: DeviceBatch, workspace, rec_code, groups=None, lam: float = 1e-3,
                 k: int = 3, tau: float = 1.05, flags: int = 0, opt_mask: int = 0x3F, fit_status=None,
                 rec_pred=None, pred_all=None, counters=None):
        """Table 2 transfer: problem q trains on the runs ``groups[q] .. groups[q+1]-1`` of
        ``train`` (a device int64 tensor of offsets; None: run q) and ranks the versions of
        ``test``'s program q; rows are the test set's versions in order."""
        ac, bc = train.c(), test.c()
        g = _groups_c(groups, test)
        self._check(self.L.rs_transfer(
            self.h, C.byref(ac), C.byref(bc), None if g is None else C.byref(g), float(lam), int(k), float(tau),
            int(flags), int(opt_mask), _ptr(workspace), workspace.numel() * workspace.element_size(),
            _ptr(fit_status), _ptr(rec_code), _ptr(rec_pred), _ptr(pred_all), _ptr(counters)))


def _groups_c(groups, test: "DeviceBatch"):
    """(offsets tensor on the device, max runs) -> the C struct; None stays None."""
    if groups is None:
        return None
    offs, max_runs = groups
    if offs.dtype != torch.int64 or offs.numel() != test.n_programs + 1:
        raise ValueError("group offsets: int64 tensor of n_programs + 1 entries")
    return _Groups(test.n_programs, int(max_runs), 0, _ptr(offs))


class Surrogate:
    """The MLP surrogate's state (one device blob) and its training / inference calls."""
    NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")
    SHAPES = {"W1": (512, 256), "b1": (512,), "W2": (512, 512), "b2": (512,), "W3": (16, 512), "b3": (16,)}

    def __init__(self, ctx: "Context", batch_rows: int = 8192, infer_chunk: int = 0):
        self.ctx = ctx
        L = ctx.L
        self.blob = torch.zeros(L.rs_surrogate_blob_bytes() // 4, dtype=torch.float32,
                                device=f"cuda:{ctx.device}")
        self.batch_rows = batch_rows
        self.ws = ctx.workspace(L.rs_surrogate_workspace_bytes(batch_rows))
        self.infer_chunk = infer_chunk or batch_rows
        self.iws = self.ws if self.infer_chunk == batch_rows else ctx.workspace(
            L.rs_surrogate_workspace_bytes(self.infer_chunk))
        self.off = {n: int(L.rs_surrogate_offset(i)) for i, n in enumerate(self.NAMES)}
        self.off.update({"m": int(L.rs_surrogate_offset(6)), "v": int(L.rs_surrogate_offset(7)),
                         "grad": int(L.rs_surrogate_offset(8)), "stats": int(L.rs_surrogate_offset(9))})

    def view(self, name: str, region: str = "param") -> torch.Tensor:
        base = {"param": 0, "m": self.off["m"], "v": self.off["v"], "grad": self.off["grad"]}[region]
        o = base + self.off[name]
        shp = self.SHAPES[name]
        n = int(np.prod(shp))
        return self.blob[o:o + n].view(*shp)

    def load(self, params: dict):
        """Write initial weights (numpy, shapes of the FP64 reference; W3 is [6][512])."""
        self.blob.zero_()
        for k, v in params.items():
            t = torch.from_numpy(np.asarray(v, dtype=np.float32)).to(self.blob.device)
            dst = self.view(k)
            if k in ("W3", "b3"):
                dst[:t.shape[0]].copy_(t)
            else:
                dst.copy_(t)

    def save(self, path: str) -> int:
        """Write a checkpoint of the whole state (rs_surrogate_save) to `path`; returns the
        optimizer steps taken so far."""
        n = int(self.ctx.L.rs_surrogate_checkpoint_bytes())
        buf = (C.c_ubyte * n)()
        self.ctx._check(self.ctx.L.rs_surrogate_save(self.ctx.h, _ptr(self.blob), buf, n))
        data = bytes(buf)
        with open(path, "wb") as f:
            f.write(data)
        return int.from_bytes(data[32:40], "little", signed=True)

    def restore(self, path: str) -> None:
        """Load a checkpoint written by save (rs_surrogate_restore checks its header); training
        then continues where the saved run stopped."""
        with open(path, "rb") as f:
            data = f.read()
        buf = (C.c_ubyte * len(data)).from_buffer_copy(data)
        self.ctx._check(self.ctx.L.rs_surrogate_restore(self.ctx.h, _ptr(self.blob), buf, len(data)))

    def train(self, X, Y, steps: int, lr: float = 1e-3, weight_decay: float = 0.0, use_graph: bool = True,
              loss_curve=None):
        cfg = _MlpCfg(self.batch_rows, 1 if use_graph else 0, int(steps), float(lr), float(weight_decay))
        self.ctx._check(self.ctx.L.rs_surrogate_train(
            self.ctx.h, _ptr(self.blob), _ptr(X), _ptr(Y), X.shape[0], C.byref(cfg), _ptr(loss_curve),
            _ptr(self.ws), self.ws.numel()))

    def infer(self, X, ood_threshold: float = 1e30, want_ood: bool = False, chunk_rows=None,
              want_pred: bool = True, masks=None, k: int = 3, tau: float = 1.05, flags: int = 0,
              rec_code=None, rec_pred=None):
        n = X.shape[0]
        pred = torch.empty(n, 6, dtype=torch.float32, device=X.device) if want_pred else None
        score = torch.empty(n, dtype=torch.float32, device=X.device) if want_ood else None
        fb = torch.empty(n, dtype=torch.uint8, device=X.device) if want_ood else None
        self.ctx._check(self.ctx.L.rs_surrogate_infer(
            self.ctx.h, _ptr(self.blob), _ptr(X), n, float(ood_threshold), _ptr(pred), _ptr(score), _ptr(fb),
            _ptr(masks), int(k), float(tau), int(flags), _ptr(rec_code), _ptr(rec_pred),
            _ptr(self.iws), self.iws.numel(), int(chunk_rows or self.infer_chunk)))
        return pred, score, fb


def check_reciprocals(d: torch.Tensor) -> torch.Tensor:
    """[n][4]: the solvers' reciprocal and reciprocal square root of each positive double in
    d, beside CUDA's 1.0 / d and 1.0 / sqrt(d) (rs_check_reciprocals)."""
    L = load()
    out = torch.empty(d.numel(), 4, dtype=torch.float64, device=d.device)
    st = L.rs_check_reciprocals(_ptr(d), d.numel(), _ptr(out),
                                C.c_void_p(torch.cuda.current_stream(d.device).cuda_stream))
    if st != RS_OK:
        raise RsError(st, "rs_check_reciprocals failed")
    return out


def measure_fma_peak(f64: bool = True, iters: int = 4096) -> float:
    """GFLOP/s of independent FMA chains over the whole device (FP64 or FP32)."""
    L = load()
    g = C.c_double(0.0)
    st = L.rs_measure_fma_peak(1 if f64 else 0, int(iters), C.byref(g))
    if st != RS_OK:
        raise RsError(st, "rs_measure_fma_peak failed")
    return g.value


@dataclass
class CVOutputs:
    rec_offsets: torch.Tensor
    rec_code: torch.Tensor
    rec_pred: Optional[torch.Tensor]
    pred_all: Optional[torch.Tensor]
    counters: torch.Tensor


def alloc_outputs(n_rows_total: int, n_splits: int, k: int, device="cuda", pred_all=True,
                  rec_pred=True) -> CVOutputs:
    return CVOutputs(
        rec_offsets=torch.empty(n_splits + 1, dtype=torch.int64, device=device),
        rec_code=torch.empty(n_rows_total, dtype=torch.int32, device=device),
        rec_pred=torch.empty(n_rows_total * k, dtype=torch.float64, device=device) if rec_pred else None,
        pred_all=torch.empty(n_rows_total * NOPT, dtype=torch.float64, device=device) if pred_all else None,
        counters=torch.zeros(NCOUNTERS, dtype=torch.int64, device=device))


def cv_run(ctx: Context, b: DeviceBatch, s: DeviceSplits, lam=1e-3, k=3, tau=1.05, flags=0,
           precision=RS_GRAM_F64, form=RS_FORM_BATCHED, want_pred_all=True, want_Z=False):
    """The whole pass through the individual entry points; returns host numpy outputs.
    With RS_MODEL_IBK in flags the block is the distance block (RS_GRAM_DIST2)."""
    if flags & RS_MODEL_IBK:
        precision = RS_GRAM_DIST2
    dev = b.X.device
    Z = torch.empty(b.x_elems, dtype=torch.float64, device=dev)
    mu = torch.empty(b.feat_total, dtype=torch.float64, device=dev)
    sg = torch.empty(b.feat_total, dtype=torch.float64, device=dev)
    ctx.standardize(b, Z, mu, sg)
    zb = b.with_X(Z)
    K = ctx.gram(zb, precision)
    ro = ctx.rec_offsets(zb, s)
    R = int(ro[-1].item())
    out = alloc_outputs(R, s.n_splits, k, dev, pred_all=want_pred_all)
    out.rec_offsets = ro
    ctx.predict_rank(zb, K, s, ro, out.rec_code, lam=lam, k=k, tau=tau, flags=flags, form=form,
                     rec_pred=out.rec_pred, pred_all=out.pred_all, counters=out.counters)
    torch.cuda.synchronize(dev)
    ctx.check_device_status()
    res = dict(rec_offsets=ro.cpu().numpy(), rec_code=out.rec_code.cpu().numpy().view(np.uint32),
               rec_pred=out.rec_pred.cpu().numpy().reshape(R, k),
               counters=out.counters.cpu().numpy().view(np.uint64), mu=mu.cpu().numpy(),
               sigma=sg.cpu().numpy(), K=K)
    if want_pred_all:
        res["pred_all"] = out.pred_all.cpu().numpy().reshape(R, NOPT)
    if want_Z:
        res["Z"] = Z.cpu().numpy()
    return res


def transfer_run(ctx: Context, train: DeviceBatch, test: DeviceBatch, groups=None, lam=1e-3, k=3, tau=1.05,
                 flags=0, opt_mask=0x3F):
    """One transfer call with fresh outputs; returns host numpy outputs.  groups: host array of
    Q + 1 run offsets, or None (run q trains problem q)."""
    dev = train.X.device
    R, Q = test.n_rows, test.n_programs
    g = None
    if groups is not None:
        offs = np.ascontiguousarray(groups, dtype=np.int64)
        g = (torch.from_numpy(offs).to(dev), int(np.diff(offs).max()))
    ws = ctx.workspace(ctx.transfer_workspace_bytes(train, test, g, flags))
    out = alloc_outputs(R, 0, k, dev)
    st = torch.empty(Q * NOPT, dtype=torch.uint8, device=dev)
    ctx.transfer(train, test, ws, out.rec_code, groups=g, lam=lam, k=k, tau=tau, flags=flags, opt_mask=opt_mask,
                 fit_status=st, rec_pred=out.rec_pred, pred_all=out.pred_all, counters=out.counters)
    torch.cuda.synchronize(dev)
    ctx.check_device_status()
    return dict(rec_code=out.rec_code.cpu().numpy().view(np.uint32),
                rec_pred=out.rec_pred.cpu().numpy().reshape(R, k),
                pred_all=out.pred_all.cpu().numpy().reshape(R, NOPT),
                counters=out.counters.cpu().numpy().view(np.uint64),
                fit_status=st.cpu().numpy().reshape(Q, NOPT))
