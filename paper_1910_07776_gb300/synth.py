"""Seeded synthetic inputs shaped like the paper's profiling data (generator "gen/v1").

The paper profiles 64 versions of each subject program, one per combination of six
source-code optimizations (Sec. 3.3), and normalises hardware-counter readings by the
cycle count to form feature vectors (Sec. 2).  Its profiles are not available, so this
module draws stand-ins with the same structure:

* a version is a 6-bit optimization mask; a program owns a set of distinct masks;
* every version has F positive counter readings, a cycle count and a run time;
* adding optimization ``j`` to version ``v`` changes the run time by a program- and
  mask-dependent factor (per-optimization main effects plus pairwise interactions).

This module holds input generation only.  It computes no log/z-score, no pair, no fit,
no prediction and no ranking: those belong to the method and live on each side of the
parity check (the CPU reference and the CUDA library) separately.

Recipe (all draws from one numpy PCG64 stream per call, so a seed fixes every byte):

* latent program state ``h_p ~ N(0, I_8)``;
* main effect of optimization j: ``a_pj = 0.3 * w_j.h_p / |w_j|`` (marginally N(0, 0.3^2));
* pairwise interaction: ``b_pjk = 0.1 * u_jk.h_p / |u_jk|`` (marginally N(0, 0.1^2));
* log speedup of mask m: ``LS(m) = sum_{j in m} a_j + sum_{j<k in m} b_jk + N(0, 0.05^2)``;
  ``log t(m) = t0_p - LS(m)``;
* log counter rate: ``log x_{m,f} = (M h_p)_f + sum_{k in m} s_{p,k,f} + N(0, 0.3^2)`` with
  per-optimization shifts ``s_{p,k,f} = U_{k,f} + 0.3 (C_k h_p)_f / sqrt(8)``,
  ``U ~ N(0, 0.5^2)``; ``M`` is scaled so the marginal of ``log x`` is about N(0, 1.5^2)
  (the "log-normal(0, 1.5) with a per-mask additive shift" of the workloads);
* raw counters ``X = x * cycles`` with ``cycles = exp(log t + 20 + N(0, 0.02^2))`` when a
  cycle column is requested, else ``X = x``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence, Union

import numpy as np

GEN_VERSION = "gen/v1"
N_OPT = 6
N_MASK = 1 << N_OPT
LATENT = 8

IntOrRange = Union[int, Sequence[int]]


@dataclass
class ProgramBatch:
    """A ragged batch of programs.

    Program ``p`` owns rows ``row_offsets[p] .. row_offsets[p+1]-1`` (its versions, at most
    64); its counter block starts at element ``x_offsets[p]`` of ``X`` and is row-major
    ``[V_p, F_p]`` with ``F_p = feat_width[p]``.
    """

    X: np.ndarray              # flat float32/float64 raw counters
    x_offsets: np.ndarray      # int64 [P]
    row_offsets: np.ndarray    # int64 [P+1]
    feat_width: np.ndarray     # int32 [P]
    masks: np.ndarray          # uint8 [R] 6-bit optimization mask per version
    log_time: np.ndarray       # float64 [R]
    cycles: Optional[np.ndarray]  # float64 [R] or None
    meta: dict = field(default_factory=dict)

    @property
    def n_programs(self) -> int:
        return int(self.feat_width.shape[0])

    @property
    def n_rows(self) -> int:
        return int(self.row_offsets[-1])

    def versions(self, p: int) -> int:
        return int(self.row_offsets[p + 1] - self.row_offsets[p])

    def program_X(self, p: int) -> np.ndarray:
        V, F = self.versions(p), int(self.feat_width[p])
        o = int(self.x_offsets[p])
        return self.X[o:o + V * F].reshape(V, F)

    def program_rows(self, p: int) -> slice:
        return slice(int(self.row_offsets[p]), int(self.row_offsets[p + 1]))


def _pick(rng: np.random.Generator, spec: IntOrRange, n: int) -> np.ndarray:
    """Integers: a fixed value, a (lo, hi) inclusive uniform range, or a set to choose from."""
    if isinstance(spec, (int, np.integer)):
        return np.full(n, int(spec), dtype=np.int64)
    spec = list(spec)
    if len(spec) == 2 and spec[0] <= spec[1] and not isinstance(spec, set):
        return rng.integers(spec[0], spec[1] + 1, size=n).astype(np.int64)
    raise ValueError("use an int or a (lo, hi) pair; for a choice set call with choices=")


def make_batch(n_programs: int,
               versions: IntOrRange = 64,
               feat: IntOrRange = 96,
               feat_choices: Optional[Sequence[int]] = None,
               dtype=np.float64,
               seed: int = 0,
               with_cycles: bool = True,
               label_noise: float = 0.05,
               feat_noise: float = 0.3,
               mixing_kappa: Optional[float] = None) -> ProgramBatch:
    """Draw ``n_programs`` programs (recipe in the module docstring).

    ``versions``: versions per program (int, or inclusive (lo, hi) range; subsets of the
    64 masks drawn without replacement, all 64 when V=64).  ``feat`` / ``feat_choices``:
    feature width per program.  ``mixing_kappa``: if given, each program's log-features
    are mixed by ``Q diag(s) Q^T`` (one random orthogonal ``Q`` per width, ``s`` log-spaced
    from 1 down to ``1/sqrt(kappa)`` over the leading directions) to make counters
    correlated and the Gram matrices ill-conditioned.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    P = int(n_programs)
    Vs = _pick(rng, versions, P)
    if np.any(Vs < 1) or np.any(Vs > N_MASK):
        raise ValueError("versions per program must lie in 1..64")
    if feat_choices is not None:
        Fs = rng.choice(np.asarray(feat_choices, dtype=np.int64), size=P)
    else:
        Fs = _pick(rng, feat, P)

    # Global (workload-level) structure shared by all programs.
    w = rng.standard_normal((N_OPT, LATENT))
    u = rng.standard_normal((N_OPT, N_OPT, LATENT))
    Fmax = int(Fs.max())
    U = 0.5 * rng.standard_normal((N_OPT, Fmax))
    C = rng.standard_normal((N_OPT, Fmax, LATENT))
    sM = np.sqrt(max(2.25 - 3.0 * (0.25 + 0.09 * 1.0) - feat_noise ** 2, 0.1) / LATENT)
    M = sM * rng.standard_normal((Fmax, LATENT))
    mixers = {}

    X_parts, masks_parts, lt_parts, cyc_parts = [], [], [], []
    x_off = np.zeros(P, dtype=np.int64)
    row_off = np.zeros(P + 1, dtype=np.int64)
    pos = 0
    all_masks = np.arange(N_MASK, dtype=np.int64)
    pop = np.array([bin(m).count("1") for m in range(N_MASK)])
    bits = ((all_masks[:, None] >> np.arange(N_OPT)[None, :]) & 1).astype(np.float64)  # [64,6]
    for p in range(P):
        V, F = int(Vs[p]), int(Fs[p])
        h = rng.standard_normal(LATENT)
        a = 0.3 * (w @ h) / np.linalg.norm(w, axis=1)
        b = 0.1 * (u @ h) / np.linalg.norm(u, axis=2)
        b = np.triu(b, 1)
        if V == N_MASK:
            ms = all_masks.copy()
        else:
            ms = np.sort(rng.choice(N_MASK, size=V, replace=False)).astype(np.int64)
        mb = bits[ms]                                           # [V,6]
        ls = mb @ a + np.einsum("vj,jk,vk->v", mb, b, mb)
        ls = ls + label_noise * rng.standard_normal(V)
        t0 = rng.standard_normal()
        log_t = t0 - ls
        shift = U[:, :F] + 0.3 * np.einsum("kfl,l->kf", C[:, :F, :], h) / np.sqrt(LATENT)
        logx = (M[:F] @ h)[None, :] + mb @ shift + feat_noise * rng.standard_normal((V, F))
        if mixing_kappa is not None:
            key = F
            if key not in mixers:
                Q, _ = np.linalg.qr(rng.standard_normal((F, F)))
                r = min(F, 64)
                s = np.full(F, 1.0 / np.sqrt(mixing_kappa))
                s[:r] = np.logspace(0.0, -0.5 * np.log10(mixing_kappa), r)
                mixers[key] = (Q * s[None, :]) @ Q.T
            logx = logx @ mixers[key]
        x = np.exp(logx)
        if with_cycles:
            cyc = np.exp(log_t + 20.0 + 0.02 * rng.standard_normal(V))
            Xp = x * cyc[:, None]
            cyc_parts.append(cyc)
        else:
            Xp = x
        x_off[p] = pos
        pos += V * F
        row_off[p + 1] = row_off[p] + V
        X_parts.append(Xp.reshape(-1))
        masks_parts.append(ms.astype(np.uint8))
        lt_parts.append(log_t)
    del pop
    X = np.concatenate(X_parts).astype(dtype)
    return ProgramBatch(
        X=X, x_offsets=x_off, row_offsets=row_off, feat_width=Fs.astype(np.int32),
        masks=np.concatenate(masks_parts), log_time=np.concatenate(lt_parts).astype(np.float64),
        cycles=(np.concatenate(cyc_parts).astype(np.float64) if with_cycles else None),
        meta=dict(gen=GEN_VERSION, seed=seed, n_programs=P, mixing_kappa=mixing_kappa),
    )


@dataclass
class Splits:
    """Train/test splits: program ``p`` owns splits ``split_offsets[p] .. split_offsets[p+1]-1``;
    split ``i`` trains on the version slots whose bit is set in ``train_masks[i]`` (bit ``r``
    = the program's ``r``-th row) and tests on the others."""

    split_offsets: np.ndarray  # int64 [P+1]
    train_masks: np.ndarray    # uint64 [S]

    @property
    def n_splits(self) -> int:
        return int(self.train_masks.shape[0])


def make_splits(batch: ProgramBatch, kind: str = "half", n_splits: int = 16,
                seed: int = 0) -> Splits:
    """``kind``: ``"half"`` (random train subsets of exactly floor(V/2) versions, ``n_splits``
    per program), ``"lovo"`` (leave one version out: V splits per program), ``"all"`` (one
    split that trains on every version), or ``"frac"`` (each version in train with prob. 1/2)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    P = batch.n_programs
    offs = np.zeros(P + 1, dtype=np.int64)
    out = []
    for p in range(P):
        V = batch.versions(p)
        full = (1 << V) - 1 if V < 64 else (1 << 64) - 1
        if kind == "lovo":
            ms = [full & ~(1 << r) for r in range(V)]
        elif kind == "all":
            ms = [full]
        elif kind == "half":
            k = V // 2
            ms = []
            for _ in range(n_splits):
                sel = rng.choice(V, size=k, replace=False)
                m = 0
                for r in sel:
                    m |= 1 << int(r)
                ms.append(m)
        elif kind == "frac":
            ms = []
            for _ in range(n_splits):
                sel = np.nonzero(rng.random(V) < 0.5)[0]
                m = 0
                for r in sel:
                    m |= 1 << int(r)
                ms.append(m)
        else:
            raise ValueError(kind)
        offs[p + 1] = offs[p] + len(ms)
        out.extend(ms)
    return Splits(split_offsets=offs, train_masks=np.array(out, dtype=np.uint64))


def make_half_splits_fast(batch: ProgramBatch, n_splits: int, seed: int = 0) -> Splits:
    """Vectorised ``kind="half"`` for large workloads (same distribution, different stream)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0xBA7C4))
    P = batch.n_programs
    offs = np.arange(P + 1, dtype=np.int64) * n_splits
    tm = np.zeros(P * n_splits, dtype=np.uint64)
    for p in range(P):
        V = batch.versions(p)
        k = V // 2
        keys = rng.random((n_splits, V))
        sel = np.argsort(keys, axis=1)[:, :k]
        bitsv = np.zeros((n_splits, V), dtype=bool)
        np.put_along_axis(bitsv, sel, True, axis=1)
        weights = (np.uint64(1) << np.arange(V, dtype=np.uint64))
        tm[p * n_splits:(p + 1) * n_splits] = (bitsv.astype(np.uint64) * weights[None, :]).sum(
            axis=1, dtype=np.uint64)
    return Splits(split_offsets=offs, train_masks=tm)


def make_batch_fast(n_programs: int, versions: IntOrRange = 64, feat: int = 256,
                    feat_choices: Optional[Sequence[int]] = None, dtype=np.float32, seed: int = 0,
                    with_cycles: bool = True, label_noise: float = 0.05, feat_noise: float = 0.3,
                    chunk: int = 512) -> ProgramBatch:
    """The recipe of ``make_batch`` drawn in vectorised chunks of programs (for batches of
    thousands of programs).  Same distribution, different random stream."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0xFA57))
    P = int(n_programs)
    Vs = _pick(rng, versions, P)
    if feat_choices is not None:
        Fs = rng.choice(np.asarray(feat_choices, dtype=np.int64), size=P)
    else:
        Fs = np.full(P, int(feat), dtype=np.int64)
    w = rng.standard_normal((N_OPT, LATENT))
    u = rng.standard_normal((N_OPT, N_OPT, LATENT))
    Fmax = int(Fs.max())
    U = (0.5 * rng.standard_normal((N_OPT, Fmax))).astype(np.float32)
    Cm = rng.standard_normal((N_OPT, Fmax, LATENT)).astype(np.float32)
    sM = np.sqrt(max(2.25 - 3.0 * (0.25 + 0.09 * 1.0) - feat_noise ** 2, 0.1) / LATENT)
    M = (sM * rng.standard_normal((Fmax, LATENT))).astype(np.float32)
    all_masks = np.arange(N_MASK)
    bits = ((all_masks[:, None] >> np.arange(N_OPT)[None, :]) & 1).astype(np.float32)
    wn = w / np.linalg.norm(w, axis=1, keepdims=True)
    un = u / np.linalg.norm(u, axis=2, keepdims=True)
    row_off = np.zeros(P + 1, dtype=np.int64)
    row_off[1:] = np.cumsum(Vs)
    x_off = np.zeros(P, dtype=np.int64)
    x_off[1:] = np.cumsum(Vs * Fs)[:-1]
    X = np.empty(int((Vs * Fs).sum()), dtype=dtype)
    masks = np.empty(int(row_off[-1]), dtype=np.uint8)
    log_time = np.empty(int(row_off[-1]), dtype=np.float64)
    cycles = np.empty(int(row_off[-1]), dtype=np.float64) if with_cycles else None
    for F in np.unique(Fs):
        idx = np.nonzero(Fs == F)[0]
        for c0 in range(0, len(idx), chunk):
            ps = idx[c0:c0 + chunk]
            G = len(ps)
            h = rng.standard_normal((G, LATENT))
            a = 0.3 * h @ wn.T                                            # [G,6]
            b = 0.1 * np.einsum("jkl,gl->gjk", un, h)
            b = np.triu(b, 1) if b.ndim == 2 else b * np.triu(np.ones((N_OPT, N_OPT)), 1)[None]
            keys = rng.random((G, N_MASK))
            order = np.argsort(keys, axis=1)
            t0 = rng.standard_normal(G)
            shift = U[None, :, :F] + 0.3 * (Cm[:, :F, :].reshape(-1, LATENT) @ h.astype(np.float32).T).T.reshape(
                G, N_OPT, F) / np.sqrt(LATENT)
            base = (h.astype(np.float32) @ M[:F].T)                         # [G,F]
            if np.all(Vs[ps] == N_MASK):     # every program owns all 64 masks: fully vectorised
                mb = bits                                                  # [64,6]
                ls = a @ mb.T + np.einsum("vj,gjk,vk->gv", mb, b, mb)
                ls = ls + label_noise * rng.standard_normal((G, N_MASK))
                lt = t0[:, None] - ls                                      # [G,64]
                logx = base[:, None, :] + np.matmul(mb[None], shift)
                logx = logx + feat_noise * rng.standard_normal((G, N_MASK, F), dtype=np.float32)
                xx = np.exp(logx)
                if with_cycles:
                    cyc = np.exp(lt + 20.0 + 0.02 * rng.standard_normal((G, N_MASK)))
                    xx = xx * cyc[:, :, None].astype(np.float32)
                for gi, p in enumerate(ps):
                    r0 = int(row_off[p])
                    X[int(x_off[p]):int(x_off[p]) + N_MASK * F] = xx[gi].reshape(-1)
                    masks[r0:r0 + N_MASK] = all_masks.astype(np.uint8)
                    log_time[r0:r0 + N_MASK] = lt[gi]
                    if with_cycles:
                        cycles[r0:r0 + N_MASK] = cyc[gi]
                continue
            for gi, p in enumerate(ps):
                V = int(Vs[p])
                ms = all_masks.copy() if V == N_MASK else np.sort(order[gi, :V])
                mb = bits[ms]                                             # [V,6]
                ls = mb @ a[gi] + np.einsum("vj,jk,vk->v", mb, b[gi], mb) + label_noise * rng.standard_normal(V)
                lt = t0[gi] - ls
                logx = base[gi][None, :] + mb @ shift[gi] + feat_noise * rng.standard_normal((V, F), dtype=np.float32)
                xx = np.exp(logx)
                r0 = int(row_off[p])
                if with_cycles:
                    cyc = np.exp(lt + 20.0 + 0.02 * rng.standard_normal(V))
                    xx = xx * cyc[:, None]
                    cycles[r0:r0 + V] = cyc
                X[int(x_off[p]):int(x_off[p]) + V * F] = xx.reshape(-1).astype(dtype)
                masks[r0:r0 + V] = ms.astype(np.uint8)
                log_time[r0:r0 + V] = lt
    return ProgramBatch(X=X, x_offsets=x_off, row_offsets=row_off, feat_width=Fs.astype(np.int32),
                        masks=masks, log_time=log_time, cycles=cycles,
                        meta=dict(gen=GEN_VERSION + "-fast", seed=seed, n_programs=P))


def apply_mixing(batch: ProgramBatch, kappa: float, seed: int = 0) -> ProgramBatch:
    """A copy of a uniform-width batch whose log counter rates are mixed by Q diag(s) Q^T
    (Q random orthogonal, s log-spaced from 1 to 1/sqrt(kappa) over the first 64 directions,
    1/sqrt(kappa) after), making counters correlated and the Gram matrices ill-conditioned.
    The cycle normalisation is kept: X' = exp(log(X / c) @ mix) * c."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x31C5))
    F = int(batch.feat_width[0])
    assert np.all(batch.feat_width == F), "uniform feature width only"
    Q, _ = np.linalg.qr(rng.standard_normal((F, F)))
    r = min(F, 64)
    sv = np.full(F, 1.0 / np.sqrt(kappa))
    sv[:r] = np.logspace(0.0, -0.5 * np.log10(kappa), r)
    mix = (Q * sv[None, :]) @ Q.T
    c = batch.cycles if batch.cycles is not None else np.ones(batch.n_rows)
    L = np.log(batch.X.reshape(batch.n_rows, F).astype(np.float64) / c[:, None])
    X2 = np.exp(L @ mix) * c[:, None]
    out = ProgramBatch(X=X2.reshape(-1).astype(batch.X.dtype), x_offsets=batch.x_offsets.copy(),
                       row_offsets=batch.row_offsets.copy(), feat_width=batch.feat_width.copy(),
                       masks=batch.masks.copy(), log_time=batch.log_time.copy(),
                       cycles=None if batch.cycles is None else batch.cycles.copy(),
                       meta=dict(batch.meta, mixing_kappa=kappa))
    return out


def make_complementary_halves(batch: ProgramBatch, seed: int = 0) -> Splits:
    """Two splits per program: a random half of its versions and the other half, so that every
    version is a test row exactly once (its prediction comes from a fit on the other half)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0xC0FE))
    P = batch.n_programs
    offs = np.arange(P + 1, dtype=np.int64) * 2
    tm = np.zeros(2 * P, dtype=np.uint64)
    for p in range(P):
        V = batch.versions(p)
        sel = np.argsort(rng.random(V))[:V // 2]
        m = 0
        for r in sel:
            m |= 1 << int(r)
        full = (1 << V) - 1 if V < 64 else (1 << 64) - 1
        tm[2 * p] = np.uint64(m)
        tm[2 * p + 1] = np.uint64(full & ~m)
    return Splits(split_offsets=offs, train_masks=tm)


def make_vectors(n: int, F: int = 256, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """Standard-normal stand-ins for standardized feature vectors (surrogate inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x7EC7))
    return rng.standard_normal((n, F)).astype(dtype)


# ---------------------------------------------------------------------- Table 2 protocols
# Two subject codes, an irregular one ("BH", six inputs) and a regular one ("NB", four inputs),
# each profiled three times per input (Sec. 5, Table 1).  Optimizations 4 and 5 (FTZ and RSQRT
# in the paper's numbering) are the only ones the two codes share (Sec. 6.2); bits 0-3 stand
# for different source changes in each code.
CODES = (("BH", 6), ("NB", 4))
SHARED_OPTS = 0b110000


def make_runs(codes=CODES, runs: int = 3, feat: int = 96, dtype=np.float64, seed: int = 0,
              with_cycles: bool = True, input_spread: float = 0.4, version_noise: float = 0.3,
              run_noise: float = 0.05, label_noise: float = 0.05, run_label_noise: float = 0.01,
              code_similarity: float = 0.8) -> ProgramBatch:
    """One program entry per (code, input, run), all 64 versions, in that nesting order; the
    list of (code, input, run) is ``meta["index"]``.

    Recipe (one PCG64 stream): per code a latent state ``h_c = rho h_0 + sqrt(1 - rho^2) e_c``
    (``h_0, e_c ~ N(0, I_8)``, ``rho = code_similarity``: the codes are two GPU n-body
    programs, alike in part) and, for its own
    optimizations (bits 0-3), its own effect directions and counter shifts; the shared ones
    (bits 4, 5) use directions and shifts common to both codes.  Input i moves the state,
    ``h_ci = h_c + input_spread * N(0, I_8)``, and scales the effects by
    ``0.6 + 0.4 i / (n_inputs - 1)`` (larger inputs, clearer effects).  A version's log
    speedup and log counter rates get a per-input draw (``label_noise``, ``version_noise``)
    that every run of that input repeats, and each run adds its own small noise
    (``run_label_noise``, ``run_noise``).  Otherwise as ``make_batch``: main effects
    ``0.3 w_j.h / |w_j|``, interactions ``0.1 u_jk.h / |u_jk|``, counter shifts
    ``U_{k,f} + 0.3 (C_k h)_f / sqrt(8)``, cycles ``exp(log t + 20 + N(0, 0.02^2))``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    F = int(feat)
    w_sh = rng.standard_normal((N_OPT, LATENT))
    u_sh = rng.standard_normal((N_OPT, N_OPT, LATENT))
    U_sh = 0.5 * rng.standard_normal((N_OPT, F))
    C_sh = rng.standard_normal((N_OPT, F, LATENT))
    sM = np.sqrt(max(2.25 - 3.0 * (0.25 + 0.09) - version_noise ** 2, 0.1) / LATENT)
    M = sM * rng.standard_normal((F, LATENT))
    all_masks = np.arange(N_MASK, dtype=np.int64)
    mb = ((all_masks[:, None] >> np.arange(N_OPT)[None, :]) & 1).astype(np.float64)   # [64,6]
    own = np.arange(N_OPT) < 4
    h_0 = rng.standard_normal(LATENT)
    X_parts, m_parts, lt_parts, cyc_parts, index = [], [], [], [], []
    for code, n_inputs in codes:
        h_c = code_similarity * h_0 + np.sqrt(1.0 - code_similarity ** 2) * rng.standard_normal(LATENT)
        w = np.where(own[:, None], rng.standard_normal((N_OPT, LATENT)), w_sh)
        u = np.where(own[:, None, None] | own[None, :, None], rng.standard_normal((N_OPT, N_OPT, LATENT)), u_sh)
        U = np.where(own[:, None], 0.5 * rng.standard_normal((N_OPT, F)), U_sh)
        Cc = np.where(own[:, None, None], rng.standard_normal((N_OPT, F, LATENT)), C_sh)
        t0_c = rng.standard_normal()
        for i in range(n_inputs):
            h = h_c + input_spread * rng.standard_normal(LATENT)
            scale = 0.6 + 0.4 * i / max(n_inputs - 1, 1)
            a = scale * 0.3 * (w @ h) / np.linalg.norm(w, axis=1)
            b = np.triu(scale * 0.1 * (u @ h) / np.linalg.norm(u, axis=2), 1)
            ls_in = mb @ a + np.einsum("vj,jk,vk->v", mb, b, mb) + label_noise * rng.standard_normal(N_MASK)
            shift = U + 0.3 * np.einsum("kfl,l->kf", Cc, h) / np.sqrt(LATENT)
            logx_in = (M @ h)[None, :] + mb @ shift + version_noise * rng.standard_normal((N_MASK, F))
            t0 = t0_c + 0.7 * i
            for r in range(runs):
                ls = ls_in + run_label_noise * rng.standard_normal(N_MASK)
                log_t = t0 - ls
                x = np.exp(logx_in + run_noise * rng.standard_normal((N_MASK, F)))
                if with_cycles:
                    cyc = np.exp(log_t + 20.0 + 0.02 * rng.standard_normal(N_MASK))
                    x = x * cyc[:, None]
                    cyc_parts.append(cyc)
                X_parts.append(x.reshape(-1))
                m_parts.append(all_masks.astype(np.uint8))
                lt_parts.append(log_t)
                index.append((code, i, r))
    P = len(index)
    return ProgramBatch(
        X=np.concatenate(X_parts).astype(dtype), x_offsets=np.arange(P, dtype=np.int64) * N_MASK * F,
        row_offsets=np.arange(P + 1, dtype=np.int64) * N_MASK, feat_width=np.full(P, F, dtype=np.int32),
        masks=np.concatenate(m_parts), log_time=np.concatenate(lt_parts).astype(np.float64),
        cycles=(np.concatenate(cyc_parts).astype(np.float64) if with_cycles else None),
        meta=dict(gen=GEN_VERSION + "/runs", seed=seed, index=index, runs=runs, codes=tuple(codes)))


def take_programs(batch: ProgramBatch, programs: Sequence[int]) -> ProgramBatch:
    """A new batch holding copies of the given programs, in the given order."""
    xs, ms, lts, cys, xo, ro, fw = [], [], [], [], [], [0], []
    pos = 0
    for p in programs:
        V, F = batch.versions(p), int(batch.feat_width[p])
        rows = batch.program_rows(p)
        xs.append(batch.program_X(p).reshape(-1))
        ms.append(batch.masks[rows])
        lts.append(batch.log_time[rows])
        if batch.cycles is not None:
            cys.append(batch.cycles[rows])
        xo.append(pos)
        pos += V * F
        ro.append(ro[-1] + V)
        fw.append(F)
    return ProgramBatch(
        X=np.concatenate(xs), x_offsets=np.asarray(xo, dtype=np.int64), row_offsets=np.asarray(ro, dtype=np.int64),
        feat_width=np.asarray(fw, dtype=np.int32), masks=np.concatenate(ms), log_time=np.concatenate(lts),
        cycles=np.concatenate(cys) if batch.cycles is not None else None, meta=dict(batch.meta, taken=list(programs)))


@dataclass
class TransferProblems:
    """The problems of one Table 2 experiment: problem q trains on runs
    ``groups[q] .. groups[q+1]-1`` of ``train`` and tests on program q of ``test``."""
    experiment: int
    train: ProgramBatch
    test: ProgramBatch
    groups: np.ndarray          # int64 [Q+1]
    opt_mask: int
    pairs: list                 # (train (code, input, runs), test (code, input, run)) per problem


def table2_problems(runs: ProgramBatch, experiment: int, code: str = "BH") -> TransferProblems:
    """Table 2's six experiments on a batch from ``make_runs`` (Sec. 5 / 6); experiments 1-4
    use the runs of ``code`` (BH in the paper; any code of the batch, e.g. a measured NB):
    1. one run of a BH input trains; every run of that input (its own included) is tested;
    2. as 1, but only the other runs are tested;
    3. two runs of a BH input train; the third is tested;
    4. all runs of a BH input train; every run of every other BH input is tested;
    5. all runs of a BH input train; every run of every NB input is tested (FTZ and RSQRT only);
    6. all runs of an NB input train; every run of every BH input is tested (FTZ and RSQRT only)."""
    idx = {key: p for p, key in enumerate(runs.meta["index"])}
    n_runs = runs.meta["runs"]
    n_in = dict(runs.meta["codes"])
    probs = []          # (list of training programs, test program, description)
    if experiment in (1, 2):
        for i in range(n_in[code]):
            for r in range(n_runs):
                for r2 in range(n_runs):
                    if experiment == 2 and r2 == r:
                        continue
                    probs.append(([idx[(code, i, r)]], idx[(code, i, r2)], ((code, i, (r,)), (code, i, r2))))
    elif experiment == 3:
        for i in range(n_in[code]):
            for r2 in range(n_runs):
                tr = tuple(r for r in range(n_runs) if r != r2)
                probs.append(([idx[(code, i, r)] for r in tr], idx[(code, i, r2)], ((code, i, tr), (code, i, r2))))
    elif experiment in (4, 5, 6):
        src, dst = {4: (code, code), 5: ("BH", "NB"), 6: ("NB", "BH")}[experiment]
        for i in range(n_in[src]):
            tr = tuple(range(n_runs))
            for i2 in range(n_in[dst]):
                if experiment == 4 and i2 == i:
                    continue
                for r2 in range(n_runs):
                    probs.append(([idx[(src, i, r)] for r in tr], idx[(dst, i2, r2)],
                                  ((src, i, tr), (dst, i2, r2))))
    else:
        raise ValueError("experiment must be 1..6")
    train_list = [p for tr, _, _ in probs for p in tr]
    groups = np.zeros(len(probs) + 1, dtype=np.int64)
    groups[1:] = np.cumsum([len(tr) for tr, _, _ in probs])
    return TransferProblems(
        experiment=experiment, train=take_programs(runs, train_list),
        test=take_programs(runs, [te for _, te, _ in probs]), groups=groups,
        opt_mask=SHARED_OPTS if experiment in (5, 6) else 0x3F, pairs=[d for _, _, d in probs])


def init_mlp_params(seed: int = 0, dims=(256, 512, 512, 6)):
    """Seeded initial weights of the surrogate MLP: W_i [fan_out][fan_in] and b_i [fan_out]
    uniform in (-1/sqrt(fan_in), 1/sqrt(fan_in)).  Random inputs, no arithmetic of the method."""
    import math
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5A5A))
    p = {}
    for i in range(3):
        fi, fo = dims[i], dims[i + 1]
        s = 1.0 / math.sqrt(fi)
        p[f"W{i + 1}"] = rng.uniform(-s, s, size=(fo, fi))
        p[f"b{i + 1}"] = rng.uniform(-s, s, size=fo)
    return p


def with_anomalous_versions(batch: ProgramBatch, frac_programs: float, per_program: int = 3,
                            factor: float = float(np.exp(4.0)), seed: int = 0):
    """A copy of ``batch`` in which a random ``frac_programs`` of the programs have
    ``per_program`` random versions whose every counter is multiplied by ``factor`` (profiles
    unlike the rest of their program: out-of-distribution rows for a learned predictor).
    Returns (batch, sorted array of the affected programs)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0xA70A))
    P = batch.n_programs
    progs = np.sort(rng.choice(P, size=max(1, int(round(frac_programs * P))), replace=False))
    X = batch.X.copy()
    for p in progs:
        V, F, o = batch.versions(int(p)), int(batch.feat_width[p]), int(batch.x_offsets[p])
        for v in rng.choice(V, size=min(per_program, V), replace=False):
            X[o + int(v) * F:o + (int(v) + 1) * F] *= X.dtype.type(factor)
    out = ProgramBatch(X=X, x_offsets=batch.x_offsets.copy(), row_offsets=batch.row_offsets.copy(),
                       feat_width=batch.feat_width.copy(), masks=batch.masks.copy(),
                       log_time=batch.log_time.copy(),
                       cycles=None if batch.cycles is None else batch.cycles.copy(), meta=dict(batch.meta))
    return out, progs
