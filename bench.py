#!/usr/bin/env python
"""Ranked recommendations per second of the batched cross-validation pass.

Workload (the batched-CV configuration): 64 programs, each with 16..64 versions (random
subsets of the 64 optimization masks), 256 FP32 counter features per version (synthetic,
log-normal(0, 1.5) with per-mask shifts, generator gen/v1, seed 0), 4096 random 50/50
train/test splits per program (262,144 splits, about 1.57 M ridge fits), lambda 1e-3,
top-3, threshold 1.05.  A step = one whole pass: standardize, Gram, test-row planning and
the fused fit / predict / rank / score kernel, all in the sm_103a library.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU reference on the
host cores instead (bounded samples of the same workload).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ranked recommendations/sec (CV-split fits+predicts) vs plain GPU form at equal accuracy"
UNIT = "recommendations/s"
WORKLOAD = "batched_cv: 64 programs x U{16..64} versions x 256 f32 features, 4096 half splits/program"
# kernels of one step: standardize, Gram, row planning (count, block sums, finish), pairs,
# plan, bucket, the Gram diagonal + lambda, three solvers, rank pass
LAUNCHES_PER_STEP = 13
CFG = dict(programs=64, versions=(16, 64), feat=256, splits=4096, lam=1e-3, k=3, tau=1.05, seed=0)
FP64_PEAK_NOMINAL_GFLOPS = 152 * 4 * 2.07   # 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz


def source_sha():
    """sha256 prefix of the sources of the profiled step kernels (the fit/predict/rank file and
    the ranking header it includes)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("k_fit.cu", "rank_row.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1910_07776_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(stage):
    """DRAM bytes per step of a stage from the committed ncu summary, or None when the kernel
    sources have changed since the capture (their sha256 prefix is recorded in the summary)."""
    try:
        txt = open(os.path.join(ROOT, "profiles", "batched_cv_kernels.md")).read()
        sha = source_sha()
    except OSError:
        return None
    if f"source_sha256_prefix k_fit.cu+rank_row.cuh = {sha}" not in txt:
        return None
    for line in txt.splitlines():
        if line.startswith(f"traffic_bytes_per_step {stage} = "):
            return float(line.split("=")[1].split()[0])
    return None


def aggregate_over_ranks(total_ms, recs, world, device):
    """Weak scaling: every rank times its own batch; the job's time is the slowest rank's and
    its work is the sum of all ranks' recommendations (no data-path collective)."""
    if world <= 1:
        return float(total_ms), float(recs)
    import torch
    import torch.distributed as dist
    dist.barrier()
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    r = torch.tensor([float(recs)], dtype=torch.float64, device=device)
    dist.all_reduce(r)
    return float(t.item()), float(r.item())


def measured_hbm_peak():
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the machine's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


def make_inputs(seed, programs=None):
    from paper_1910_07776_gb300 import synth
    b = synth.make_batch(programs or CFG["programs"], versions=CFG["versions"], feat=CFG["feat"],
                         dtype=np.float32, seed=seed)
    s = synth.make_half_splits_fast(b, CFG["splits"], seed=seed)
    return b, s


def rank_inputs(rank, world):
    """This rank's share of the job.  One GPU: the whole batched-CV workload.  N GPUs (weak
    scaling): the job is N times the workload (64 N programs), split over the ranks by the
    longest-processing-time rule on each program's estimated work, so every rank holds about
    one workload's worth of fits and no data moves between ranks."""
    if world <= 1:
        return make_inputs(CFG["seed"])
    from paper_1910_07776_gb300 import shard
    b, s = make_inputs(CFG["seed"], CFG["programs"] * world)
    mine = shard.lpt_partition(shard.program_costs(b, s), world)[rank]
    return shard.shard(b, s, mine)


def fit_flops(n):
    """FP64 operations of one ridge fit of n >= 2 pairs by the square-root-free LDL^T route
    the solvers take (an FMA counts 2, a multiply 1, a reciprocal 1):
      factorisation   (n-1)n(n+1)/6 FMAs, n(n-1)/2 multiplies (L = c / d), n reciprocals;
      two forward solves with the unit lower factor   n(n-1) FMAs;
      num, den = t_1^T D^-1 (t_y, t_1)   n multiplies, 2n FMAs; b   1 multiply, 1 reciprocal;
      D^-1 (t_y - b t_1)   n FMAs, n multiplies;  backward solve   n(n-1)/2 FMAs.
    Total (n-1)n(n+1)/3 + 3.5 n(n-1) + 9n + 2.  Each prediction adds n FMAs (2n flops)."""
    n = np.asarray(n, dtype=np.float64)
    return (n - 1) * n * (n + 1) / 3 + 3.5 * n * (n - 1) + 9 * n + 2


def algorithmic_work(batch, splits, k=3, nreg=10):
    """Algorithmic work of the fit/predict stages, counted from the definitions.
    FP64 flops: per fit with n pairs fit_flops(n); per prediction 2 n.  A fit of one pair
    needs no arithmetic (alpha = 0, b = y: every prediction is b), so it counts zero flops.
    Fits with n <= nreg (and their predictions) belong to the register solvers, larger ones
    to the shared-memory solver.  Rank stage bytes: per test row the version mask (1 B), its
    scoring summary (4 B), the code word (4 B) and k reported values (8 B each), plus 8 B per
    prediction read."""
    out = {"solve_small": 0.0, "solve_large": 0.0, "rows": 0, "preds": 0}
    for p in range(batch.n_programs):
        rs_ = batch.program_rows(p)
        m = batch.masks[rs_].astype(np.int64)
        V = len(m)
        slot = {int(x): i for i, x in enumerate(m)}
        T = splits.train_masks[splits.split_offsets[p]:splits.split_offsets[p + 1]].astype(np.uint64)
        full = np.uint64((1 << V) - 1) if V < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        test = (~T) & full
        x = test.copy()
        rows = np.zeros(x.shape, dtype=np.int64)
        for _ in range(V):
            rows += (x & np.uint64(1)).astype(np.int64)
            x = x >> np.uint64(1)
        out["rows"] += int(rows.sum())
        for j in range(6):
            pm = [(1 << v) | (1 << slot[int(m[v]) | (1 << j)]) for v in range(V)
                  if not (m[v] >> j) & 1 and (int(m[v]) | (1 << j)) in slot]
            if not pm:
                continue
            pm = np.array(pm, dtype=np.uint64)
            n = ((T[:, None] & pm[None, :]) == pm[None, :]).sum(axis=1).astype(np.float64)
            nomask = np.uint64(sum(1 << v for v in range(V) if not (m[v] >> j) & 1))
            x = test & nomask
            cnt = np.zeros(x.shape, dtype=np.float64)
            for _ in range(V):
                cnt += (x & np.uint64(1)).astype(np.float64)
                x = x >> np.uint64(1)
            fl = fit_flops(n) + 2 * n * cnt
            out["solve_small"] += float(np.sum(fl * (n >= 2) * (n <= nreg)))
            out["solve_large"] += float(np.sum(fl * (n > nreg)))
            out["preds"] += int(np.sum(cnt * (n > 0)))
    out["rank_bytes"] = float(out["rows"] * (1 + 4 + 4 + 8 * k) + 8 * out["preds"])
    # the other stages' minimum work: the standardization reads X and writes Z (FP64); the
    # Gram's upper triangle is V (V + 1) / 2 dot products of F features (2 flops each); the
    # row planning reads each split's train mask once
    V = np.diff(batch.row_offsets).astype(np.float64)
    F = batch.feat_width.astype(np.float64)
    out["std_bytes"] = float(np.sum(V * F) * (batch.X.dtype.itemsize + 8))
    out["gram_flops"] = float(np.sum(V * (V + 1) / 2 * F * 2))
    out["mask_bytes"] = float(len(splits.train_masks) * 8)
    return out


class ClockSampler:
    """SM clock, power and clock-event reasons of one GPU, sampled every millisecond through
    NVML (read-only queries of libnvidia-ml) on a background thread; nvidia-smi at 50 ms if
    NVML cannot be loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_s=0.001):
        self.gpu = gpu_index
        self.period = period_s
        self.samples = []          # (t, sm_mhz, max_mhz, power_w, reasons bitmask)
        self.marks = {}
        self.proc = None
        self.nvml = self._load_nvml()
        self._stop = threading.Event()

    def _load_nvml(self):
        import ctypes as C
        try:
            L = C.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() != 0:
                return None
            h = C.c_void_p()
            if L.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.gpu), C.byref(h)) != 0:
                return None
            reasons = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                L.nvmlDeviceGetCurrentClocksThrottleReasons
            return (C, L, h, reasons)
        except (OSError, AttributeError):
            return None

    def _poll_nvml(self):
        C, L, h, reasons = self.nvml
        sm, mx, mw, rs = C.c_uint(), C.c_uint(), C.c_uint(), C.c_ulonglong()
        L.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))
        while not self._stop.is_set():
            ok = L.nvmlDeviceGetClockInfo(h, 1, C.byref(sm)) == 0
            L.nvmlDeviceGetPowerUsage(h, C.byref(mw))
            reasons(h, C.byref(rs))
            if ok:
                self.samples.append((time.perf_counter(), float(sm.value), float(mx.value),
                                     mw.value / 1e3, int(rs.value)))
            time.sleep(self.period)

    def _read_smi(self):
        bits = [0x8, 0x40, 0x20, 0x4]
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                r = sum(b for b, v in zip(bits, f[5:9]) if v.lower() == "active")
                self.samples.append((time.perf_counter(), float(f[1]), float(f[2]), float(f[3]), r))
            except ValueError:
                continue

    def start(self):
        if self.nvml is not None:
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
        else:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits", "-lms", "50"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except FileNotFoundError:
                return
            self.t = threading.Thread(target=self._read_smi, daemon=True)
        self.t.start()
        t0 = time.time()                # the timed region starts once sampling runs
        while not self.samples and time.time() - t0 < 3.0:
            time.sleep(0.001)
        self.samples.clear()

    def mark(self, name):
        self.marks[name] = time.perf_counter()

    def stop(self):
        self._stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if getattr(self, "t", None) is not None:
            self.t.join(timeout=5)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": ["no clock samples"]}
        arr = list(self.samples)

        def summary(rows):
            sm = [r[1] for r in rows]
            rs_ = set()
            for r in rows:
                for bit, nm in self.REASONS.items():
                    if r[4] & bit:
                        rs_.add(nm)
            return {"sm_mhz": float(np.median(sm)) if sm else None, "samples": len(sm),
                    "reasons": sorted(rs_)}

        out = summary(arr)
        out["sm_max_mhz"] = float(max(r[2] for r in arr))
        out["power_w_max"] = float(max(r[3] for r in arr))
        out["source"] = "NVML, 1 ms" if self.nvml is not None else "nvidia-smi, 50 ms"
        if "timed_end" in self.marks:
            out["timed_region"] = summary([r for r in arr if r[0] <= self.marks["timed_end"]])
            out["seconds"] = arr[-1][0] - arr[0][0]
        return out


def cpu_reference_sample(batch, splits, target_s, seed=1):
    """Time the FP64 CPU reference on a random sample of splits (all host cores)."""
    import oracle
    from paper_1910_07776_gb300 import synth
    oracle.build()
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    rng = np.random.default_rng(seed)

    def run(nsplit):
        pick = np.sort(rng.choice(splits.n_splits, size=nsplit, replace=False))
        prog = np.searchsorted(splits.split_offsets, pick, side="right") - 1
        off = np.zeros(batch.n_programs + 1, dtype=np.int64)
        np.add.at(off, prog + 1, 1)
        off = np.cumsum(off)
        sub = synth.Splits(split_offsets=off, train_masks=splits.train_masks[pick])
        t0 = time.perf_counter()
        r = oracle.cv_batch(batch, sub, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"],
                            nthreads=threads, want_Z=False)
        dt = time.perf_counter() - t0
        return int(r.counters[0]), dt, nsplit

    run(threads)                                 # warms the library and the thread pool
    # random samples of growing size until about target_s of oracle time has been spent;
    # each sample's rate sizes the next one (the per-program standardization is a fixed
    # cost of every sample, so small samples overstate the time per split)
    rows = n = 0
    dt = 0.0
    chunks = 0
    nxt = 8 * threads
    while dt < 0.9 * target_s:
        r_, d_, n_ = run(int(min(splits.n_splits, max(threads, nxt))))
        rows, dt, n, chunks = rows + r_, dt + d_, n + n_, chunks + 1
        nxt = (target_s - dt) * n_ / max(d_, 1e-6)
    return dict(value=rows / dt, unit=UNIT, cores=threads, kind="oracle", seconds=dt,
                sample=f"{n} random splits of the {splits.n_splits} in {chunks} samples "
                       f"({rows} ranked rows), {dt:.1f} s of oracle wall time, FP64 primal normal "
                       f"equations, OpenMP over splits")


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    batch, splits = make_inputs(CFG["seed"])
    for _ in range(args.warmup):
        cpu_reference_sample(batch, splits, args.ref_step_seconds, seed=7)
    vals, cores, sample, secs = [], None, None, []
    for i in range(args.steps):
        c = cpu_reference_sample(batch, splits, args.ref_step_seconds, seed=100 + i)
        vals.append(c["value"])
        secs.append(c["seconds"])
        cores, sample = c["cores"], c["sample"]
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, **{k: (list(v_) if isinstance(v_, tuple) else v_) for k, v_ in CFG.items()}},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: " + sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=6.0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-ibk", action="store_true")
    ap.add_argument("--no-transfer", action="store_true")
    ap.add_argument("--no-lovo", action="store_true")
    ap.add_argument("--profile-gram", type=int, default=0, metavar="PROGRAMS",
                    help="a short run of the tensor-core Gram (BF16 hi/lo split) on this many programs x 64 "
                         "versions x 1024 FP64 features, each tile shape three times, and of the pooled "
                         "fit of the batched-CV workload's first 48 programs (for profiler captures)")
    ap.add_argument("--only-lovo", type=int, default=0, metavar="PROGRAMS",
                    help="time only the leave-one-version-out form on this many programs (for profiler "
                         "captures of its solver)")
    ap.add_argument("--surrogate-epochs", type=int, default=2)
    ap.add_argument("--profile-surrogate", action="store_true",
                    help="a short surrogate run for profiler captures of its tensor-core GEMMs: 16 training "
                         "steps of 8192 rows and one ranked inference of 131,072 rows (seeded random rows)")
    ap.add_argument("--only-step", action="store_true",
                    help="time the batched step only (no plain form, e2e, CPU baseline or FMA peak); "
                         "used for profiler captures")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.profile_surrogate:
        return profile_surrogate()

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1910_07776_gb300 import build as _b
    _b.build()
    from paper_1910_07776_gb300 import rs

    batch, splits = rank_inputs(rank, world)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = rs.Context(local, stream)
    if args.profile_gram:
        from paper_1910_07776_gb300 import synth
        b = synth.make_batch_fast(args.profile_gram, versions=64, feat=1024, dtype=np.float64, seed=21)
        db = rs.DeviceBatch.from_host(b, dev)
        zb = db.with_X(ctx.standardize(db))
        ws = ctx.workspace(ctx.cv_workspace_bytes(db, rs.DeviceSplits.from_host(synth.make_splits(b, "all"), dev, b)))
        K = torch.zeros(db.n_programs * 64 * 64, dtype=torch.float64, device=dev)
        for tile_n, ksplit in ((64, 1), (32, 1), (64, 3), (32, 3)):
            ctx.set_gram_tuning(1024, tile_n, ksplit)
            for _ in range(3):
                ctx.gram(zb, rs.RS_GRAM_BF16X3, K, ws)
        tr = synth.take_programs(batch, list(range(48)))
        dtr = rs.DeviceBatch.from_host(tr, dev)
        ztr = dtr.with_X(ctx.standardize(dtr))
        for _ in range(3):
            ctx.fit_pooled(ztr, None, lam=CFG["lam"], flags=rs.RS_REFINE_X)
        torch.cuda.synchronize()
        ctx.check_device_status()
        print(json.dumps({"profile_gram": args.profile_gram}), flush=True)
        ctx.close()
        return 0
    if args.only_lovo:
        flush = torch.empty(32 * 1024 * 1024, dtype=torch.int64, device=dev)
        print(json.dumps({"lovo_form": run_lovo(rs, ctx, dev, stream, flush, args, args.only_lovo)}), flush=True)
        ctx.close()
        return 0
    db = rs.DeviceBatch.from_host(batch, dev)
    ds = rs.DeviceSplits.from_host(splits, dev, batch)
    Z = torch.empty(db.x_elems, dtype=torch.float64, device=dev)
    zb = db.with_X(Z)
    K = torch.zeros(db.n_programs * 64 * 64, dtype=torch.float64, device=dev)
    ro = ctx.rec_offsets(db, ds)
    R = int(ro[-1].item())
    out = rs.alloc_outputs(R, ds.n_splits, CFG["k"], dev, pred_all=False)
    out.rec_offsets = ro
    # 256 MB (twice the L2) written between timed steps; as 8-byte words the fill runs at the
    # write bandwidth (37.5 us; 70 us as bytes)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.int64, device=dev)
    cws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    # the whole step (rs_cv_step: the planning on the context's second stream beside the
    # standardization and the Gram) captured once as a CUDA graph, one launch per step
    graph = ctx.cv_graph(db, ds, cws, out.rec_offsets, out.rec_code, lam=CFG["lam"], k=CFG["k"],
                         tau=CFG["tau"], rec_pred=out.rec_pred, counters=out.counters)

    def step():
        ev[0].record(stream)
        graph.launch()
        ev[1].record(stream)

    def eager_step():
        ev[0].record(stream)
        ctx.cv_step(db, ds, cws, out.rec_offsets, out.rec_code, lam=CFG["lam"], k=CFG["k"],
                    tau=CFG["tau"], rec_pred=out.rec_pred, counters=out.counters)
        ev[1].record(stream)

    def between():
        flush.fill_(1)   # evicts the 129 MB L2 between timed steps (not timed)
        out.counters.zero_()

    for _ in range(args.warmup):
        between()
        step()
    torch.cuda.synchronize()
    ctx.check_device_status()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_clk = time.perf_counter()
    tot = 0.0
    for _ in range(args.steps):
        between()
        step()
        torch.cuda.synchronize()
        tot += ev[0].elapsed_time(ev[1])
    torch.cuda.synchronize()
    clocks.mark("timed_end")
    # the same step keeps running until the clock record spans at least one second (a short
    # timed region alone would hold few samples); these steps are timed separately
    sus_ms, sus_n = 0.0, 0
    while time.perf_counter() - t_clk < 1.0:
        between()
        step()
        torch.cuda.synchronize()
        sus_ms += ev[0].elapsed_time(ev[1])
        sus_n += 1
    clk = clocks.stop()
    graph.close()
    clk["after_timed_region"] = {"steps": sus_n, "ms_per_step": sus_ms / sus_n if sus_n else None}
    tot, R_total = aggregate_over_ranks(tot, R, world, dev)
    ctx.check_device_status()
    ms_step = tot / args.steps
    value = R_total * args.steps / (tot / 1e3)
    if world > 1:                              # the job's accuracy counters: a sum over the ranks
        from paper_1910_07776_gb300 import shard
        shard.allreduce_counters(out.counters)
    cnt = out.counters.cpu().numpy().view(np.uint64).astype(np.float64)
    acc = {"sign_accuracy": cnt[3] / max(cnt[2], 1), "top1_hit_rate": cnt[8] / max(cnt[7], 1),
           "rec_precision": cnt[6] / max(cnt[5], 1), "recs_per_row": cnt[4] / max(cnt[0], 1)}

    # the stage breakdown (not part of the value): the same step as an eager rs_cv_step call
    # with the library's stage events on
    ctx.profile_enable(True)
    between()
    eager_step()
    torch.cuda.synchronize()
    ctx.profile_read()
    stages = {}
    eager_tot = 0.0
    for _ in range(args.steps):
        between()
        eager_step()
        torch.cuda.synchronize()
        eager_tot += ev[0].elapsed_time(ev[1])
        for k_, v_ in ctx.profile_read().items():
            stages[k_] = stages.get(k_, 0.0) + v_
    ctx.profile_enable(False)
    ctx.check_device_status()

    # the stages before the solvers, each alone (not part of the value): in the step the
    # planning overlaps the standardization and the Gram
    alone = {"standardize": 0.0, "gram_f64": 0.0, "plan_rows": 0.0}
    for _ in range(3):
        between()
        ev[0].record(stream)
        ctx.standardize(db, Z)
        ev[1].record(stream)
        ctx.gram(zb, rs.RS_GRAM_F64, K)
        ev[2].record(stream)
        ctx.rec_offsets(zb, ds, out.rec_offsets)
        ev[3].record(stream)
        torch.cuda.synchronize()
        for i_, k_ in enumerate(alone):
            alone[k_] += ev[i_].elapsed_time(ev[i_ + 1]) / 3

    work = algorithmic_work(batch, splits, CFG["k"])
    stage_ms = {k_: v_ / args.steps for k_, v_ in stages.items()}
    # the fit-predict path after the planning: the solver group and the rank pass
    fit_ms = stage_ms.get("solve", 0.0) + stage_ms.get("solve_join", 0.0) + stage_ms.get("rank", 0.0)
    # the three solver kernels run on two streams: they are timed as one group, from the end of
    # the bucketing to the join (stage events on the call's stream)
    stage_ms["solve_group"] = stage_ms.get("solve", 0.0) + stage_ms.get("solve_join", 0.0)
    work["solve_group"] = work["solve_small"] + work["solve_large"]
    top = max(("solve_group", "rank"), key=lambda k_: stage_ms.get(k_, 0.0))
    peak_meas = None if args.only_step else rs.measure_fma_peak(True, 2048) / 1e3
    fp64_peak = FP64_PEAK_NOMINAL_GFLOPS / 1e3
    hbm_peak = measured_hbm_peak()
    if top == "rank":
        achieved = work["rank_bytes"] / (stage_ms[top] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "rank_pass_kernel", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": profiled_traffic("rank"),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)",
                "bytes_per_launch": work["rank_bytes"]}
    else:
        achieved = work[top] / (stage_ms[top] * 1e-3) / 1e12
        roof = {"bound": "alu",
                "kernel": "solve_small_kernel x2 + solve_mid_kernel (one group on two streams)",
                "achieved": achieved,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "traffic": profiled_traffic("solve"),
                "peak_source": "FP64 1.25 TFLOP/s nominal (152 SMs x 2 FMA/clk x 2.07 GHz)",
                "flops_per_launch": work[top]}
    path_flops = work["solve_group"]
    roof["peak_measured_fp64_fma_chains"] = peak_meas
    roof["stages"] = {
        "solve_group": {"ms": stage_ms["solve_group"], "flops": work["solve_group"],
                        "frac_fp64": work["solve_group"] / (stage_ms["solve_group"] * 1e-3) / 1e12 / fp64_peak,
                        "note": "n <= split on the call's stream; n > 10 (shared memory) then "
                                "split < n <= 10 on a second stream; joined before the rank pass"},
        "rank": {"ms": stage_ms.get("rank"), "bytes": work["rank_bytes"],
                 "frac_hbm": work["rank_bytes"] / (stage_ms["rank"] * 1e-3) / 1e9 / hbm_peak,
                 "traffic": profiled_traffic("rank"),
                 "note": "bound by the integer ALU pipe (75 % busy in profiles/batched_cv_kernels.md: "
                         "64-bit order-preserving keys, 15 comparisons, threshold, top-k and scoring "
                         "per row), not by HBM"},
        "fit_predict_path": {"ms": fit_ms, "fp64_flops": path_flops,
                             "frac_fp64": path_flops / (fit_ms * 1e-3) / 1e12 / fp64_peak}}
    # the whole step against the sum of its stages' roofline times (HBM bytes at the measured
    # copy bandwidth, FP64 flops at the FP64 peak), on the executed (dual) form
    bounds = {"standardize": work["std_bytes"] / (hbm_peak * 1e6),
              "gram": work["gram_flops"] / (fp64_peak * 1e9),
              "plan": work["mask_bytes"] / (hbm_peak * 1e6),
              "solve": work["solve_group"] / (fp64_peak * 1e9),
              "rank": work["rank_bytes"] / (hbm_peak * 1e6)}
    # the stages before the solvers, from their stand-alone times
    roof["stages"]["gram_alone"] = {"ms": alone["gram_f64"], "flops": work["gram_flops"],
                                    "frac_fp64": work["gram_flops"] / (alone["gram_f64"] * 1e-3) / 1e12 / fp64_peak}
    roof["stages"]["standardize_alone"] = {
        "ms": alone["standardize"], "bytes": work["std_bytes"],
        "frac_hbm": work["std_bytes"] / (alone["standardize"] * 1e-3) / 1e9 / hbm_peak,
        "note": "bound by the FP64 logarithm (9 FP64 instructions per element), not by HBM"}
    roof["stages"]["step"] = {"ms": ms_step, "bound_ms": sum(bounds.values()),
                              "frac": sum(bounds.values()) / ms_step,
                              "bound_ms_parts": bounds,
                              "note": "sum of the stages' roofline times / measured step time"}

    ctx.profile_enable(False)                  # (stage events only for the step above)

    # plain GPU form: one launch per step per program, FP64, one warp per fit, no persistence
    plain = None
    if not args.no_plain and not args.only_step and rank == 0:
        plain = run_plain(rs, ctx, batch, splits, dev, stream, flush, args)

    # end to end through the C ABI single call with host buffers (pinned), copies timed
    e2e = None if args.only_step else run_e2e(rs, ctx, batch, splits, dev, stream, flush, args, R)

    ibk = None
    if rank == 0 and not args.only_step and not args.no_ibk:
        ibk = run_ibk(rs, ctx, batch, splits, dev, stream, flush, args)

    lovo = None
    if rank == 0 and not args.only_step and not args.no_lovo:
        lovo = run_lovo(rs, ctx, dev, stream, flush, args)

    xfer = None
    if rank == 0 and not args.only_step and not args.no_transfer:
        xfer = run_transfer(rs, ctx, dev, stream, flush, args)

    pooled = None
    if rank == 0 and not args.only_step and not args.no_transfer:
        pooled = run_pooled(rs, ctx, batch, dev, stream, flush, args)

    real = None
    if rank == 0 and not args.only_step and not args.no_transfer:
        real = run_real_nb(rs, ctx, dev, stream, flush, args)

    unev = None
    if rank == 0 and not args.only_step and not args.no_uneven:
        unev = run_uneven(rs, ctx, dev, stream, flush, args)

    prec = None
    if rank == 0 and not args.only_step and not args.no_precision:
        prec = run_precision(rs, ctx, dev, stream, flush, args)

    sur = None
    if rank == 0 and not args.only_step and not args.no_surrogate:
        sur = run_surrogate(rs, ctx, dev, stream, flush, args)

    cpu = None
    if rank == 0 and world == 1 and not args.only_step:
        cpu = cpu_reference_sample(batch, splits, args.cpu_seconds)
        cpu.pop("seconds")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "programs": CFG["programs"], "versions": "16..64",
                   "features": CFG["feat"], "splits_per_program": CFG["splits"],
                   "recs_per_step": R, "lambda": CFG["lam"], "k": CFG["k"], "tau": CFG["tau"],
                   "l2": "flushed between timed steps (256 MB write, untimed)",
                   "parallelism": (f"{world} GPUs, a job of {world} x 64 programs split by the longest-"
                                   "processing-time rule, no data-path collective, counters summed at the end"
                                   if world > 1 else "1 GPU")},
        "kernels_ms": {"step": ms_step, "eager_step": eager_tot / args.steps,
                       **{k_ + "_alone": v_ for k_, v_ in alone.items()},
                       "solve_and_rank": fit_ms,
                       **{"fit." + k_: v_ for k_, v_ in stage_ms.items()},
                       "note": "step: one CUDA-graph launch of the whole rs_cv_step per step (the value); "
                               "eager_step and the fit.* stages: the same step as an eager rs_cv_step "
                               "call with the library's stage events; the planning (fit.pairs, "
                               "fit.plan_fits, fit.bucket_fits) runs on a second stream beside the "
                               "standardization and the Gram, so fit.bucket_fits spans the bucketing and "
                               "the wait for the Gram; *_alone: those stages timed on their own"},
        "roofline": roof,
        "accuracy": acc,
        "plain_form": plain,
        "surrogate_form": sur,
        "precision_form": prec,
        "uneven_form": unev,
        "ibk_form": ibk,
        "lovo_form": lovo,
        "table2_transfer": xfer,
        "real_nb": real,
        "pooled_form": pooled,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    ctx.close()
    return 0


def run_plain(rs, ctx, batch, splits, dev, stream, flush, args):
    import torch
    progs = []
    for p in range(batch.n_programs):
        rsl = batch.program_rows(p)
        V, F = batch.versions(p), int(batch.feat_width[p])
        o = int(batch.x_offsets[p])
        s0, s1 = int(splits.split_offsets[p]), int(splits.split_offsets[p + 1])
        from paper_1910_07776_gb300 import synth
        sub = synth.ProgramBatch(
            X=batch.X[o:o + V * F], x_offsets=np.zeros(1, np.int64),
            row_offsets=np.array([0, V], np.int64), feat_width=np.array([F], np.int32),
            masks=batch.masks[rsl], log_time=batch.log_time[rsl],
            cycles=None if batch.cycles is None else batch.cycles[rsl])
        ss = synth.Splits(split_offsets=np.array([0, s1 - s0], np.int64),
                          train_masks=splits.train_masks[s0:s1])
        db = rs.DeviceBatch.from_host(sub, dev)
        ds = rs.DeviceSplits.from_host(ss, dev, sub)
        Z = torch.empty(db.x_elems, dtype=torch.float64, device=dev)
        K = torch.zeros(64 * 64, dtype=torch.float64, device=dev)
        ro = ctx.rec_offsets(db, ds)
        R = int(ro[-1].item())
        o_ = rs.alloc_outputs(R, ds.n_splits, CFG["k"], dev, pred_all=False)
        progs.append((db, ds, Z, db.with_X(Z), K, ro, o_, R))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step():
        for db, ds, Z, zb, K, ro, o_, R in progs:
            ctx.standardize(db, Z)
            ctx.gram(zb, rs.RS_GRAM_F64, K)
            ctx.rec_offsets(zb, ds, ro)
            ctx.predict_rank(zb, K, ds, ro, o_.rec_code, lam=CFG["lam"], k=CFG["k"],
                             tau=CFG["tau"], form=rs.RS_FORM_PLAIN, rec_pred=o_.rec_pred,
                             counters=o_.counters)

    def between():
        flush.fill_(1)
        for pr in progs:
            pr[6].counters.zero_()

    for _ in range(3):
        between()
        step()
    torch.cuda.synchronize()
    tot = 0.0
    n = max(2, min(args.steps, 5))
    for _ in range(n):
        between()
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    R = sum(pr[7] for pr in progs)
    cnt = sum(pr[6].counters.cpu().numpy().view(np.uint64).astype(np.float64) for pr in progs)
    return {"value": R * n / (tot / 1e3), "unit": UNIT, "ms_per_step": tot / n,
            "launches_per_step": 6 * len(progs),
            "sign_accuracy": cnt[3] / max(cnt[2], 1), "top1_hit_rate": cnt[8] / max(cnt[7], 1)}


def run_ibk(rs, ctx, batch, splits, dev, stream, flush, args):
    """The instance-based learner (Sec. 3.4, IBK k = 10) beside ridge, through the one-call
    step on the same inputs: the batched-CV workload (where most fits have at most 10 pairs,
    so the mean of all labels is the prediction) and a leave-one-version-out workload over all
    64 masks (31 pairs per fit: the 10-nearest selection decides every prediction), where ridge
    is also timed with its fits in closed form (RS_LOO_CLOSED)."""
    import torch
    from paper_1910_07776_gb300 import synth
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def measure(b, sp, reps, loo=False):
        db = rs.DeviceBatch.from_host(b, dev)
        ds = rs.DeviceSplits.from_host(sp, dev, b)
        R = ds.n_test_rows
        ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
        res = {}
        forms = [("ridge", 0), ("ibk", rs.RS_MODEL_IBK)]
        if loo:
            forms.append(("ridge_closed_form", rs.RS_LOO_CLOSED))
        for name, flags in forms:
            o = rs.alloc_outputs(R, ds.n_splits, CFG["k"], dev, pred_all=False)
            step = lambda: ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"],
                                       tau=CFG["tau"], flags=flags, rec_pred=o.rec_pred, counters=o.counters)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            o.counters.zero_()
            tot = 0.0
            for _ in range(reps):
                flush.fill_(1)
                e0.record(stream)
                step()
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            ctx.check_device_status()
            c = o.counters.cpu().numpy().view(np.uint64).astype(np.float64)
            ms = tot / reps
            res[name] = {"ms": ms, "value": R / (ms * 1e-3), "unit": UNIT,
                         "sign_accuracy": c[3] / max(c[2], 1), "top1_hit_rate": c[8] / max(c[7], 1),
                         "rec_precision": c[6] / max(c[5], 1)}
        res["recs_per_step"] = R
        return res

    out = {"neighbors": rs.IBK_NEIGHBORS,
           "batched_cv": {"workload": WORKLOAD, **measure(batch, splits, 20)}}
    b = synth.make_batch_fast(256, versions=64, feat=256, dtype=np.float32, seed=41)
    sp = synth.make_splits(b, "lovo")
    out["lovo"] = {"workload": "256 programs x 64 versions (all masks) x 256 f32 features, leave-one-"
                               "version-out (16,384 splits, 98,304 fits of 31 pairs)", **measure(b, sp, 20, loo=True)}
    return out


def run_lovo(rs, ctx, dev, stream, flush, args, programs=256):
    """Leave-one-version-out (the paper's protocol over all 64 masks, Sec. 5) at the
    precision form's shape: 256 programs x 64 versions x 1024 FP64 features, 16,384 splits,
    98,304 ridge fits of 31 pairs each, every stage in FP64 through the one-call step.  The
    fits of more than 16 pairs run in solve_wide_kernel; its stage time (from the end of the
    planning to the join of the solver streams) against its FP64 flops gives its roofline
    fraction, and the Gram (1.07 GFLOP) is timed alone beside it.  The same step with
    RS_LOO_CLOSED (one inverse per program and optimization, every fit from it in O(n)) is
    timed beside it, with its largest prediction difference from the direct solves."""
    import torch
    from paper_1910_07776_gb300 import synth
    b = synth.make_batch_fast(programs, versions=64, feat=1024, dtype=np.float64, seed=43)
    sp = synth.make_splits(b, "lovo")
    db = rs.DeviceBatch.from_host(b, dev)
    ds = rs.DeviceSplits.from_host(sp, dev, b)
    R = ds.n_test_rows
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(flags):
        o = rs.alloc_outputs(R, ds.n_splits, CFG["k"], dev)
        step = lambda: ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"],
                                   tau=CFG["tau"], flags=flags, rec_pred=o.rec_pred, pred_all=o.pred_all,
                                   counters=o.counters)
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        o.counters.zero_()
        ctx.profile_enable(True)
        reps, tot, stages = 10, 0.0, {}
        for _ in range(reps):
            flush.fill_(1)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
            for k_, v_ in ctx.profile_read().items():
                stages[k_] = stages.get(k_, 0.0) + v_ / reps
        ctx.profile_enable(False)
        ctx.check_device_status()
        return tot / reps, stages, o

    ms, stages, o = timed(0)
    ms_c, stages_c, oc = timed(rs.RS_LOO_CLOSED)
    Z = torch.empty(db.x_elems, dtype=torch.float64, device=dev)
    K = torch.zeros(db.n_programs * 64 * 64, dtype=torch.float64, device=dev)
    ctx.standardize(db, Z)
    g_ms = 0.0
    for _ in range(3):
        flush.fill_(1)
        e0.record(stream)
        ctx.gram(db.with_X(Z), rs.RS_GRAM_F64, K)
        e1.record(stream)
        torch.cuda.synchronize()
        g_ms += e0.elapsed_time(e1) / 3
    work = algorithmic_work(b, sp, CFG["k"])
    fp64_peak = FP64_PEAK_NOMINAL_GFLOPS / 1e3
    solve_ms = stages.get("solve", 0.0) + stages.get("solve_join", 0.0)
    flops = work["solve_small"] + work["solve_large"]
    c = o.counters.cpu().numpy().view(np.uint64).astype(np.float64)
    cc = oc.counters.cpu().numpy().view(np.uint64).astype(np.float64)
    pa, pc = o.pred_all.cpu().numpy(), oc.pred_all.cpu().numpy()
    fin = ~np.isnan(pa)
    same_nan = bool(np.array_equal(np.isnan(pa), np.isnan(pc)))
    diff = np.abs(pa[fin] - pc[fin])
    # the closed form's FP64 work: one Gauss-Jordan inverse per (program, optimization) with at
    # least one pair, padded to 32 x 32 with two right-hand sides (2 flops per FMA)
    n_inv = 0
    for p_ in range(b.n_programs):
        m_ = set(int(x) for x in b.masks[b.program_rows(p_)])
        n_inv += sum(1 for j in range(6) if any(not (x >> j) & 1 and (x | 1 << j) in m_ for x in m_))
    inv_flops = n_inv * 2.0 * 32 * 32 * (32 + 2)
    fit_ms_c = stages_c.get("solve", 0.0) + stages_c.get("solve_join", 0.0)
    closed = {"ms_per_step": ms_c, "value": R / (ms_c * 1e-3), "unit": UNIT, "stages_ms": stages_c,
              "fit_ms": fit_ms_c, "inverses": n_inv, "inverse_flops": inv_flops,
              "fit_stage_frac_fp64": inv_flops / (fit_ms_c * 1e-3) / 1e12 / fp64_peak if fit_ms_c > 0 else None,
              "fit_stage_note": "the inverses' FMAs (1,536 x 32 x 32 x 34 at 256 programs) over the stage time, "
                                "which also holds the diagonal kernel and the O(1) per-fit kernel",
              "sign_accuracy": cc[3] / max(cc[2], 1), "top1_hit_rate": cc[8] / max(cc[7], 1),
              "fits_ok": int(cc[9]),
              "max_abs_pred_diff_vs_direct": float(diff.max()) if diff.size else 0.0,
              "max_rel_pred_diff_vs_direct": float((diff / np.maximum(np.abs(pa[fin]), 1e-300)).max()) if diff.size else 0.0,
              "nan_pattern_equal": same_nan,
              "rec_code_rows_differing": int((o.rec_code != oc.rec_code).sum().item())}
    return {"workload": f"{programs} programs x 64 versions (all masks) x 1024 f64 features, "
                        f"leave-one-version-out ({64 * programs:,} splits, {384 * programs:,} fits of 31 pairs)",
            "ms_per_step": ms, "value": R / (ms * 1e-3), "unit": UNIT, "recs_per_step": R,
            "sign_accuracy": c[3] / max(c[2], 1), "top1_hit_rate": c[8] / max(c[7], 1),
            "stages_ms": stages,
            "roofline": {"bound": "alu", "kernel": "solve_wide_kernel (fits of 17..32 pairs)",
                         "achieved": flops / (solve_ms * 1e-3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": flops / (solve_ms * 1e-3) / 1e12 / fp64_peak, "flops_per_launch": flops,
                         "ms": solve_ms,
                         "peak_source": "FP64 1.25 TFLOP/s nominal (152 SMs x 2 FMA/clk x 2.07 GHz)"},
            "closed_form": closed,
            "gram_alone": {"ms": g_ms, "flops": work["gram_flops"],
                           "frac_fp64": work["gram_flops"] / (g_ms * 1e-3) / 1e12 / fp64_peak}}


PAPER_TABLE3_IBK = {1: 97.3, 2: 96.0, 3: 96.3, 4: 92.0, 5: 83.6, 6: 55.7}   # Table 3, % (real profiles)
PAPER_TABLE3_M5P = {1: 86.4, 2: 86.4, 3: 33.3, 4: 81.6, 5: 33.3, 6: 60.1}


def run_pooled(rs, ctx, batch, dev, stream, flush, args):
    """Pooled ridge in primal form (rs_fit_pooled): one model per optimization trained on the
    pairs of 48 programs of the batched-CV workload (256 features; the Gram X^T W X of each
    optimization's ~600 pairs as one batched tcgen05 GEMM of the BF16 hi/lo split, FP64
    Cholesky, one FP64 refinement step), then ranking the 16 held-out programs' versions
    (rs_predict_pooled) -- a model trained on other codes, as in Sec. 5's transfer."""
    import torch
    from paper_1910_07776_gb300 import synth
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tr = synth.take_programs(batch, list(range(48)))
    te = synth.take_programs(batch, list(range(48, 64)))
    dtr, dte = rs.DeviceBatch.from_host(tr, dev), rs.DeviceBatch.from_host(te, dev)
    ztr = dtr.with_X(ctx.standardize(dtr))
    zte = dte.with_X(ctx.standardize(dte))
    ws = ctx.workspace(ctx.pooled_workspace_bytes(ztr))
    fit = lambda: ctx.fit_pooled(ztr, None, lam=CFG["lam"], flags=rs.RS_REFINE_X, workspace=ws)
    for _ in range(3):
        coef, st = fit()
    torch.cuda.synchronize()
    reps, tot = 10, 0.0
    for _ in range(reps):
        flush.fill_(1)
        e0.record(stream)
        coef, st = fit()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    n = zte.n_rows
    code = torch.empty(n, dtype=torch.int32, device=dev)
    rp = torch.empty(n * CFG["k"], dtype=torch.float64, device=dev)
    cnt = torch.zeros(16, dtype=torch.int64, device=dev)
    ctx.predict_pooled(zte, coef, st, code, k=CFG["k"], tau=CFG["tau"], rec_pred=rp, counters=cnt)
    torch.cuda.synchronize()
    ctx.check_device_status()
    c = cnt.cpu().numpy().astype(np.float64)
    pairs = [sum(1 for p in range(tr.n_programs) for v in range(tr.versions(p))
                 for mm in [tr.masks[tr.program_rows(p)].astype(int)]
                 if not (mm[v] >> j) & 1 and (mm[v] | 1 << j) in set(mm.tolist())) for j in range(6)]
    Np = (max(pairs) + 63) // 64 * 64
    F = int(tr.feat_width[0])
    gemm_flops = 6 * F * F * 3 * Np * 2
    return {"workload": "pooled ridge: 48 programs of the batched-CV workload train (256 f32 features), "
                        "16 held-out programs ranked",
            "fit_ms": tot / reps, "pairs_per_optimization": pairs, "status": st.cpu().numpy().tolist(),
            "gram_gemm_flops": gemm_flops,
            "held_out": {"rows": n, "sign_accuracy": c[3] / max(c[2], 1), "top1_hit_rate": c[8] / max(c[7], 1),
                         "rec_precision": c[6] / max(c[5], 1)}}


def _transfer_experiment(rs, ctx, dev, stream, flush, pr, e):
    """One Table 2 experiment: per learner (ridge, IBK, M5P) one rs_transfer call timed on the
    device after warm-up, the sign accuracy of Table 3, the top-1 hit rate and the AC/EX ratios
    (actual over expected speedup, Sec. 5) of every scored prediction."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dtr = rs.DeviceBatch.from_host(pr.train, dev)
    dte = rs.DeviceBatch.from_host(pr.test, dev)
    offs = torch.from_numpy(pr.groups).to(dev)
    g = (offs, int(np.diff(pr.groups).max()))
    ws = ctx.workspace(ctx.transfer_workspace_bytes(dtr, dte, g, rs.RS_MODEL_M5P))
    R = dte.n_rows
    # actual log speedups of the test rows (host, from the test set's own times)
    act = np.full((R, 6), np.nan)
    for q in range(pr.test.n_programs):
        rows = pr.test.program_rows(q)
        m = pr.test.masks[rows].astype(int)
        lt = pr.test.log_time[rows]
        slot = {int(v): i for i, v in enumerate(m)}
        for t in range(len(m)):
            for j in range(6):
                w = slot.get(int(m[t]) | (1 << j))
                if not (m[t] >> j) & 1 and w is not None:
                    act[rows.start + t, j] = lt[t] - lt[w]
    res = {"problems": int(pr.test.n_programs), "train_runs_per_problem": int(np.diff(pr.groups).max()),
           "test_rows": int(R), "opt_mask": int(pr.opt_mask), "paper_ibk_accuracy_pct": PAPER_TABLE3_IBK[e],
           "paper_m5p_accuracy_pct": PAPER_TABLE3_M5P[e]}
    for name, flags in (("ridge", 0), ("ibk", rs.RS_MODEL_IBK), ("m5p", rs.RS_MODEL_M5P)):
        o = rs.alloc_outputs(R, 0, CFG["k"], dev)
        call = lambda: ctx.transfer(dtr, dte, ws, o.rec_code, groups=g, lam=CFG["lam"], k=CFG["k"],
                                    tau=CFG["tau"], flags=flags, opt_mask=pr.opt_mask, rec_pred=o.rec_pred,
                                    pred_all=o.pred_all, counters=o.counters)
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        o.counters.zero_()
        reps, tot = 10, 0.0
        for _ in range(reps):
            flush.fill_(1)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ctx.check_device_status()
        c = o.counters.cpu().numpy().view(np.uint64).astype(np.float64) / reps
        pa = o.pred_all.cpu().numpy().reshape(R, 6)
        sc = ~np.isnan(pa) & ~np.isnan(act)
        ratio = np.exp(act[sc] - pa[sc])
        res[name] = {"ms": tot / reps, "sign_accuracy": c[3] / max(c[2], 1),
                     "top1_hit_rate": c[8] / max(c[7], 1), "rec_precision": c[6] / max(c[5], 1),
                     "scored": int(c[2]),
                     "ac_ex_quantiles_5_25_50_75_95": [float(x) for x in np.quantile(ratio, [.05, .25, .5, .75, .95])]
                     if ratio.size else None,
                     "ac_ex_within_10pct": float(np.mean(np.abs(ratio - 1.0) <= 0.1)) if ratio.size else None}
    return res


def run_transfer(rs, ctx, dev, stream, flush, args):
    """Table 2's six experiments (Sec. 5) on the seeded stand-ins of the BH / NB runs
    (synth.make_runs: 6 + 4 inputs x 3 runs x 64 versions x 96 counters).  Table 3's values come
    from the paper's real profiles: context only."""
    from paper_1910_07776_gb300 import synth
    runs = synth.make_runs(seed=0)
    out = {"data": "synthetic stand-ins: 2 codes (6 and 4 inputs) x 3 runs x 64 versions x 96 f64 counters",
           "experiments": {}}
    for e in range(1, 7):
        out["experiments"][str(e)] = _transfer_experiment(rs, ctx, dev, stream, flush,
                                                          synth.table2_problems(runs, e), e)
    return out


def run_real_nb(rs, ctx, dev, stream, flush, args):
    """Measured tier-1 data: the 64 versions of the n-body code NB (tier1/nbody.cu, the six
    optimizations of Sec. 3.3) profiled on this GPU (tier1/capture.py; 4 inputs x 3 runs x 64
    versions, counters / cycles).  Leave-one-version-out on every (input, run) with ridge and
    IBK through rs_cv_step, and Table 2's experiments 1-4 with NB in the place of BH through
    rs_transfer.  Table 3's figures (BH / NB on a K20c) are context only."""
    import torch
    from paper_1910_07776_gb300 import synth, tier1
    if not tier1.available():
        return None
    runs = tier1.load_nb()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sp = synth.make_splits(runs, "lovo")
    db = rs.DeviceBatch.from_host(runs, dev)
    ds = rs.DeviceSplits.from_host(sp, dev, runs)
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    out = {"data": f"measured: {runs.meta['gpu']}, n-body 64 versions x {runs.feat_width[0]} counters / cycles, "
                   f"inputs (bodies, steps) {runs.meta['inputs']}, {runs.meta['runs']} runs",
           "capture": runs.meta["command"], "lovo": {}, "experiments": {}}
    for name, flags in (("ridge", 0), ("ibk", rs.RS_MODEL_IBK)):
        o = rs.alloc_outputs(ds.n_test_rows, ds.n_splits, CFG["k"], dev, pred_all=False)
        ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"], flags=flags,
                    rec_pred=o.rec_pred, counters=o.counters)
        torch.cuda.synchronize()
        o.counters.zero_()
        e0.record(stream)
        ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"], flags=flags,
                    rec_pred=o.rec_pred, counters=o.counters)
        e1.record(stream)
        torch.cuda.synchronize()
        c = o.counters.cpu().numpy().view(np.uint64).astype(np.float64)
        out["lovo"][name] = {"ms": e0.elapsed_time(e1), "sign_accuracy": c[3] / max(c[2], 1),
                             "top1_hit_rate": c[8] / max(c[7], 1), "scored": int(c[2])}
    for e in range(1, 5):
        out["experiments"][str(e)] = _transfer_experiment(rs, ctx, dev, stream, flush,
                                                          synth.table2_problems(runs, e, code="NB"), e)
    return out


def run_uneven(rs, ctx, dev, stream, flush, args):
    """Uneven stream: 10,000 programs x U{8..64} versions x feature widths from {64, 128, 256,
    512}, 1,024 random half splits per program (10.24 M splits), FP32 counters, FP64 Gram and
    fits; eager step vs autotuned vs one CUDA-graph launch per step."""
    import torch
    from paper_1910_07776_gb300 import synth
    t0 = time.perf_counter()
    b = synth.make_batch_fast(10000, versions=(8, 64), feat_choices=[64, 128, 256, 512], dtype=np.float32,
                              seed=31)
    sp = synth.make_half_splits_fast(b, 1024, seed=31)
    db = rs.DeviceBatch.from_host(b, dev)
    ds = rs.DeviceSplits.from_host(sp, dev, b)
    gen_s = time.perf_counter() - t0
    R = ds.n_test_rows
    o = rs.alloc_outputs(R, ds.n_splits, CFG["k"], dev, pred_all=False)
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    step = lambda: ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"],
                               tau=CFG["tau"], rec_pred=o.rec_pred)
    eager_default = timed(step)
    tune = ctx.autotune(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"],
                        rec_pred=o.rec_pred)
    eager_tuned = timed(step)
    g = ctx.cv_graph(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"],
                     rec_pred=o.rec_pred, counters=o.counters)
    o.counters.zero_()
    graph_ms = timed(g.launch)
    torch.cuda.synchronize()
    g.close()
    cnt = o.counters.cpu().numpy().view(np.uint64).astype(np.float64)
    ctx.check_device_status()
    # the precision split of the precision form on the same stream: the Gram on the tensor cores
    # (BF16 hi/lo, tile shape autotuned for the batch's width), FP64 fits
    gram_tune = ctx.autotune_gram(db, ws)
    o.counters.zero_()
    bf_step = lambda: ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"],
                                  tau=CFG["tau"], precision=rs.RS_GRAM_BF16X3, rec_pred=o.rec_pred,
                                  counters=o.counters)
    bf_ms = timed(bf_step)
    cnt_bf = o.counters.cpu().numpy().view(np.uint64).astype(np.float64) / 4
    ctx.check_device_status()
    return {"workload": "10,000 programs x U{8..64} versions x F in {64,128,256,512} f32, 1,024 half "
                        "splits/program (10,240,000 splits)",
            "recs_per_step": R, "value": R / (graph_ms * 1e-3), "unit": UNIT, "graph_ms": graph_ms,
            "eager_default_ms": eager_default, "eager_tuned_ms": eager_tuned,
            "autotune": {"solve_split": tune["solve_split"], "rank_waves": tune["rank_waves"],
                         "solve_order": tune["solve_order"]},
            "sign_accuracy": cnt[3] / max(cnt[2], 1), "data_gen_s": gen_s,
            "bf16x3_gram": {"ms": bf_ms, "value": R / (bf_ms * 1e-3), "gram_autotune": gram_tune,
                            "sign_accuracy": cnt_bf[3] / max(cnt_bf[2], 1),
                            "note": "tensor-core Gram (BF16 hi/lo split) with the autotuned tile shape, "
                                    "FP64 fits, eager calls"}}


def _rel_stats(d, ref):
    d, ref = np.abs(np.ravel(d)), np.abs(np.ravel(ref))
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.where(ref > 0, d / ref, np.where(d > 0, np.inf, 0.0))
    return {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)), "max": float(e.max()),
            "normwise_max": float(d.max() / max(ref.max(), 1e-300))}


def precision_coef_errors(rs, ctx, batch, dev, programs=4):
    """Per-coefficient errors of the BF16x3 forms (raw, refined) against the FP64 GPU path on
    the first `programs` programs of a leave-one-version-out batch: the dual alpha and b of
    every fit and the primal beta = sum_a alpha_a z_a it implies (computed on the host in FP64
    from the standardized features), each as elementwise relative error (median, 99th
    percentile, max) and normwise (max |error| / max |value|)."""
    import torch
    from paper_1910_07776_gb300 import synth
    sub = synth.take_programs(batch, list(range(programs)))
    sp = synth.make_splits(sub, "lovo")
    db = rs.DeviceBatch.from_host(sub, dev)
    ds = rs.DeviceSplits.from_host(sp, dev, sub)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    Zh = Z.cpu().numpy()
    S = ds.n_splits
    coefs = {}
    for name, prec, flags in (("f64", rs.RS_GRAM_F64, 0), ("bf16x3", rs.RS_GRAM_BF16X3, 0),
                              ("bf16x3_refined", rs.RS_GRAM_BF16X3, rs.RS_REFINE_X)):
        K = ctx.gram(zb, prec)
        c = torch.zeros(S * 6 * 33, dtype=torch.float64, device=dev)
        ctx.fit_batched(zb, K, ds, CFG["lam"], rs.RS_FORM_BATCHED | flags, c)
        coefs[name] = c.cpu().numpy().reshape(S, 6, 33)
    beta = {k: [] for k in coefs}
    alpha = {k: [] for k in coefs}
    bias = {k: [] for k in coefs}
    for p in range(programs):
        V, F = sub.versions(p), int(sub.feat_width[p])
        Zp = Zh[int(sub.x_offsets[p]):int(sub.x_offsets[p]) + V * F].reshape(V, F)
        m = sub.masks[sub.program_rows(p)].astype(int)
        slot = {int(x): i for i, x in enumerate(m)}
        for s_ in range(int(sp.split_offsets[p]), int(sp.split_offsets[p + 1])):
            T = int(sp.train_masks[s_])
            for j in range(6):
                vs = [v for v in range(V) if not (m[v] >> j) & 1 and (m[v] | 1 << j) in slot
                      and (T >> v) & 1 and (T >> slot[m[v] | 1 << j]) & 1]
                n = len(vs)
                if n == 0:
                    continue
                for k_, cf in coefs.items():
                    al = cf[s_, j, 1:1 + n]
                    alpha[k_].append(al)
                    beta[k_].append(al @ Zp[vs])
                    bias[k_].append(cf[s_, j, :1])
    out = {"sample": f"{programs} programs, {S} leave-one-out splits, {S * 6} fits"}
    ref = {"beta": np.concatenate(beta["f64"]), "alpha": np.concatenate(alpha["f64"]),
           "b": np.concatenate(bias["f64"])}
    for k_ in ("bf16x3", "bf16x3_refined"):
        out[k_] = {"beta": _rel_stats(np.concatenate(beta[k_]) - ref["beta"], ref["beta"]),
                   "alpha": _rel_stats(np.concatenate(alpha[k_]) - ref["alpha"], ref["alpha"]),
                   "b": _rel_stats(np.concatenate(bias[k_]) - ref["b"], ref["b"])}
    return out


def run_precision(rs, ctx, dev, stream, flush, args):
    """Precision form: 256 programs x 64 versions x 1024 FP64 features, leave-one-version-out,
    a condition-number sweep by random mixing; BF16-split tensor-core Gram + FP64 factorisation
    + one refinement step through Z, against the FP64 path (itself within 1e-9 of the CPU
    reference).  Reports errors of the raw and refined forms per kappa and their timings, and
    those of the FP64 and the tensor-core paths with their fits in closed form (RS_LOO_CLOSED)."""
    import torch
    from paper_1910_07776_gb300 import synth
    base = synth.make_batch_fast(256, versions=64, feat=1024, dtype=np.float64, seed=21)
    splits = synth.make_splits(base, "lovo")
    res = {"workload": "256 programs x 64 versions x 1024 f64 features, LOVO (16,384 splits, 98,304 fits)",
           "per_kappa": {}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for kappa in (1e2, 1e4, 1e6, 1e8):
        b = synth.apply_mixing(base, kappa, seed=21)
        db = rs.DeviceBatch.from_host(b, dev)
        ds = rs.DeviceSplits.from_host(splits, dev, b)
        R = ds.n_test_rows
        ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
        if "gram_autotune" not in res:              # the tensor-core Gram's tile shape, 1024 features
            res["gram_autotune"] = ctx.autotune_gram(db, ws)
        outs = {}
        times = {}
        for name, prec, flags in (("f64", rs.RS_GRAM_F64, 0), ("bf16x3", rs.RS_GRAM_BF16X3, 0),
                                  ("bf16x3_refined", rs.RS_GRAM_BF16X3, rs.RS_REFINE_X),
                                  ("f64_closed_form", rs.RS_GRAM_F64, rs.RS_LOO_CLOSED),
                                  ("bf16x3_closed_form", rs.RS_GRAM_BF16X3, rs.RS_LOO_CLOSED)):
            o = rs.alloc_outputs(R, ds.n_splits, CFG["k"], dev)
            ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"],
                        flags=flags, precision=prec, rec_pred=o.rec_pred, pred_all=o.pred_all)
            torch.cuda.synchronize()
            flush.fill_(1)
            e0.record(stream)
            ctx.cv_step(db, ds, ws, o.rec_offsets, o.rec_code, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"],
                        flags=flags, precision=prec, rec_pred=o.rec_pred, pred_all=o.pred_all)
            e1.record(stream)
            torch.cuda.synchronize()
            times[name] = e0.elapsed_time(e1)
            outs[name] = (o.pred_all.cpu().numpy().reshape(R, 6), o.rec_code.cpu().numpy())
        ref, rcode = outs["f64"]
        ok = ~np.isnan(ref)
        sc = float(np.abs(ref[ok]).max())
        ent = {}
        for name in ("bf16x3", "bf16x3_refined", "f64_closed_form", "bf16x3_closed_form"):
            pa, code = outs[name]
            d = np.abs(pa[ok] - ref[ok])
            ent[name] = {"max_rel_err_pred": float(d.max() / sc), "median_rel_err_pred": float(np.median(d) / sc),
                         "pred_elementwise": _rel_stats(pa[ok] - ref[ok], ref[ok]),
                         "ranking_rows_changed": int(np.sum(code != rcode)), "ms": times[name],
                         "recs_per_s": R / (times[name] * 1e-3)}
        ent["f64"] = {"ms": times["f64"], "recs_per_s": R / (times["f64"] * 1e-3)}
        ent["coefficients_vs_f64_path"] = precision_coef_errors(rs, ctx, b, dev, programs=4)
        # achieved condition number of one training system (program 0, split 0, optimization 0)
        Zp = np.log(b.program_X(0) / b.cycles[b.program_rows(0)][:, None])
        Zp = (Zp - Zp.mean(0)) / np.where(Zp.std(0) > 1e-12, Zp.std(0), 1.0)
        m = b.masks[b.program_rows(0)].astype(int)
        rows = [v for v in range(1, 64) if not m[v] & 1 and (m[v] | 1) in set(m[1:])]
        Kt = Zp[rows] @ Zp[rows].T + CFG["lam"] * np.eye(len(rows))
        ent["achieved_cond_train_system"] = float(np.linalg.cond(Kt))
        res["per_kappa"][f"{kappa:.0e}"] = ent
    return res


def profile_surrogate():
    """The surrogate's kernels on a small seeded case, for ncu captures (not a bench line)."""
    import torch
    from paper_1910_07776_gb300 import build as _b
    _b.build()
    from paper_1910_07776_gb300 import rs, synth
    dev = torch.device("cuda", 0)
    ctx = rs.Context(0, torch.cuda.current_stream(dev))
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    Xtr = torch.randn(65536, 256, device=dev, dtype=torch.float64, generator=g)
    Ytr = 0.3 * torch.randn(65536, 6, device=dev, dtype=torch.float64, generator=g)
    Xte = torch.randn(131072, 256, device=dev, dtype=torch.float64, generator=g)
    masks = torch.randint(0, 64, (131072,), device=dev, dtype=torch.uint8, generator=g)
    sur = rs.Surrogate(ctx, 8192, infer_chunk=131072)
    sur.load(synth.init_mlp_params(11))
    sur.train(Xtr, Ytr, steps=16)
    code = torch.empty(131072, dtype=torch.int32, device=dev)
    rp = torch.empty(131072 * CFG["k"], dtype=torch.float64, device=dev)
    sur.infer(Xte, ood_threshold=3.0, want_ood=True, masks=masks, k=CFG["k"], tau=CFG["tau"], rec_code=code,
              rec_pred=rp, want_pred=False)
    torch.cuda.synchronize()
    ctx.check_device_status()
    print(json.dumps({"profile": "surrogate", "train_rows": 65536, "train_steps": 16, "infer_rows": 131072}))
    ctx.close()
    return 0


def run_surrogate(rs, ctx, dev, stream, flush, args):
    """Learned surrogate: 2 M training vectors labelled by the plain ridge predictor, ranked
    inference on 1 M held-out vectors, against the batched plain method on the same rows."""
    import torch
    from paper_1910_07776_gb300 import synth
    P_tr, P_te = 31250, 15625
    t0 = time.perf_counter()
    b = synth.make_batch_fast(P_tr + P_te, versions=64, feat=256, dtype=np.float32, seed=11)
    sp = synth.make_complementary_halves(b, seed=11)
    gen_s = time.perf_counter() - t0
    n_all = b.n_rows
    db = rs.DeviceBatch.from_host(b, dev)
    ds = rs.DeviceSplits.from_host(sp, dev, b)
    # plain labels: every version predicted by the fit on the other half of its program
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    K = ctx.gram(zb)
    ro = ctx.rec_offsets(zb, ds)
    R = ds.n_test_rows
    out = rs.alloc_outputs(R, ds.n_splits, CFG["k"], dev)
    ctx.predict_rank(zb, K, ds, ro, out.rec_code, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"],
                     flags=rs.RS_RANK_ALL, rec_pred=out.rec_pred, pred_all=out.pred_all)
    torch.cuda.synchronize()
    # row -> version: split 2p tests the complement of A, split 2p+1 tests A (slot order)
    tm = sp.train_masks.astype(np.uint64)
    bitsv = ((tm[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)) == 0   # test slots
    split_prog = np.repeat(np.arange(b.n_programs), 2)
    ver = (split_prog[:, None] * 64 + np.arange(64)[None, :])[bitsv]      # split-major, slot order
    assert ver.shape[0] == R
    inv = torch.from_numpy(np.argsort(ver)).to(dev)
    Y = out.pred_all.view(R, 6)[inv].contiguous()                         # [n_all][6], version order
    Zm = Z.view(n_all, 256)
    n_tr = P_tr * 64
    Xtr, Ytr = Zm[:n_tr], Y[:n_tr]
    Xte = Zm[n_tr:].contiguous()
    masks_te = db.masks[n_tr:].contiguous()
    sur = rs.Surrogate(ctx, 8192, infer_chunk=131072)
    sur.load(synth.init_mlp_params(11))
    steps = args.surrogate_epochs * (n_tr // 8192)
    lc = torch.zeros(steps, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sur.train(Xtr, Ytr, steps=steps, lr=1e-3, use_graph=True, loss_curve=lc)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    n_te = Xte.shape[0]
    code = torch.empty(n_te, dtype=torch.int32, device=dev)
    rp = torch.empty(n_te * CFG["k"], dtype=torch.float64, device=dev)
    thr = 3.0
    # timed: ranked surrogate inference with OOD flags
    for _ in range(2):
        sur.infer(Xte, ood_threshold=thr, want_ood=True, masks=masks_te, k=CFG["k"], tau=CFG["tau"],
                  rec_code=code, rec_pred=rp, want_pred=False)
    torch.cuda.synchronize()
    reps = 5
    inf_ms = 0.0
    for _ in range(reps):
        flush.fill_(1)
        e0.record(stream)
        _, score, fb = sur.infer(Xte, ood_threshold=thr, want_ood=True, masks=masks_te, k=CFG["k"],
                                 tau=CFG["tau"], rec_code=code, rec_pred=rp, want_pred=False)
        e1.record(stream)
        torch.cuda.synchronize()
        inf_ms += e0.elapsed_time(e1)
    inf_ms /= reps
    pred_s, _, _ = sur.infer(Xte)
    torch.cuda.synchronize()
    fb_frac = float(fb.float().mean())
    # the plain batched method on the held-out programs (same protocol), timed
    te = synth.ProgramBatch(X=b.X[n_tr * 256:], x_offsets=b.x_offsets[P_tr:] - b.x_offsets[P_tr],
                            row_offsets=b.row_offsets[P_tr:] - b.row_offsets[P_tr],
                            feat_width=b.feat_width[P_tr:], masks=b.masks[n_tr:],
                            log_time=b.log_time[n_tr:], cycles=b.cycles[n_tr:])
    tsp = synth.Splits(split_offsets=sp.split_offsets[P_tr:] - sp.split_offsets[P_tr],
                       train_masks=sp.train_masks[2 * P_tr:])
    tdb = rs.DeviceBatch.from_host(te, dev)
    tds = rs.DeviceSplits.from_host(tsp, dev, te)
    tout = rs.alloc_outputs(tds.n_test_rows, tds.n_splits, CFG["k"], dev, pred_all=False)
    ws = ctx.workspace(ctx.cv_workspace_bytes(tdb, tds))
    for _ in range(2):
        ctx.cv_step(tdb, tds, ws, tout.rec_offsets, tout.rec_code, lam=CFG["lam"], k=CFG["k"],
                    tau=CFG["tau"], rec_pred=tout.rec_pred)
    torch.cuda.synchronize()
    plain_ms = 0.0
    for _ in range(reps):
        flush.fill_(1)
        e0.record(stream)
        ctx.cv_step(tdb, tds, ws, tout.rec_offsets, tout.rec_code, lam=CFG["lam"], k=CFG["k"],
                    tau=CFG["tau"], rec_pred=tout.rec_pred)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms += e0.elapsed_time(e1)
    plain_ms /= reps
    # accuracy against the ground truth (all 64 masks present: t|j always exists)
    lt = b.log_time[n_tr:].reshape(P_te, 64)
    m = np.arange(64)
    act = np.stack([lt - lt[:, m | (1 << j)] for j in range(6)], axis=2)   # [P,64,6]
    cand = ((m[:, None] >> np.arange(6)[None, :]) & 1) == 0                 # [64,6]
    ps = pred_s.cpu().numpy().reshape(P_te, 64, 6).astype(np.float64)
    pp = Y[n_tr:].cpu().numpy().reshape(P_te, 64, 6)
    cm = np.broadcast_to(cand, ps.shape) & np.isfinite(pp)

    def acc(pr):
        sign = float(np.mean(((pr > 0) == (act > 0))[cm]))
        prm = np.where(cm, pr, -np.inf)
        acm = np.where(cm, act, -np.inf)
        rows = cm.any(axis=2)
        top1 = float(np.mean((prm.argmax(2) == acm.argmax(2))[rows]))
        return sign, top1

    s_sign, s_top1 = acc(ps)
    p_sign, p_top1 = acc(pp)
    mae = float(np.mean(np.abs(ps - pp)[cm]))
    rate_s = n_te / (inf_ms * 1e-3)
    rate_p = tds.n_test_rows / (plain_ms * 1e-3)

    # the plain fallback, executed and timed: the held-out programs again, with 5 % of them
    # holding three versions whose every counter is scaled by e^4 (profiles unlike the rest
    # of their program).  Timed per repetition: ranked surrogate inference with OOD flags, then
    # rs_surrogate_fallback (selection, gather, the plain pass over the flagged programs, merge)
    shifted, sprogs = synth.with_anomalous_versions(te, 0.05, per_program=3, seed=12)
    sdb = rs.DeviceBatch.from_host(shifted, dev)
    Zs = ctx.standardize(sdb).view(n_te, 256)
    fws = ctx.workspace(ctx.fallback_workspace_bytes(sdb, tds))
    code2 = torch.empty(n_te, dtype=torch.int32, device=dev)
    rp2 = torch.empty(n_te * CFG["k"], dtype=torch.float64, device=dev)

    def infer_with_fallback():
        _, _, fb2 = sur.infer(Zs, ood_threshold=thr, want_ood=True, masks=sdb.masks, k=CFG["k"], tau=CFG["tau"],
                              rec_code=code2, rec_pred=rp2, want_pred=False)
        refit = ctx.surrogate_fallback(sdb, tds, fb2, code2, rp2, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"],
                                       workspace=fws)
        return fb2, refit

    for _ in range(2):
        infer_with_fallback()
    torch.cuda.synchronize()
    fbk_ms = 0.0
    for _ in range(reps):
        flush.fill_(1)
        e0.record(stream)
        fb2, refit = infer_with_fallback()
        e1.record(stream)
        torch.cuda.synchronize()
        fbk_ms += e0.elapsed_time(e1)
    fbk_ms /= reps
    ctx.check_device_status()
    # agreement of the merged ranking with the plain method's own ranking of the same rows
    sout = rs.alloc_outputs(tds.n_test_rows, tds.n_splits, CFG["k"], dev, pred_all=False)
    ctx.cv_step(sdb, tds, ws, sout.rec_offsets, sout.rec_code, lam=CFG["lam"], k=CFG["k"], tau=CFG["tau"],
                rec_pred=sout.rec_pred)
    tm_te = tsp.train_masks.astype(np.uint64)
    tbits = ((tm_te[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)) == 0
    tver = (np.repeat(np.arange(P_te), 2)[:, None] * 64 + np.arange(64)[None, :])[tbits]
    plain_code = np.empty(n_te, dtype=np.int32)
    plain_code[tver] = sout.rec_code.cpu().numpy()
    merged = code2.cpu().numpy()
    flg = fb2.cpu().numpy().astype(bool)
    fallback = {"workload": "the 1,000,000 held-out vectors with 5 % of their programs holding 3 versions "
                            "whose counters are all scaled by e^4 (anomalous profiles)",
                "value_with_plain_fallback": n_te / (fbk_ms * 1e-3), "unit": UNIT, "ms": fbk_ms,
                "fallback_fraction": float(flg.mean()), "programs_refitted": refit[0],
                "versions_refitted": refit[1], "programs_shifted": int(len(sprogs)),
                "rec_code_equal_to_plain": {"all_rows": float(np.mean(merged == plain_code)),
                                            "flagged_rows": float(np.mean(merged[flg] == plain_code[flg]))
                                            if flg.any() else None,
                                            "unflagged_rows": float(np.mean(merged[~flg] == plain_code[~flg]))}}
    return {"workload": "surrogate MLP 256-512-512-6: train 2,000,000 vectors (31,250 programs x 64 "
                        "versions, labels = plain ridge CV predictions), infer 1,000,000 held-out vectors",
            "value": rate_s, "unit": UNIT, "infer_ms": inf_ms, "train_ms": train_ms,
            "train_steps": steps, "batch_rows": 8192, "loss_first": float(lc[0]), "loss_last": float(lc[-1]),
            "plain_batched_same_rows": {"value": rate_p, "ms": plain_ms},
            "speedup_vs_plain_batched": rate_s / rate_p,
            "ood_threshold": thr, "fallback_fraction": fb_frac, "value_with_plain_fallback": fallback["value_with_plain_fallback"],
            "plain_fallback": fallback,
            "accuracy": {"surrogate_sign": s_sign, "surrogate_top1": s_top1, "plain_sign": p_sign,
                         "plain_top1": p_top1, "mae_vs_plain_log_speedup": mae},
            "data_gen_s": gen_s}


def run_e2e(rs, ctx, batch, splits, dev, stream, flush, args, R):
    """End to end through rs_cv_step with host buffers, as a stream of batches: every step
    copies its inputs from pinned host memory, flushes L2, computes, and brings its
    recommendations back into pinned host memory -- rec_code and the reported predictions
    packed back to back (RS_PACK_PRED: ~1.2 values per row instead of k = 3, ~73 MB per step
    instead of ~150) -- with the counters.  Inputs and outputs are double-buffered: step i + 1's
    inputs arrive and step i - 1's results leave on two more streams while step i computes.  The timed region runs from the
    first step's input copy to the last step's results landing in host memory; ms_per_step is
    that time over the steps."""
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    fo = np.zeros(batch.n_programs + 1, np.int64)
    fo[1:] = np.cumsum(batch.feat_width.astype(np.int64))
    host = dict(X=pin(batch.X), row_offsets=pin(batch.row_offsets.astype(np.int64)),
                feat_width=pin(batch.feat_width.astype(np.int32)),
                x_offsets=pin(batch.x_offsets.astype(np.int64)), feat_offsets=pin(fo),
                masks=pin(batch.masks), log_time=pin(batch.log_time), cycles=pin(batch.cycles),
                split_offsets=pin(splits.split_offsets.astype(np.int64)),
                train_masks=pin(splits.train_masks.view(np.int64)))
    # inputs and outputs double-buffered: set b serves steps b, b + 2, ...
    devbs = [{k: torch.empty_like(v, device=dev) for k, v in host.items()} for _ in range(2)]

    def views(devb):
        db = rs.DeviceBatch(n_programs=batch.n_programs, dtype=rs.RS_F32, n_rows=batch.n_rows,
                            max_versions=64, max_feat=int(batch.feat_width.max()),
                            x_elems=int(batch.X.shape[0]), feat_total=int(fo[-1]),
                            row_offsets=devb["row_offsets"], feat_width=devb["feat_width"],
                            x_offsets=devb["x_offsets"], feat_offsets=devb["feat_offsets"],
                            X=devb["X"], masks=devb["masks"], log_time=devb["log_time"],
                            cycles=devb["cycles"])
        ds = rs.DeviceSplits(n_splits=splits.n_splits, max_train=int(CFG["versions"][1]) // 2 + 1,
                             split_offsets=devb["split_offsets"], train_masks=devb["train_masks"],
                             n_test_rows=R)
        return db, ds

    vw = [views(d) for d in devbs]
    ws = torch.empty(ctx.cv_workspace_bytes(*vw[0]), dtype=torch.uint8, device=dev)
    k = CFG["k"]
    outs = [rs.alloc_outputs(R, splits.n_splits, k, dev, pred_all=False) for _ in range(2)]
    h_code = [torch.empty(R, dtype=torch.int32).pin_memory() for _ in range(2)]
    h_pred = [torch.empty(R * k, dtype=torch.float64).pin_memory() for _ in range(2)]
    h_cnt = [torch.empty(16, dtype=torch.int64).pin_memory() for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    cs = torch.cuda.Stream(dev)                # device -> host copies
    ins = torch.cuda.Stream(dev)               # host -> device copies of the next step's inputs
    computed = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    loaded = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    moved = [0]
    # the step of each buffer set as one CUDA graph (rs_cv_graph_create, packed predictions)
    for devb in devbs:
        for k_, v in host.items():
            devb[k_].copy_(v, non_blocking=True)
    graphs = [ctx.cv_graph(vw[b][0], vw[b][1], ws, outs[b].rec_offsets, outs[b].rec_code, lam=CFG["lam"], k=k,
                           tau=CFG["tau"], flags=rs.RS_PACK_PRED, rec_pred=outs[b].rec_pred,
                           counters=outs[b].counters) for b in range(2)]

    def load(i):
        # step i's inputs, on their own stream once step i - 2 (the same set) has computed
        b = i % 2
        ins.wait_event(computed[b])
        with torch.cuda.stream(ins):
            for k_, v in host.items():
                devbs[b][k_].copy_(v, non_blocking=True)
        loaded[b].record(ins)

    def step(i):
        b = i % 2
        o = outs[b]
        stream.wait_event(loaded[b])
        flush.fill_(1)
        stream.wait_event(copied[b])           # this output set's previous copy has landed
        o.counters.zero_()
        graphs[b].launch()
        h_cnt[b].copy_(o.counters, non_blocking=True)
        computed[b].record(stream)

    def bring_back(i):
        # issued after step i + 1 is queued: the host waits for step i's counters (the packed
        # length) while the device works on step i + 1
        b = i % 2
        o = outs[b]
        computed[b].synchronize()
        total = int(h_cnt[b][4].item())
        cs.wait_event(computed[b])
        with torch.cuda.stream(cs):
            h_code[b].copy_(o.rec_code, non_blocking=True)
            h_pred[b][:total].copy_(o.rec_pred[:total], non_blocking=True)
        copied[b].record(cs)
        moved[0] += R * 4 + total * 8 + 16 * 8

    def run(n_steps):
        ins.wait_stream(stream)                # the first input copy starts inside the region
        load(0)
        for i in range(n_steps):
            if i + 1 < n_steps:
                load(i + 1)                    # beside step i's compute
            step(i)
            if i > 0:
                bring_back(i - 1)
        bring_back(n_steps - 1)

    for b in range(2):
        copied[b].record(cs)
        computed[b].record(stream)
    run(3)
    torch.cuda.synchronize()
    moved[0] = 0
    # a stream of 40 batches: the pipeline's fill (the first input copy) and drain (the last
    # output copy) are inside the region, once
    n = max(4, min(args.steps, 40))
    e0.record(stream)
    run(n)
    for b in range(2):
        stream.wait_event(copied[b])
    e1.record(stream)
    torch.cuda.synchronize()
    tot = e0.elapsed_time(e1)
    ctx.check_device_status()
    for g in graphs:
        g.close()
    d2h = moved[0] / n
    # the host link's own rates (one bulk copy each way of a step's output size), the bound of
    # this leg: a step cannot finish before its outputs have crossed the link
    big_d = outs[0].rec_pred
    reps, t_d2h, t_h2d = 3, 0.0, 0.0
    for _ in range(reps):
        e0.record(stream)
        h_pred[0].copy_(big_d, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t_d2h += e0.elapsed_time(e1)
        e0.record(stream)
        big_d.copy_(h_pred[0], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t_h2d += e0.elapsed_time(e1)
    nb = big_d.numel() * 8
    d2h_gbs, h2d_gbs = nb * reps / (t_d2h * 1e6), nb * reps / (t_h2d * 1e6)
    return {"value": R * n / (tot / 1e3), "unit": UNIT, "ms_per_step": tot / n, "steps": n,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "host_link_gbs": {"d2h": d2h_gbs, "h2d": h2d_gbs},
            "copy_bound_ms_per_step": d2h / (d2h_gbs * 1e6) + h2d / (h2d_gbs * 1e6),
            "path": "per step: pinned host -> device copies of the inputs (on a third stream, beside the "
                    "previous step's compute), L2 flush, the step as one CUDA-graph launch "
                    "(rs_cv_graph_create with packed predictions, RS_PACK_PRED), device -> pinned "
                    "host copies of rec_code, the packed "
                    "predictions and the counters on a second stream (outputs double-buffered: a step's "
                    "copies overlap the next step's compute)"}


if __name__ == "__main__":
    sys.exit(main())
