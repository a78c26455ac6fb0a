"""Tier 1 of the tool (Sec. 2) on this GPU: profile the 64 versions of the n-body code NB
(nbody.cu, the six optimizations of Sec. 3.3 as compile-time switches) and write the feature
vectors and run times that the speedup-prediction path trains and tests on.

For each input of Table 1's NB column (bodies halved for this GPU: 25,000 / 50,000 / 50,000 /
100,000 bodies over 2 / 2 / 5 / 5 time steps) and each of three runs (Sec. 5: every version
was profiled three times per input):
  * the run time of every version: the median of 5 timed runs of the whole input (CUDA events);
  * its hardware counters: one profiled time step of the force-and-update kernel per body
    count, captured by Nsight Compute (one invocation per version, three launches, a fixed
    list of raw counters), each counter divided by the kernel's elapsed SM cycles (Sec. 2:
    counters normalised by the cycle count).
Inputs with the same body count share their profiled time step within a run.

Run on the GPU machine from the repository root:
    python -m paper_1910_07776_gb300.tier1.capture out/nb_gb300.npz
and copy the file next to this script as nb_gb300.npz.  Needs nvcc and ncu on PATH."""
from __future__ import annotations

import csv
import io
import os
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
EXE = os.path.join(HERE, "_build", "nbody")
INPUTS = [(25000, 2), (50000, 2), (50000, 5), (100000, 5)]
RUNS = 3
TIME_REPS = 5
CYCLES = "sm__cycles_elapsed.max"
COUNTERS = [
    "smsp__inst_executed.sum", "smsp__thread_inst_executed.sum",
    "smsp__sass_thread_inst_executed_op_fadd_pred_on.sum",
    "smsp__sass_thread_inst_executed_op_fmul_pred_on.sum",
    "smsp__sass_thread_inst_executed_op_ffma_pred_on.sum",
    "smsp__sass_thread_inst_executed_op_fp32_pred_on.sum",
    "smsp__sass_thread_inst_executed_op_integer_pred_on.sum",
    "smsp__sass_thread_inst_executed_op_conversion_pred_on.sum",
    "smsp__inst_executed_pipe_xu.sum", "smsp__inst_executed_pipe_fma.sum",
    "smsp__inst_executed_pipe_fmaheavy.sum", "smsp__inst_executed_pipe_alu.sum",
    "smsp__inst_executed_pipe_lsu.sum", "smsp__inst_executed_pipe_uniform.sum",
    "smsp__inst_executed_pipe_cbu.sum", "smsp__inst_executed_pipe_adu.sum",
    "smsp__sass_inst_executed_op_branch.sum", "smsp__sass_branch_targets_threads_divergent.sum",
    "smsp__sass_inst_executed_op_global_ld.sum", "smsp__sass_inst_executed_op_global_st.sum",
    "smsp__sass_inst_executed_op_shared_ld.sum", "smsp__sass_inst_executed_op_shared_st.sum",
    "smsp__sass_inst_executed_op_memory_32b.sum", "smsp__sass_inst_executed_op_memory_128b.sum",
    "smsp__inst_executed_op_ldc.sum", "idc__requests.sum",
    "l1tex__t_requests_pipe_lsu_mem_global_op_ld.sum", "l1tex__t_sectors_pipe_lsu_mem_global_op_ld.sum",
    "l1tex__data_pipe_lsu_wavefronts_mem_shared.sum", "l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum",
    "lts__t_sectors.sum", "dram__bytes_read.sum", "smsp__warps_launched.sum", "sm__ctas_launched.sum",
    "smsp__warps_active.sum", "smsp__cycles_active.sum", "smsp__issue_active.sum",
]


def build() -> str:
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    src = os.path.join(HERE, "nbody.cu")
    if not os.path.exists(EXE) or os.path.getmtime(EXE) < os.path.getmtime(src):
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                               "-lineinfo", "-o", EXE, src])
    return EXE


def run_times(exe):
    """[run][input][mask] median milliseconds."""
    out = np.zeros((RUNS, len(INPUTS), 64))
    for r in range(RUNS):
        for i, (n, steps) in enumerate(INPUTS):
            txt = subprocess.check_output([exe, "time", str(n), str(steps), str(TIME_REPS)], text=True)
            for row in csv.DictReader(io.StringIO(txt)):
                out[r, i, int(row["mask"])] = float(row["ms_median"])
    return out


def _value(s):
    return float(s.replace(",", ""))


def profile(exe, mask, bodies):
    """{bodies: {metric: value}} for one version (one Nsight Compute invocation)."""
    cmd = ["ncu", "--clock-control", "none", "--csv", "--metrics", ",".join([CYCLES] + COUNTERS),
           "-k", "regex:nbody_step", "-c", str(len(bodies)), exe, "profile", str(mask), *map(str, bodies)]
    txt = subprocess.check_output(cmd, text=True, stderr=subprocess.DEVNULL)
    lines = [ln for ln in txt.splitlines() if ln.startswith('"')]
    rows = list(csv.DictReader(io.StringIO("\n".join(lines))))
    by_id = {}
    for row in rows:
        by_id.setdefault(int(row["ID"]), {})[row["Metric Name"]] = _value(row["Metric Value"])
    ids = sorted(by_id)
    if len(ids) != len(bodies):
        raise RuntimeError(f"mask {mask}: expected {len(bodies)} profiled launches, got {len(ids)}")
    return {n: by_id[i] for n, i in zip(bodies, ids)}


def main(out_path):
    exe = build()
    t0 = time.time()
    times = run_times(exe)
    bodies = sorted(set(n for n, _ in INPUTS))
    for mask in range(64):      # every command the profiler will run, first without it
        subprocess.check_call([exe, "profile", str(mask), *map(str, bodies)])
    feats = np.zeros((RUNS, len(INPUTS), 64, len(COUNTERS)))
    cycles = np.zeros((RUNS, len(INPUTS), 64))
    for r in range(RUNS):
        for mask in range(64):
            prof = profile(exe, mask, bodies)
            for i, (n, _) in enumerate(INPUTS):
                c = prof[n][CYCLES]
                cycles[r, i, mask] = c
                feats[r, i, mask] = [prof[n][m] / c for m in COUNTERS]
    gpu = subprocess.check_output(["nvidia-smi", "--query-gpu=name,driver_version", "--format=csv,noheader"],
                                  text=True).strip()
    if os.path.dirname(out_path):
        os.makedirs(os.path.dirname(out_path), exist_ok=True)
    np.savez_compressed(out_path, features=feats, cycles=cycles, time_ms=times,
                        inputs=np.array(INPUTS), counters=np.array(COUNTERS), cycles_metric=CYCLES,
                        gpu=gpu, seconds=time.time() - t0,
                        command="python -m paper_1910_07776_gb300.tier1.capture " + out_path)
    print(f"wrote {out_path}: {feats.shape} features, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "nb_gb300.npz")
