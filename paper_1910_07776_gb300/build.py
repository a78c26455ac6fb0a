"""Builds ``_build/librs.so`` from ``csrc/*.cu`` for sm_103a with nvcc (in-tree, no cmake).

Each translation unit compiles in its own nvcc process (in parallel), then one nvcc call
links the shared library with the CUDA runtime linked statically.  ``-Xptxas -v`` output
(registers, spills, shared memory) is kept in ``_build/ptxas.log``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
SO = os.path.join(OUT, "librs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(srcs, target) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(HERE, "..", "include", "rs.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def write_log_table(path: str) -> None:
    """Constants of the table-driven logarithm of the standardization kernel, correctly
    rounded to FP64 from exact decimal arithmetic (the same values on every build machine):
    log F_i and 1 / F_i for the centres F_i = 1 + (2 i + 1) / 512 of the 256 intervals of
    width 1/256 that split the mantissa range [1, 2); ln 2; and log(1e-30), the clamp value."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    lines = ["// generated by build.py (write_log_table): do not edit", "#pragma once", ""]
    logs, invs = [], []
    for i in range(256):
        F = Decimal(1) + Decimal(2 * i + 1) / Decimal(512)
        logs.append(float(F.ln()).hex())
        invs.append(float(Decimal(1) / F).hex())
    ln2 = Decimal(2).ln()
    eps = Decimal(1e-30)                 # the FP64 value nearest 1e-30, exactly
    lines.append("__device__ const double kLogTabF[256] = {" + ", ".join(logs) + "};")
    lines.append("__device__ const double kLogTabInv[256] = {" + ", ".join(invs) + "};")
    lines.append(f"constexpr double kLn2 = {float(ln2).hex()};")
    lines.append(f"constexpr double kLogClamp = {float(eps.ln()).hex()};   // log(1e-30)")
    txt = "\n".join(lines) + "\n"
    if not os.path.exists(path) or open(path).read() != txt:
        with open(path, "w") as f:
            f.write(txt)


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if not force and not _stale(srcs, SO):
        return SO
    os.makedirs(OUT, exist_ok=True)
    write_log_table(os.path.join(OUT, "rs_log_table.h"))
    nv = nvcc()

    def one(src):
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + ".o")
        cmd = [nv, *ARCH, *FLAGS, "-I", OUT, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        res = list(ex.map(one, srcs))
    with open(os.path.join(OUT, "ptxas.log"), "w") as f:
        for (obj, log), src in zip(res, srcs):
            f.write(f"==== {os.path.basename(src)}\n{log}\n")
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *[o for o, _ in res], "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO)
    if verbose:
        print(open(os.path.join(OUT, "ptxas.log")).read())
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
