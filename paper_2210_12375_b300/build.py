"""Builds ``libtode.so`` in-tree with nvcc for sm_103a (B300).

Every translation unit is compiled separately, side by side (the solver
units with ``-fmad=false``), and linked into one shared library with the CUDA runtime
linked statically; no other library is linked.  Rebuilds only what changed.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtode.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
          "--expt-relaxed-constexpr"]

# translation unit -> extra flags
UNITS = {
    "tode_api.cu": [],
    "tode_simt_f64.cu": ["-fmad=false"],
    "tode_simt_f32.cu": ["-fmad=false"],
    "tode_simt_ts5_f64.cu": ["-fmad=false"],
    "tode_simt_ts5_f32.cu": ["-fmad=false"],
    "tode_static.cu": [],
    "tode_tc_gemm.cu": [],
    "tode_mlp.cu": ["-fmad=false"],
    "tode_mlp_tb.cu": [],
    "tode_peak.cu": [],
}


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(INCLUDE, "tode.h"))
    return max(os.path.getmtime(h) for h in hdrs)


def build(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    hdr_time = _deps()
    objs, cmds = [], []
    changed = force or not os.path.exists(LIB)
    for src, extra in UNITS.items():
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".o"))
        objs.append(o)
        if (not force and os.path.exists(o)
                and os.path.getmtime(o) >= max(os.path.getmtime(s), hdr_time)):
            continue
        cmd = [NVCC, *ARCH, *COMMON, *extra, "-c", s, "-o", o]
        if ptxas_verbose:
            cmd += ["-Xptxas", "-v"]
        cmds.append(cmd)
    # the units are independent: compile them side by side
    jobs = max(1, min(len(cmds), os.cpu_count() or 1))
    running = []
    for cmd in cmds:
        if verbose:
            print(" ".join(cmd), flush=True)
        running.append(subprocess.Popen(cmd))
        while len(running) >= jobs:
            _reap(running)
    while running:
        _reap(running)
    changed = changed or bool(cmds)
    if changed or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs,]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def _reap(running: list) -> None:
    """Waits for the oldest compile of the list; a failed one raises (after
    the others have finished, so that no object is left half written)."""
    p = running.pop(0)
    if p.wait() != 0:
        for q in running:
            q.wait()
        raise subprocess.CalledProcessError(p.returncode, p.args)


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv)
    print(LIB)
