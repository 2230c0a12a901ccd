"""Build ``libmp.so`` (the CUDA library behind include/mp.h) in-tree.

Several translation units (the host API and one per group of sweep kernels),
compiled in parallel by nvcc for sm_103a only and linked into one library:
    nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo -c ...
    nvcc -shared ... -o libmp.so
The result lands in ``paper_1901_05708_gb300/_build/libmp.so``; it is rebuilt
when any source under ``csrc/`` or ``include/mp.h`` is newer.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libmp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmp")


def units() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def sources() -> list[str]:
    return sorted(units() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + [os.path.join(INCLUDE, "mp.h")])


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in sources())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile every translation unit (in parallel) and link libmp.so.
    `extra` adds nvcc flags (e.g. -Xptxas -v) to every compile."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tag = f".tmp{os.getpid()}"
    objs, procs = [], []
    for cu in units():
        obj = os.path.join(BUILD, os.path.basename(cu)[:-3] + tag + ".o")
        cmd = [nvcc(), *ARCH, *FLAGS, *(extra or []), "-I", INCLUDE, "-c", cu, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    log, failed = [], None
    for cmd, pr in procs:
        out, _ = pr.communicate()
        log.append(out)
        if pr.returncode != 0 and failed is None:
            failed = (cmd, out)
    try:
        if failed:
            raise RuntimeError("nvcc failed:\n" + " ".join(failed[0]) + "\n" + failed[1])
        tmp = LIB + tag
        cmd = [nvcc(), *ARCH, "-shared", *objs, "-o", tmp]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
        if verbose:
            print("".join(log) + res.stdout + res.stderr)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra=sys.argv[1:]))
