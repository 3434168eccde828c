"""Build the TILD CUDA library in-tree for sm_103a (nvcc, no cmake).

Sources under ``csrc/`` are compiled in parallel and linked into
``_lib/libtild.so`` next to this file. Nothing is installed elsewhere.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from typing import List

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(OUT_DIR, "libtild.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -split-compile=0: the device code of each translation unit is optimised in
# parallel jobs (one per core), which keeps the build to a few minutes
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-split-compile=0", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or put the CUDA toolkit on PATH)")


def sources() -> List[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target: str, deps: List[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


DEBUG_LIB_PATH = os.path.join(OUT_DIR, "libtild_debug.so")


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every .cu under csrc/ and link libtild.so; returns its path.
    debug=True builds libtild_debug.so instead, with the kernels' bounds
    checks on (-DTILD_DEBUG=1: a failed check records a flag and skips the
    access; the next synchronising call returns TILD_EDEVICE)."""
    out_dir = os.path.join(OUT_DIR, "debug") if debug else OUT_DIR
    lib_path = DEBUG_LIB_PATH if debug else LIB_PATH
    os.makedirs(out_dir, exist_ok=True)
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "tild.h"))
    nvcc = _nvcc()
    flags = FLAGS + (["-DTILD_DEBUG=1"] if debug else [])
    objs, procs = [], []
    for s in srcs:
        o = os.path.join(out_dir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc, *ARCH, *flags, "-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(f"{os.path.basename(s)}:\n{out}")
        elif verbose and out.strip():
            print(out, file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    if force or procs or _stale(lib_path, objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", lib_path, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
