"""Build libkc.so in-tree: CUDA sources for sm_103a plus host C++, compiled in parallel."""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libkc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr", "-I", INCLUDE]

_lock = threading.Lock()


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkc")


def sources():
    cu = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every source and link libkc.so; returns its path."""
    with _lock:
        if not force and up_to_date():
            return LIB
        nvcc = _nvcc()
        os.makedirs(BUILD, exist_ok=True)
        cu, cpp = sources()
        jobs = []
        for src in cu:
            obj = os.path.join(BUILD, os.path.basename(src) + ".o")
            extra = ["-Xptxas", "-v"] if ptxas_info else []
            jobs.append(([nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj], obj))
        for src in cpp:
            obj = os.path.join(BUILD, os.path.basename(src) + ".o")
            jobs.append((["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I", INCLUDE, "-c", src, "-o", obj], obj))

        def run(cmd):
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
            return r.stdout + r.stderr

        with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
            logs = list(ex.map(run, [c for c, _ in jobs]))
        if verbose or ptxas_info:
            for (cmd, _), log in zip(jobs, logs):
                if log.strip():
                    print(os.path.basename(cmd[-3]), log, sep="\n")
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-lpthread"])
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
