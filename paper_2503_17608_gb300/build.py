"""Build the CUDA library libceler_gb.so in-tree for sm_103a (GB300).

Each translation unit is compiled in parallel with nvcc, then linked into
one shared library exposing the C ABI of include/celer_gb.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libceler_gb.so")
# diagnostic variant: the same library with the active-lane counters compiled in
LANES_BUILD = os.path.join(HERE, "_build_lanes")
LANES_LIB = os.path.join(HERE, "libceler_gb_lanes.so")
SOURCES = ["step.cu", "tables.cu", "driver.cu", "debug.cu", "noalloc.cu", "serve.cu"]
HEADERS = ["common.cuh", "physics.cuh", "fastmath.cuh", "launch.h", "tables.h", "block_pass.cuh", "async_loop.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None, lanes: bool = False) -> str:
    """Compile the library (lanes=True: the diagnostic variant with the
    active-lane counters, libceler_gb_lanes.so); returns its path."""
    build_dir, lib = (LANES_BUILD, LANES_LIB) if lanes else (BUILD, LIB)
    if lanes:
        extra_flags = list(extra_flags or []) + ["-DCELER_LANE_COUNTERS"]
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "celer_gb.h")]
    common = [nvcc(), "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              "-Xptxas", "-warn-spills"] + list(extra_flags or [])
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append(common + ["-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs):
        run([nvcc(), "-shared", *ARCH, "-o", lib + ".tmp", *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"])
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, lanes="--lanes" in sys.argv))
