"""Build the CUDA library in-tree for sm_103a (GB300).

``python -m paper_2004_13475_gb300.build`` compiles every translation unit of
``csrc/`` in parallel with nvcc and links ``libfractal.so`` beside this file.
The input generator's device twin (``synth/libsynth.so``) is built by the same
routine because GPU tests and the benchmark need it; it shares no source with
the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from typing import List, Optional

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfractal.so")
SYNTH_SRC = os.path.join(ROOT, "synth", "synth.cu")
SYNTH_LIB = os.path.join(ROOT, "synth", "libsynth.so")
EXPORTS_MAP = os.path.join(CSRC, "exports.map")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                 "-Xcompiler", "-Wall", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources() -> List[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers() -> List[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "fractal.h"))
    return hs


def _stale(target: str, deps: List[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd: List[str], log: Optional[str] = None) -> None:
    res = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if log:
        with open(log, "w") as f:
            f.write(" ".join(cmd) + "\n" + res.stdout)
    if res.returncode != 0:
        raise RuntimeError(f"command failed ({res.returncode}): {' '.join(cmd)}\n{res.stdout}")


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile (if stale) and return the path of libfractal.so."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    hdrs = _headers()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc] + CFLAGS + ["-I", os.path.join(ROOT, "include"), "-c", s, "-o", o]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append((cmd, o + ".log"))
    synth_job = None
    if force or _stale(SYNTH_LIB, [SYNTH_SRC]):
        synth_job = ([nvcc] + CFLAGS + ["-shared", SYNTH_SRC, "-o", SYNTH_LIB], None)
    workers = max(1, min(len(jobs) + 1, os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(_run, c, l) for c, l in jobs]
        if synth_job:
            futs.append(ex.submit(_run, *synth_job))
        for f in futs:
            f.result()
    if force or jobs or _stale(LIB, objs + [EXPORTS_MAP]):
        # export the C ABI only (the library's internal C++ symbols stay local)
        _run([nvcc] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart", "-Xlinker",
                                                              "--version-script=" + EXPORTS_MAP])
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
