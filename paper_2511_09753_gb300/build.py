"""Build libspai.so in-tree with nvcc for sm_103a (no CMake).

Compiles the .cu files of ``csrc/`` in parallel into objects under
``_build/`` and links ``paper_2511_09753_gb300/libspai.so``.  Flags:
``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo --fmad=false``
(``--fmad=false`` keeps a*b+c unfused unless the code calls fma; the
method's arithmetic order depends on it).
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libspai.so")
SOURCES = ["colpass_f32.cu", "colpass_f64.cu", "colpass_hot.cu", "colpass_pi_f32.cu",
           "colpass_pi_f64.cu", "vec_kernels.cu", "bpcg.cu", "fixed_pattern.cu", "fpmr.cu",
           "dropping.cu", "api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC, "--expt-relaxed-constexpr",
                   "-extended-lambda"]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, variant: str = "") -> str:
    """Build libspai.so; variant="phase" builds libspai_phase.so instead, the
    same sources compiled with SPAI_PHASE_CLOCKS (per-phase clock64() counts
    in the column pass, read with spai_phase_clocks; a profiling build)."""
    if variant not in ("", "phase"):
        raise ValueError(variant)
    build_dir = BUILD + ("_" + variant if variant else "")
    lib_path = os.path.join(HERE, "libspai_phase.so") if variant else LIB
    extra = ["-DSPAI_PHASE_CLOCKS"] if variant == "phase" else []
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "spai.h"))
    cc = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([cc] + _flags() + extra + ["-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if verbose and (r.stdout or r.stderr):
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed: " + " ".join(j) + "\n" + r.stdout + r.stderr)
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt",
                           "-lpthread", "-ldl"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed\n" + r.stdout + r.stderr)
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv,
                variant="phase" if "--phase" in sys.argv else ""))
