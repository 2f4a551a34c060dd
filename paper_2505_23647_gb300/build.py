"""Build the CUDA library in-tree: paper_2505_23647_gb300/_lib/libsclbm.so.

Translation units are compiled in parallel with nvcc for sm_103a only:
``fp64.cu``, ``noalloc.cu`` and ``observe.cu`` with ``-fmad=false`` (binary64 expressions
round exactly as written, the documented FP64 order), the binary32 and API
units with the defaults; the objects are linked into one shared library with the CUDA
runtime linked statically.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
SO = os.path.join(OUT_DIR, "libsclbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                 "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]
UNITS = {
    "api.cu": [],
    "fp64.cu": ["-fmad=false"],
    "fp32.cu": [],
    "fused3d.cu": [],
    "fused3d_tma.cu": [],
    "noalloc.cu": ["-fmad=false"],
    "observe.cu": ["-fmad=false"],
    "batch2d.cu": [],
    "adjoint.cu": [],
}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    return [u for u in UNITS if os.path.exists(os.path.join(CSRC, u))]


def _stale():
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "sclbm.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False, extra=()):
    """Compile and link the library; returns the .so path."""
    if not force and not _stale():
        return SO
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(OUT_DIR, unit.replace(".cu", ".o"))
        cmd = [nvcc, "-c", src, "-o", obj] + COMMON + UNITS[unit] + list(extra)
        if verbose:
            cmd.append("-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
        return obj, r.stderr

    units = _sources()
    with ThreadPoolExecutor(max_workers=len(units)) as ex:
        for obj, log in ex.map(compile_one, units):
            objs.append(obj)
            if verbose and log:
                sys.stderr.write(log)
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
