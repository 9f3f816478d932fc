"""Builds the CUDA library ``libtheseus_gb.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` file compiles to an object in parallel; the objects link
into one shared library exporting the ``tp_*`` C ABI of
``include/theseus_gb.h``.  Only the CUDA runtime is linked (statically);
NVRTC, for plan-specialised kernels, is loaded at run time when present.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libtheseus_gb.so")
BUILD_DIR = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtheseus_gb.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _sources() + _headers() + [__file__])


# Device headers embedded in the library for run-time (NVRTC) compilation of
# plan-specialised kernels, in include order.
JIT_HEADERS = ["kernels.cuh", "device.cuh", "pipeline.cuh", "jit_common.cuh", "jit_dense.cuh", "jit_batch.cuh"]


def _write_jit_sources() -> None:
    """Writes _build/jit_sources.inc: the JIT headers as C++ raw strings."""
    parts = ["struct JitSource { const char* name; const char* text; };",
             "const JitSource kJitSources[] = {"]
    for name in JIT_HEADERS:
        with open(os.path.join(CSRC, name)) as f:
            text = f.read()
        if ')TPJIT"' in text:
            raise RuntimeError(f"{name} contains the raw-string delimiter")
        parts.append(f'    {{"{name}", R"TPJIT({text})TPJIT"}},')
    parts.append("};")
    out = os.path.join(BUILD_DIR, "jit_sources.inc")
    new = "\n".join(parts) + "\n"
    if os.path.exists(out):
        with open(out) as f:
            if f.read() == new:
                return
    with open(out, "w") as f:
        f.write(new)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    _write_jit_sources()
    srcs = _sources()
    objs = [os.path.join(BUILD_DIR, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-I", BUILD_DIR, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose:
        for log in logs:
            if log.strip():
                print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-cudart", "static", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else ()))
