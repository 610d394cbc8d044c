"""Build the sm_103a shared library ``_build/libcts.so`` in-tree with nvcc.

Three translation units are compiled in parallel (kernels, runtime, host
planner) and linked into one shared object with the static CUDA runtime, so
the library loads on machines without a GPU driver (its entry points then
report SIM_ENODEV).  Only sm_103a code is generated.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcts.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["cts_kernels.cu", "cts_runtime.cu", "cts_host.cpp", "cts_noalloc.cu"]
HEADERS = ["cts_internal.h", "cts_host_impl.h"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcts.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", CSRC, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
               "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return obj


def build(force: bool = False, extra: list[str] | None = None) -> str:
    """Compile (if stale) and return the path of libcts.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    try:
        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs,
                        "-lpthread", "-ldl"], check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as e:
        raise RuntimeError(f"libcts build failed:\n{' '.join(e.cmd)}\n{e.stdout}\n{e.stderr}") from e
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
