"""Build the sm_103a shared library ``_build/libcts.so`` in-tree with nvcc.

The translation units are compiled in parallel (kernels, runtime, host
planner, no-alloc field) and linked into one shared object with the static
CUDA runtime, so the library loads on machines without a GPU driver (its
entry points then report SIM_ENODEV).  Only sm_103a code is generated.

``build(checked=True)`` makes the checked build ``_build_checked/
libcts_checked.so`` from the same sources with -DCTS_BOUNDS_CHECK: device
index checks that record an error and skip the access (the calls then fail
with SIM_ECUDA), for debugging without a sanitizer.  The package loads it
instead of the default library when CTS_CHECKED=1 is set in the environment.
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
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libcts_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["cts_kernels.cu", "cts_runtime.cu", "cts_host.cpp", "cts_noalloc.cu"]
HEADERS = ["cts_internal.h", "cts_host_impl.h"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcts.so")


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra: list[str], out_dir: str) -> str:
    obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", CSRC, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
               "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return obj


def build(force: bool = False, extra: list[str] | None = None, checked: bool = False) -> str:
    """Compile (if stale) and return the path of libcts.so (or, checked=True,
    of the bounds-checked libcts_checked.so)."""
    out_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    extra = list(extra or []) + (["-DCTS_BOUNDS_CHECK"] if checked else [])
    try:
        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(lambda s: _compile(s, extra, out_dir), SOURCES))
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs,
                        "-lpthread", "-ldl"], check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as e:
        raise RuntimeError(f"libcts build failed:\n{' '.join(e.cmd)}\n{e.stdout}\n{e.stderr}") from e
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, checked="--checked" in sys.argv[1:]))
