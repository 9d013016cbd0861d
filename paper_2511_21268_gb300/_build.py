"""In-tree builds of the package's native libraries.

* ``inputs/libiga_gen.so`` -- the seeded IgA input generator (plain C, gcc).
* ``libamg_gb300.so``       -- the CUDA AMG-PCG library behind the C ABI of
  ``include/amg_gb300.h`` (nvcc, sm_103a only).

Each library is rebuilt only when one of its sources is newer than it.  The
build is deliberately short: one nvcc invocation per translation unit,
compiled in parallel, a single ``-gencode``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")

IGA_SRC = os.path.join(PKG, "inputs", "iga_gen.c")
IGA_LIB = os.path.join(PKG, "inputs", "libiga_gen.so")
AMG_LIB = os.path.join(PKG, "libamg_gb300.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)


def build_inputs(force: bool = False) -> str:
    if force or _stale(IGA_LIB, [IGA_SRC]):
        tmp = IGA_LIB + ".tmp"
        _run(["gcc", "-O3", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o", tmp, IGA_SRC, "-lm"])
        os.replace(tmp, IGA_LIB)
    return IGA_LIB


def cuda_sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def cuda_headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return sorted(hs)


def nvcc_flags(extra: list[str] | None = None) -> list[str]:
    flags = [
        GENCODE,
        "-O3",
        "-lineinfo",
        "-std=c++17",
        "-Xcompiler",
        "-fPIC",
        "-I" + INCLUDE,
        "-I" + CSRC,
        "--expt-relaxed-constexpr",
    ]
    if extra:
        flags += extra
    return flags


def build_cuda(force: bool = False, extra: list[str] | None = None, jobs: int | None = None) -> str:
    srcs = cuda_sources()
    deps = srcs + cuda_headers()
    if not force and not _stale(AMG_LIB, deps):
        return AMG_LIB
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    flags = nvcc_flags(extra)

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        _run([NVCC, *flags, "-c", src, "-o", obj])
        return obj

    with ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = AMG_LIB + ".tmp"
    _run([NVCC, GENCODE, "-shared", "-cudart", "static", "-o", tmp, *objs])
    os.replace(tmp, AMG_LIB)
    return AMG_LIB


def clean() -> None:
    for p in (IGA_LIB, AMG_LIB):
        if os.path.exists(p):
            os.remove(p)
    if os.path.isdir(BUILD):
        shutil.rmtree(BUILD)
