"""In-tree build of libflashstep.so for sm_103a (nvcc, one -gencode, the
translation units compiled in parallel and linked into one shared library),
and of its bounds-checked twin libflashstep_bounds.so (FS_DEBUG_BOUNDS: the
step kernels check the indices of their main accesses and report the first
one out of range), used by the failure-detection tests."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB_NORMAL = os.path.join(OUT_DIR, "libflashstep.so")
LIB_BOUNDS = os.path.join(OUT_DIR, "libflashstep_bounds.so")
# FLASHSTEP_DEBUG_BOUNDS=1 makes the binding load the bounds-checked library
LIB = LIB_BOUNDS if os.environ.get("FLASHSTEP_DEBUG_BOUNDS") == "1" else LIB_NORMAL

SOURCES = ["fs_api.cu", "fs_step.cu", "fs_push.cu", "fs_markov.cu", "fs_ingest.cu", "fs_pack.cu", "fs_pack_api.cu", "fs_server.cpp",
           "fs_tune.cpp", "fs_alloc.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "fs.h"))
    files.append(os.path.abspath(__file__))
    return files


def is_fresh() -> bool:
    for lib in (LIB_NORMAL, LIB_BOUNDS):
        if not os.path.exists(lib):
            return False
        t = os.path.getmtime(lib)
        if not all(os.path.getmtime(f) <= t for f in _deps()):
            return False
    return True


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds both libraries (all translation units of both in one parallel
    pool) and returns the path of the one the binding loads."""
    if not force and is_fresh():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    variants = [(LIB_NORMAL, "", []), (LIB_BOUNDS, "_bounds", ["-DFS_DEBUG_BOUNDS"])]

    def compile_one(job) -> tuple[str, str]:
        src, suffix, defs = job
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + suffix + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {' '.join(defs)}:\n{p.stdout}\n{p.stderr}")
        return obj, p.stderr

    jobs = [(src, suffix, defs) for _, suffix, defs in variants for src in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), max(os.cpu_count() or 1, len(SOURCES)))) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose:
        for _, log in results:
            print(log)
    for lib, suffix, _ in variants:
        objs = [os.path.join(OUT_DIR, os.path.splitext(src)[0] + suffix + ".o") for src in SOURCES]
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
