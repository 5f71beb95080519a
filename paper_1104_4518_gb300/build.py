"""Builds libbfs_gb300.so in-tree with nvcc for sm_103a (GB300).

Each .cu under csrc/ is compiled to an object in parallel, then the objects
are linked into one shared library whose only interface is the C ABI of
include/bfs.h.  No PyTorch headers or libraries are involved.  build_all()
also builds the bounds-checking library libbfs_gb300_checked.so (the same
sources with -DBFS_BOUNDS_CHECK), at the same time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbfs_gb300.so")
CHECKED_LIB = os.path.join(PKG, "libbfs_gb300_checked.so")
CHECKED_BUILD_DIR = os.path.join(PKG, "_build_checked")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          ptxas_verbose: bool = False, lib_path: str = LIB, build_dir: str = BUILD_DIR) -> str:
    """Compiles and links the library if any source is newer than it; returns its path.

    `extra_flags`, `lib_path` and `build_dir` let a diagnostic variant be built
    elsewhere without touching the product library."""
    LIB_OUT = lib_path
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "bfs.h"))
    srcs = sources()
    flags = NVCC_FLAGS + (extra_flags or []) + (["-Xptxas", "-v"] if ptxas_verbose else [])
    objs = []
    jobs = []
    for src in srcs:
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc(), *ARCH, *flags, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(run, jobs))
    failed = [(c, r) for c, r in results if r.returncode != 0]
    for c, r in results:
        if verbose or ptxas_verbose or r.returncode != 0:
            sys.stderr.write(f"$ {' '.join(c)}\n{r.stdout}{r.stderr}")
    if failed:
        raise RuntimeError(f"nvcc failed for {[os.path.basename(c[-3]) for c, _ in failed]}")
    if force or jobs or _stale(LIB_OUT, objs):
        tmp = LIB_OUT + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(f"$ {' '.join(cmd)}\n{r.stdout}{r.stderr}")
            raise RuntimeError("linking libbfs_gb300.so failed")
        os.replace(tmp, LIB_OUT)
    return LIB_OUT


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The bounds-checking library (every index checked on the device, BFS_ERR_BOUNDS)."""
    return build(force=force, verbose=verbose, extra_flags=["-DBFS_BOUNDS_CHECK"], lib_path=CHECKED_LIB,
                 build_dir=CHECKED_BUILD_DIR)


def build_all(force: bool = False, verbose: bool = False) -> list[str]:
    """Both libraries, compiled side by side."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, force, verbose), ex.submit(build_checked, force, verbose)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    if "--ptxas" in sys.argv:
        build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_verbose=True)
        print(LIB)
    else:
        print("\n".join(build_all(force="--force" in sys.argv, verbose="-v" in sys.argv)))
