"""Build liblbmhd.so (the C-ABI library) from csrc/ with nvcc for sm_103a, in-tree.

Usage: ``python -m paper_1705_09807_gb300.build [--verbose-ptxas]``.  The translation units
compile in parallel; the result is ``paper_1705_09807_gb300/liblbmhd.so``.  Only nvcc and the
host compiler are needed (no GPU), so the same command cross-builds here and builds natively on
the aarch64 GPU hosts.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbmhd.so")
SOURCES = ["lbmhd_step.cu", "lbmhd_aux.cu", "lbmhd_api.cu", "lbmhd_noalloc.cu", "lbmhd_analysis.cu",
           "lbmhd_ensemble.cu", "lbmhd_closure.cu", "lbmhd_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbmhd.so")


def common_flags(extra=()) -> list:
    return ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O2",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, *common_flags(extra)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "lbmhd.h"))
    deps.append(os.path.abspath(__file__))
    return all(os.path.getmtime(d) <= t for d in deps)


def _build(lib: str, build_dir: str, extra) -> str:
    os.makedirs(build_dir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-o", tmp, *objs, *ARCH, "-cudart", "static", "-lrt", "-ldl",
           "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not verbose_ptxas and up_to_date():
        return LIB
    return _build(LIB, BUILD, ["-Xptxas", "-v"] if verbose_ptxas else [])


CHECK_LIB = os.path.join(PKG, "liblbmhd_check.so")


def build_checked(force: bool = False) -> str:
    """The bounds-checking variant of the library (-DLBMHD_BOUNDS_CHECK), beside the normal one:
    the step kernels check their shared-memory, global-memory and copy indices, skip any access
    that fails and set a flag that the next synchronising call reports as an error.  For tests;
    the normal build compiles the checks away."""
    if not force and os.path.exists(CHECK_LIB) and all(
            os.path.getmtime(os.path.join(CSRC, f)) <= os.path.getmtime(CHECK_LIB) for f in os.listdir(CSRC)):
        return CHECK_LIB
    return _build(CHECK_LIB, os.path.join(PKG, "_build_check"), ["-DLBMHD_BOUNDS_CHECK"])


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--verbose-ptxas", action="store_true")
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--bounds-check", action="store_true", help="build the bounds-checking variant")
    a = ap.parse_args()
    print(build_checked(force=a.force) if a.bounds_check else build(force=a.force, verbose_ptxas=a.verbose_ptxas))


if __name__ == "__main__":
    main()
