"""Build libtsfcde.so in-tree with nvcc for sm_103a (GB300).

The translation units under csrc/ are compiled in parallel and linked into
paper_1603_00279_gb300/_lib/libtsfcde.so; nothing is installed anywhere else.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libtsfcde.so")
# the same library with every checked device index verified (-DTSFCDE_CHECKED): an index outside
# its array sets TSFCDE_E_BOUNDS and is redirected instead of accessed; for tests on tiny problems
CHECKED_LIB = os.path.join(LIBDIR, "checked", "libtsfcde_checked.so")
SOURCES = ["level_kernels.cu", "level_wide.cu", "batch_kernels.cu", "api.cu", "batch_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtsfcde")
    return cand


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "tsfcde.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _build_one(lib: str, defines, force: bool, verbose: bool) -> str:
    if not force and not _stale(lib):
        return lib
    libdir = os.path.dirname(lib)
    os.makedirs(libdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(libdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *defines, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile (if sources changed) and return the path of libtsfcde.so, or with checked=True of
    libtsfcde_checked.so (the -DTSFCDE_CHECKED build)."""
    if checked:
        return _build_one(CHECKED_LIB, ["-DTSFCDE_CHECKED"], force, verbose)
    return _build_one(LIB, [], force, verbose)


def build_all(force: bool = False) -> None:
    """Both libraries, compiled side by side."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        for f in [ex.submit(build, force, False, False), ex.submit(build, force, False, True)]:
            f.result()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
