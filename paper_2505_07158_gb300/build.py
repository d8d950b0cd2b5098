"""Build ``libfhdcipher.so`` in-tree with nvcc for sm_103a (GB300).

The translation units are compiled in parallel and linked as one shared
library under ``paper_2505_07158_gb300/_build/``.  Device code is compiled
with ``-fmad=false`` and host code with ``-ffp-contract=off``: the chaotic
iteration must round every binary64 multiply and add on its own.

``build(checked=True)`` makes the checked build, ``libfhdcipher_checked.so``:
the same sources with ``-DFHD_BOUNDS_CHECK``, where every computed index of a
kernel's memory accesses is range-checked (a failed check is recorded and the
access skipped; ``fhd_bounds_report``).  ``FHD_CHECKED=1`` in the environment
makes the Python binding load it instead of the default library."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfhdcipher.so")
CHECKED_LIB = os.path.join(BUILD, "libfhdcipher_checked.so")
SOURCES = ["api.cu", "sha256.cu", "chaos.cu", "permute.cu", "stats.cu", "probe.cu", "persist.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfhdcipher")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "fhdcipher.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile and link the library (the checked build with checked=True) unless it is newer than every
    source; returns its path."""
    lib = CHECKED_LIB if checked else LIB
    objdir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(objdir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    cc = nvcc()
    flags = NVCC_FLAGS + (["-DFHD_BOUNDS_CHECK"] if checked else [])

    def compile_one(src: str) -> str:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False, verbose: bool = False) -> tuple[str, str]:
    """Both libraries, compiled side by side: (default, checked)."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build, force, verbose, False)
        b = ex.submit(build, force, verbose, True)
        return a.result(), b.result()


if __name__ == "__main__":
    print(*build_all(force=True, verbose=True), sep="\n")
