"""Build libhulld.so (CUDA for sm_103a) in-tree with nvcc.

Each .cu file compiles to an object in parallel, then one link step makes
paper_1402_1720_gb300/_lib/libhulld.so.  The CUDA runtime is linked
statically, so the library needs only the driver (libcuda) at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
SRC = PKG / "csrc"
OUT_DIR = PKG / "_lib"
LIB = OUT_DIR / "libhulld.so"
INCLUDE = PKG.parent / "include"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fvisibility=hidden"]
SOURCES = ["hd_api.cu", "hd_trace.cu", "hd_tiles.cu", "hd_scatter.cu", "hd_decide.cu", "hd_noalloc.cu", "hd_server.cu",
           "hd_probe.cu", "hd_rows.cu", "hd_binned.cu", "hd_diag.cu",
           "hd_canny.cu", "hd_thick.cu", "hd_thick_tiles.cu", "hd_euclid.cu"]


def nvcc() -> str:
    for cand in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhulld")


def _deps():
    files = [SRC / s for s in SOURCES] + list(SRC.glob("*.cuh")) + [INCLUDE / "hulld.h"]
    return max(f.stat().st_mtime for f in files)


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and LIB.exists() and LIB.stat().st_mtime >= _deps():
        return LIB
    OUT_DIR.mkdir(exist_ok=True)
    exe = nvcc()
    objs, procs = [], []
    for s in SOURCES:
        o = OUT_DIR / (Path(s).stem + ".o")
        cmd = [exe, *ARCH, *NVCC_FLAGS, "-I", str(INCLUDE), "-c", str(SRC / s), "-o", str(o)]
        if os.environ.get("HD_PTXAS_VERBOSE"):
            cmd.append("-Xptxas=-v")
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(o)
    failed = []
    for s, p in procs:
        out, _ = p.communicate()
        if out and (p.returncode != 0 or verbose or os.environ.get("HD_PTXAS_VERBOSE")):
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(s)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB.with_suffix(f".so.{os.getpid()}.tmp")
    link = [exe, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-cudart", "static"]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
