"""Build libbt.so (the CUDA library behind include/bt.h) for sm_103a.

Compiles each translation unit with nvcc in parallel and links a shared
library into paper_2108_00516_gb300/_build/.  No GPU is needed to build.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libbt.so"
LIB_CHECKED = BUILD / "libbt_checked.so"
INCLUDE = ROOT / "include"
SOURCES = sorted(CSRC.glob("*.cu"))
HEADERS = sorted(CSRC.glob("*.h")) + sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found (set NVCC or put CUDA's bin directory on PATH)")


def _flags(ptxas_verbose: bool):
    # -ffp-contract=off: host arithmetic is not fused, so the host reproduces
    # the device's explicitly rounded operations bit for bit
    f = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-Xcompiler", "-ffp-contract=off",
         f"-I{INCLUDE}", f"-I{CSRC}", "--expt-relaxed-constexpr"]
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, checked: bool = False) -> Path:
    """Compile libbt.so, or with checked=True libbt_checked.so: the same
    library with every index of the residual pass tested before use
    (-DBT_CHECKED; a failed test is reported as BT_ERR_INVALID)."""
    out_dir = BUILD / "checked" if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    out_dir.mkdir(parents=True, exist_ok=True)
    newest = max(p.stat().st_mtime for p in SOURCES + HEADERS + [Path(__file__)])
    if lib.exists() and not force and not ptxas_verbose and lib.stat().st_mtime >= newest:
        return lib
    cc = nvcc()
    extra = ["-DBT_CHECKED"] if checked else []

    def compile_one(src: Path):
        obj = out_dir / (src.stem + ".o")
        cmd = [cc, *_flags(ptxas_verbose), *extra, "-c", str(src), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stdout}\n{r.stderr}")
        if (verbose or ptxas_verbose) and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib.with_suffix(f".so.tmp{os.getpid()}")
    cmd = [cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *map(str, objs), "-o", str(tmp)]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True, ptxas_verbose="-v" in sys.argv, checked="--checked" in sys.argv))
