"""Compile the FP64 CPU oracle (plain C) into oracle/_build/libbt_oracle.so.

Test infrastructure: the oracle library is built so that the tests, the smoke
check and the benchmark's CPU-baseline leg can call it.  It is compiled
without fused multiply-add contraction and without fast-math so that its
single-precision association decisions follow IEEE rounding operation by
operation.
"""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent
BUILD = HERE / "_build"
LIB = BUILD / "libbt_oracle.so"
SOURCES = [HERE / "bt_oracle.c"]
HEADERS = [HERE / "bt_oracle.h"]


def build(force: bool = False, verbose: bool = False) -> Path:
    BUILD.mkdir(exist_ok=True)
    newest = max(p.stat().st_mtime for p in SOURCES + HEADERS)
    if LIB.exists() and not force and LIB.stat().st_mtime >= newest:
        return LIB
    cc = os.environ.get("CC", "gcc")
    tmp = LIB.with_suffix(f".so.tmp{os.getpid()}")
    cmd = [cc, "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-pthread", "-Wall", "-Wextra", "-Wno-unused-parameter",
           *map(str, SOURCES), "-o", str(tmp), "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
