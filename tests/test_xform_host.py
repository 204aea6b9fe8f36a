"""The single-precision pair transforms M = T_j T_i^-1 that the residual pass
reads are formed in double-float arithmetic (bt_xform.cuh), on the device
after every update and on the host for the first pass of a solve and for the
no-alloc call.  This CPU test compiles the header's host path and checks, on
random rigid poses, that every entry equals the FP64-formed entry rounded
once to single precision (the exact reference), and that T^-1 is the FP64
inverse rounded once."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def test_double_float_transforms_equal_fp64_rounded(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "xform_check"
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17",
                    f"-I{ROOT / 'paper_2108_00516_gb300' / 'csrc'}",
                    str(ROOT / "tests" / "native" / "xform_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = dict(zip(out[0::2], out[1::2]))
    assert int(vals["entries"]) == 240000
    assert int(vals["differ"]) == 0          # equal to RN32 of the FP64 entry
    assert float(vals["maxrel"]) < 1.2e-7    # one single-precision rounding
