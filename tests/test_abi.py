"""The C library loads without a GPU, exports every function include/bt.h
declares, and its structs have the layout the binding assumes."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "bt.h"


@pytest.fixture(scope="module")
def lib():
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt
    return bt.load()


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    return sorted(set(re.findall(r"\b(bt_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), f"{n} declared in bt.h but not exported"


def test_binding_covers_header():
    from paper_2108_00516_gb300 import bt
    assert set(declared_functions()) == set(bt.SIGNATURES)


def test_struct_layout_matches_c(tmp_path):
    from paper_2108_00516_gb300 import bt
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "bt.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(bt_intrinsics), sizeof(bt_config), '
                   'sizeof(bt_matches), sizeof(bt_solve_report), offsetof(bt_solve_report, cost_per_iter), '
                   'offsetof(bt_solve_report, dense_inliers));return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    want = [C.sizeof(bt.bt_intrinsics), C.sizeof(bt.bt_config), C.sizeof(bt.bt_matches),
            C.sizeof(bt.bt_solve_report), bt.bt_solve_report.cost_per_iter.offset,
            bt.bt_solve_report.dense_inliers.offset]
    assert got == want


def test_host_only_calls(lib):
    from paper_2108_00516_gb300 import bt
    c = bt.config_default()
    assert c.huber_dense == 0.005 and c.dense_max_normal_deg == 45.0 and c.precision == bt.BT_FP32
    assert lib.bt_status_str(bt.BT_ERR_SINGULAR).decode().startswith("normal equations")
    # argument checks happen before any device work
    assert lib.bt_graph_create(C.byref(c), None, None) == bt.BT_ERR_INVALID
    bad = bt.config_default()
    bad.huber_dense = -1.0
    h = C.c_void_p()
    assert lib.bt_graph_create(C.byref(bad), None, C.byref(h)) == bt.BT_ERR_INVALID
    assert "Huber" in lib.bt_last_error().decode()
    assert lib.bt_solve(None, 1, None, None) == bt.BT_ERR_INVALID
    assert lib.bt_num_active(None) == bt.BT_ERR_INVALID


def test_header_constants_match_binding(lib):
    """Every numeric #define of bt.h has the same value in the binding."""
    from paper_2108_00516_gb300 import bt
    text = HEADER.read_text()
    defs = dict(re.findall(r"#define\s+(BT_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text))
    assert {"BT_NUM_SHAPES", "BT_MAX_NODES", "BT_WS_NUM_PARAMS", "BT_ERR_SINGULAR"} <= set(defs)
    for name, val in defs.items():
        py = name.replace("BT_WS_NUM_PARAMS", "WS_NUM_PARAMS")
        assert getattr(bt, py) == int(val), name
    assert lib.bt_warmstart_num_params() == int(defs["BT_WS_NUM_PARAMS"])
