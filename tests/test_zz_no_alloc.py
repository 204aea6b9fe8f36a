"""bt_pair_dense_energy_noalloc against the FP64 oracle and the graph path.

The no-alloc entry point serves callers that cannot allocate device memory
when they need the number (a framework that owns all device memory through its
own allocator, a real-time loop that must not let cudaMalloc/cudaFree
synchronise the device, a fixed memory budget).  It keeps its scratch in a
static device array shared by every call, so this test makes several calls in
a row, of different sizes, and checks each
  - against the oracle's dense energy of the two-frame graph (Eq. 1 with the
    sparse term dropped: lambda_2 (E_g(a,b) + E_g(b,a))): association count
    within the range single-precision rounding admits, energy within 1e-6
    relative plus the cost those open decisions can move;
  - against the existing entry point that allocates its own scratch
    (bt_eval_cost of a graph of the two frames): the same decisions, so the
    same count, and the energy within 1e-6 relative (summation order).
"""
import numpy as np
import pytest

import oracle as O
import synthgen as S

pytestmark = pytest.mark.gpu

COST_RTOL_EVAL = 1e-6


def _reference(bt, g, i, j, poses):
    """Dense part of Eq. 1 for the two frames through the graph path."""
    pg = bt.PoseGraph()
    ids = []
    for k in (i, j):
        r = g.renders[k]
        ids.append(pg.add_frame(r.depth, r.normals, r.mask, g.cams[k].as_tuple(), poses[k], fixed=(k == i)))
    c = pg.eval_cost()
    pg.close()
    return c["dense"], c["dense_inliers"]


def _noalloc(bt, torch, g, i, j, poses, out, stream):
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")
    ra, rb = g.renders[i], g.renders[j]
    bt.pair_dense_energy_noalloc(dev(ra.depth), dev(ra.normals), dev(ra.mask), g.cams[i].as_tuple(), poses[i],
                                 dev(rb.depth), dev(rb.normals), dev(rb.mask), g.cams[j].as_tuple(), poses[j],
                                 out, stream=stream)
    stream.synchronize()
    return float(out[0].item()), int(round(out[1].item()))


def test_noalloc_pair_energy_matches_graph_path():
    torch = pytest.importorskip("torch")
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt
    bt.load()
    stream = torch.cuda.current_stream()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    small = S.tiny_graph(2)
    large = S.paper_graph(1, n_frames=2)
    cases = [(small, 0, 1, small.pose_init), (large, 0, 1, large.pose_init),
             (small, 2, 3, small.pose_true), (small, 0, 1, small.pose_init)]
    for (g, i, j, P) in cases:
        e_ref, n_ref = _reference(bt, g, i, j, P)
        e, n = _noalloc(bt, torch, g, i, j, P, out, stream)
        assert n_ref > 0
        assert n == n_ref
        assert abs(e - e_ref) <= COST_RTOL_EVAL * e_ref
        o = O.energy(g, P[[i, j]], nodes=[i, j])
        b = O.energy_bounds(g, P, nodes=[i, j])
        assert b["count_lo"] <= n <= b["count_hi"], (n, b)
        assert abs(e - o["dense"]) <= COST_RTOL_EVAL * o["dense"] + b["slack"], (e, o["dense"], b)


def test_noalloc_rejects_oversized_frames():
    """The C entry point itself rejects frames beyond its fixed scratch before
    it touches any buffer (called through the C interface directly: the
    binding would already refuse buffers that do not match the sizes)."""
    import ctypes as C
    torch = pytest.importorskip("torch")
    from paper_2108_00516_gb300 import bt
    L = bt.load()
    g = S.tiny_graph(0)
    r = g.renders[0]
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")
    d, n, m = dev(r.depth), dev(r.normals), dev(r.mask)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    big = bt.bt_intrinsics(140.0, 140.0, 80.0, 60.0, 32767, 32767)      # > 16,777,216 pixels
    ok = bt.bt_intrinsics(*g.cams[0].as_tuple())
    P0 = np.ascontiguousarray(g.pose_init[0]).reshape(16)
    P1 = np.ascontiguousarray(g.pose_init[1]).reshape(16)
    dp = C.POINTER(C.c_double)
    st = L.bt_pair_dense_energy_noalloc(C.c_void_p(d.data_ptr()), C.c_void_p(n.data_ptr()), C.c_void_p(m.data_ptr()),
                                        C.byref(big), P0.ctypes.data_as(dp), C.c_void_p(d.data_ptr()),
                                        C.c_void_p(n.data_ptr()), C.c_void_p(m.data_ptr()), C.byref(ok),
                                        P1.ctypes.data_as(dp), None, C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == bt.BT_ERR_INVALID
    assert "fixed scratch" in L.bt_noalloc_last_error().decode()
    # and the binding refuses mismatched buffers before any call
    with pytest.raises(ValueError, match="depth_a must be float32 with W\\*H"):
        bt.pair_dense_energy_noalloc(d, n, m, (140.0, 140.0, 80.0, 60.0, 32767, 32767), g.pose_init[0],
                                     d, n, m, g.cams[0].as_tuple(), g.pose_init[1], out,
                                     stream=torch.cuda.current_stream())
