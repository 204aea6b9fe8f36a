"""bt_pair_dense_energy_noalloc against the graph path's bt_eval_cost.

The no-alloc entry point serves callers that cannot allocate device memory
when they need the number (a framework that owns all device memory through its
own allocator, a real-time loop that must not let cudaMalloc/cudaFree
synchronise the device, a fixed memory budget).  It keeps its scratch in a
static device array shared by every call, so this test makes several calls in
a row, of different sizes, and checks each against the existing entry point
that allocates its own scratch: the association count must be identical and
the energy must agree within the tolerance the other parity tests use for an
energy evaluated at identical poses (1e-6 relative).
"""
import numpy as np
import pytest

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


def test_noalloc_rejects_oversized_frames():
    torch = pytest.importorskip("torch")
    from paper_2108_00516_gb300 import bt
    bt.load()
    g = S.tiny_graph(0)
    r = g.renders[0]
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    big = (140.0, 140.0, 80.0, 60.0, 32767, 32767)      # > 16,777,216 pixels
    with pytest.raises(RuntimeError, match="fixed scratch"):
        bt.pair_dense_energy_noalloc(dev(r.depth), dev(r.normals), dev(r.mask), big, g.pose_init[0],
                                     dev(r.depth), dev(r.normals), dev(r.mask), g.cams[0].as_tuple(),
                                     g.pose_init[1], out, stream=torch.cuda.current_stream())
