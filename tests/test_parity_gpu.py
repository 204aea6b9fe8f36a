"""GPU (through the C interface) against the FP64 CPU oracle.

Tolerances.  The GPU computes residuals, Jacobians and their block sums in
FP32 and everything from the 6x6 blocks on in FP64; the oracle is FP64
throughout.  The association decision (integers) is taken in single
precision on both sides but in different operation orders, so it may differ
for a pixel within rounding of a half-pixel edge, the image edge or a gate;
the oracle classifies every pixel (oracle.energy_bounds) and the GPU's count
must lie in the admissible range, its energy within FP32 rounding plus the
largest change those pixels can make (index-level and frozen-association
checks: test_assoc_gpu.py).  Per-pixel FP32 residuals carry ~1e-7 relative
rounding on coordinates of ~0.5 m, i.e. ~3e-8 m on residuals of ~1e-3 m;
summed over thousands of pixels with random signs this is <= 1e-6 of the
energy.  The solve tolerances are the ones the method's specification
states for the FP32 path: relative final cost 1e-5, poses 1e-5 rad and
1e-6 m; they apply to every single iteration started from identical poses,
and to whole solves that converge.

Gauss-Newton with projective re-association at every iteration and no line
search does not settle on a point on the large graphs: the association set
changes from one iterate to the next, and a start moved by the size of
single-precision rounding (1e-7 rad) leads the oracle itself 1e-5..3e-5 rad
away within 10 iterations.  The free-running
comparison on the paper-shaped graph therefore allows, on top of the stated
tolerance, twice the oracle's own spread from perturbed starts (measured in
the test); stepwise comparisons hold the stated tolerance unwidened.
"""
import numpy as np
import pytest

import oracle as O
import synthgen as S
from parity_util import oracle_self_spread, pose_err

pytestmark = pytest.mark.gpu

COST_RTOL_EVAL = 1e-6
COST_RTOL = 1e-5
ROT_TOL = 1e-5
TRANS_TOL = 1e-6


@pytest.fixture(scope="module")
def bt():
    import torch
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt as _bt
    _bt.load()
    torch.cuda.init()
    return _bt


def check_energy(gpu_total, gpu_count, g, P, nodes=None, gpu_dense=None):
    """The GPU's energy and association count at poses P against the oracle:
    count within the range single-precision rounding admits, energy within
    FP32 rounding plus the cost those open decisions can move."""
    o = O.energy(g, P, nodes=nodes)
    b = O.energy_bounds(g, P, nodes=nodes)
    assert b["count_lo"] <= gpu_count <= b["count_hi"], (gpu_count, b)
    assert b["ambiguous"] <= 5e-3 * max(b["pixels"], 1), b
    assert abs(gpu_total - o["total"]) <= COST_RTOL_EVAL * o["total"] + b["slack"], (gpu_total, o, b)
    if gpu_dense is not None:
        assert abs(gpu_dense - o["dense"]) <= COST_RTOL_EVAL * o["dense"] + b["slack"]
    return o, b


@pytest.mark.parametrize("gid", [0, 1, 2])
def test_eval_cost_matches_oracle(bt, gid):
    """Eq. 1 at the same poses: association count in the admissible range,
    energy within FP32 rounding (plus the slack of open decisions)."""
    g = S.tiny_graph(gid)
    pg = bt.graph_from_synth(g)
    c = pg.eval_cost()
    o, b = check_energy(c["total"], c["dense_inliers"], g, g.pose_init, gpu_dense=c["dense"])
    assert abs(c["sparse"] - o["sparse"]) <= COST_RTOL_EVAL * o["sparse"]


@pytest.mark.parametrize("gid", [0, 3, 7])
def test_stepwise_iterations_match_oracle(bt, gid):
    """Every Gauss-Newton iteration, started on both sides from the same poses
    (the GPU's), gives the same energy, the same association count and the same
    updated poses."""
    g = S.tiny_graph(gid)
    pg = bt.graph_from_synth(g)
    P = g.pose_init.copy()
    for it in range(7):
        pg.set_poses(P)
        Pg, rg = pg.solve(1)
        ro = O.solve(g, 1, poses=P)
        assert rg["status"] == 0 and ro["status"] == 0
        b0 = O.energy_bounds(g, P)
        assert abs(rg["cost_init"] - ro["cost_per_iter"][0]) <= COST_RTOL_EVAL * ro["cost_per_iter"][0] + b0["slack"]
        rot, tr = pose_err(Pg, ro["poses"])
        assert rot <= ROT_TOL and tr <= TRANS_TOL, (it, rot, tr)
        check_energy(rg["cost_final"], rg["dense_inliers"], g, Pg)
        P = Pg


@pytest.mark.parametrize("gid", [0, 1, 2, 3])
def test_solve_matches_oracle_tiny(bt, gid):
    """Free-running 7-iteration solve on the tiny workload (N=4, 160x120)."""
    g = S.tiny_graph(gid)
    pg = bt.graph_from_synth(g)
    Pg, rg = pg.solve(7)
    ro = O.solve(g, 7)
    rot, tr = pose_err(Pg, ro["poses"])
    # the GPU's own energy of its poses is the oracle's energy of them
    check_energy(rg["cost_final"], rg["dense_inliers"], g, Pg)
    assert abs(rg["cost_final"] - ro["cost_final"]) <= COST_RTOL * ro["cost_final"], (rot, tr)
    assert rot <= ROT_TOL and tr <= TRANS_TOL


@pytest.fixture(scope="module")
def paper():
    return S.paper_graph(0)


def test_stepwise_paper_shaped(bt, paper):
    """N=10 views at 640x480 (90 ordered pairs, ~2M associations): three
    iterations, each from the GPU's poses on both sides."""
    g = paper
    pg = bt.graph_from_synth(g)
    P = g.pose_init.copy()
    for it in range(3):
        pg.set_poses(P)
        Pg, rg = pg.solve(1)
        ro = O.solve(g, 1, poses=P)
        b0 = O.energy_bounds(g, P)
        assert abs(rg["cost_init"] - ro["cost_per_iter"][0]) <= COST_RTOL_EVAL * ro["cost_per_iter"][0] + b0["slack"]
        rot, tr = pose_err(Pg, ro["poses"])
        assert rot <= ROT_TOL and tr <= TRANS_TOL, (it, rot, tr)
        check_energy(rg["cost_final"], rg["dense_inliers"], g, Pg)
        P = Pg


def test_solve_matches_oracle_paper_shaped(bt, paper):
    """10 free-running iterations on the paper-shaped graph.  Projective
    re-association makes the iteration map discontinuous: a start moved by
    the size of single-precision rounding (1e-7 rad; 1e-9 rad already on
    this graph) flips a few of the ~6M association decisions and the oracle
    itself then ends 1e-5..3e-5 rad and ~1e-6 m away after 10 iterations (a
    1e-12 start does not move it at all).  No implementation whose rounding
    differs can follow the oracle closer than that, so the comparison allows,
    on top of the stated tolerance, twice the oracle's own spread from three
    such starts, measured here.  The unwidened numbers are printed."""
    g = paper
    pg = bt.graph_from_synth(g)
    Pg, rg = pg.solve(10)
    ro, s_rot, s_tr, s_cost = oracle_self_spread(g, 10)
    rot, tr = pose_err(Pg, ro["poses"])
    dc = abs(rg["cost_final"] - ro["cost_final"]) / ro["cost_final"]
    print(f"\npaper-0 free-running: GPU vs oracle {rot:.2e} rad {tr:.2e} m cost {dc:.2e}; "
          f"oracle self-spread {s_rot:.2e} rad {s_tr:.2e} m cost {s_cost:.2e}")
    check_energy(rg["cost_final"], rg["dense_inliers"], g, Pg)
    assert dc <= COST_RTOL + 2 * s_cost
    assert rot <= ROT_TOL + 2 * s_rot and tr <= TRANS_TOL + 2 * s_tr, (rot, tr, s_rot, s_tr)
    assert rg["dense_pixel_pairs"] == 10 * 9 * sum(
        int(((g.mask(k) > 0) & (g.depth(k) > 0) & np.isfinite(g.normals(k)).all(-1)).sum()) for k in range(10))


def test_device_inputs_bitwise_equal_host_inputs(bt):
    g = S.tiny_graph(4)
    a = bt.graph_from_synth(g)
    b = bt.graph_from_synth(g, device="cuda")
    Pa, ra = a.solve(3)
    Pb, rb = b.solve(3)
    assert np.array_equal(Pa, Pb) and ra["cost_final"] == rb["cost_final"]


def test_rerun_is_deterministic(bt):
    g = S.tiny_graph(5)
    a = bt.graph_from_synth(g)
    P1, r1 = a.solve(4)
    a.set_poses(g.pose_init)
    P2, r2 = a.solve(4)
    assert np.array_equal(P1, P2) and r1["cost_final"] == r2["cost_final"]


def test_two_nodes_and_active_subset(bt):
    g = S.tiny_graph(6)
    pg = bt.graph_from_synth(g)
    pg.set_active([pg.frame_ids[0], pg.frame_ids[2]])
    Pg, rg = pg.solve(5)
    ro = O.solve(g, 5, nodes=[0, 2])
    rot, tr = pose_err(Pg, ro["poses"])
    assert rot <= ROT_TOL and tr <= TRANS_TOL
    assert abs(rg["cost_final"] - ro["cost_final"]) <= COST_RTOL * ro["cost_final"]


def test_empty_mask_frame_and_missing_matches(bt):
    """A frame with no valid pixel contributes no dense term; a pair without
    correspondences contributes no sparse term."""
    g = S.tiny_graph(8)
    r3 = g.renders[3]
    empty = S.Render(np.zeros_like(r3.depth), r3.normals, np.zeros_like(r3.mask), r3.depth_clean, r3.normals_true)
    renders = list(g.renders[:3]) + [empty]
    matches = [m for m in g.matches if (m[0], m[1]) != (0, 1)]
    g2 = S.SynthGraph(g.cams, renders, g.pose_true, g.pose_init, g.fixed, matches, g.shape)
    pg = bt.graph_from_synth(g2)
    Pg, rg = pg.solve(4)
    ro = O.solve(g2, 4)
    rot, tr = pose_err(Pg, ro["poses"])
    assert rot <= ROT_TOL and tr <= TRANS_TOL
    assert abs(rg["cost_final"] - ro["cost_final"]) <= COST_RTOL * ro["cost_final"]


def test_singular_system_leaves_poses(bt):
    """A free node with no constraint at all: BT_ERR_SINGULAR, poses kept."""
    g = S.tiny_graph(0)
    cfg = bt.config_default()
    cfg.lambda_dense = 0.0
    g2 = S.SynthGraph(g.cams, g.renders, g.pose_true, g.pose_init, g.fixed, [], g.shape)
    pg = bt.graph_from_synth(g2, config=cfg)
    P0 = pg.get_poses()
    _, rep = pg.solve(3, raise_on_error=False)
    assert rep["status"] == bt.BT_ERR_SINGULAR
    assert np.array_equal(pg.get_poses(), P0)


def test_zero_iterations_and_fixed_only(bt):
    g = S.tiny_graph(1)
    pg = bt.graph_from_synth(g)
    P, rep = pg.solve(0)
    assert np.array_equal(P, g.pose_init)
    check_energy(rep["cost_final"], rep["dense_inliers"], g, g.pose_init)
    pg.set_active([pg.frame_ids[0]])
    P1, rep1 = pg.solve(2)
    assert np.array_equal(P1[0], g.pose_init[0]) and rep1["cost_final"] == 0.0


def test_remove_frame(bt):
    g = S.tiny_graph(2)
    pg = bt.graph_from_synth(g)
    pg.remove_frame(pg.frame_ids[3])
    Pg, rg = pg.solve(4)
    ro = O.solve(g, 4, nodes=[0, 1, 2])
    rot, tr = pose_err(Pg, ro["poses"])
    assert rot <= ROT_TOL and tr <= TRANS_TOL


def test_replaced_and_removed_sets(bt):
    # a set given again in the other order replaces the stored one; an empty
    # set removes the pair's set; removing a frame drops its sets -- the solve
    # then matches the oracle on the graph without those sets
    import dataclasses
    g = S.tiny_graph(2)
    pg = bt.graph_from_synth(g)
    ids = pg.frame_ids
    i0, j0, pa0, pb0 = g.matches[0]
    pg.set_matches(ids[j0], ids[i0], pb0, pa0)
    i1, j1, _, _ = g.matches[1]
    empty = np.zeros((0, 3), np.float32)
    pg.set_matches(ids[i1], ids[j1], empty, empty)
    pg.remove_frame(ids[3])
    Pg, rg = pg.solve(4)
    kept = [m for k, m in enumerate(g.matches) if k != 1 and 3 not in (m[0], m[1])]
    ro = O.solve(dataclasses.replace(g, matches=kept), 4, nodes=[0, 1, 2])
    rot, tr = pose_err(Pg, ro["poses"])
    assert rot <= ROT_TOL and tr <= TRANS_TOL
    assert abs(rg["cost_final"] - ro["cost_final"]) <= COST_RTOL * ro["cost_final"]


def test_invalid_arguments(bt):
    pg = bt.PoseGraph()
    with pytest.raises(bt.BTError):
        pg.solve(1)            # no frames
    g = S.tiny_graph(0)
    r = g.renders[0]
    with pytest.raises(bt.BTError):
        pg.add_frame(r.depth, r.normals, r.mask, (140.0, 140.0, 80.0, 60.0, 0, 120), g.pose_init[0])
    bad = g.pose_init[0].copy()
    bad[3, 3] = 2.0
    with pytest.raises(bt.BTError):
        pg.add_frame(r.depth, r.normals, r.mask, g.cams[0].as_tuple(), bad)
    with pytest.raises(bt.BTError):
        pg.set_active([7])
