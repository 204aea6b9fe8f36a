"""The paper's inner solver (BT_SOLVER_PCG: conjugate gradients with the
diagonal preconditioner, Sec. IV-D) on the GPU against the oracle and
against the library's Cholesky path."""
import numpy as np
import pytest

import oracle as O
import synthgen as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt as _bt
    _bt.load()
    return _bt


def pose_err(A, B):
    rot = max(S.rotation_angle(a[:3, :3] @ b[:3, :3].T) for a, b in zip(A, B))
    tr = max(np.abs(a[:3, 3] - b[:3, 3]).max() for a, b in zip(A, B))
    return rot, tr


def _pcg_config(bt, iters=500, tol=1e-12):
    c = bt.config_default()
    c.solver = bt.BT_SOLVER_PCG
    c.pcg_max_iters = iters
    c.pcg_tol = tol
    return c


def test_tiny_graph_matches_oracle(bt):
    g = S.tiny_graph(0)
    P, rep = bt.graph_from_synth(g, config=_pcg_config(bt)).solve(7)
    ro = O.solve(g, 7, params=O.Params(solver=1, pcg_tol=1e-12))
    rot, tr = pose_err(P, ro["poses"])
    assert rot <= 1e-5 and tr <= 1e-6
    assert abs(rep["cost_final"] - ro["cost_final"]) <= 1e-5 * ro["cost_final"]
    Pc, _ = bt.graph_from_synth(g).solve(7)            # the Cholesky path
    rot, tr = pose_err(P, Pc)
    assert rot <= 1e-7 and tr <= 1e-8


def test_paper_graph_one_step_matches_oracle(bt):
    g = S.paper_graph(0)
    P, rep = bt.graph_from_synth(g, config=_pcg_config(bt)).solve(1)
    ro = O.solve(g, 1, params=O.Params(solver=1, pcg_tol=1e-12))
    rot, tr = pose_err(P, ro["poses"])
    assert rot <= 1e-5 and tr <= 1e-6
    assert abs(rep["cost_init"] - ro["cost_per_iter"][0]) <= 1e-6 * ro["cost_per_iter"][0]


def test_zero_pcg_iterations_leave_poses(bt):
    g = S.tiny_graph(1)
    pg = bt.graph_from_synth(g, config=_pcg_config(bt, iters=0))
    P, rep = pg.solve(3)
    assert np.array_equal(P, g.pose_init) and rep["cost_final"] == rep["cost_init"]


def test_pcg_in_a_batch(bt):
    gs = [S.tiny_graph(k) for k in range(3)]
    singles = [bt.graph_from_synth(g, config=_pcg_config(bt)).solve(4)[0] for g in gs]
    pgs = [bt.graph_from_synth(g, config=_pcg_config(bt)) for g in gs]
    batch = bt.Batch()
    for pg in pgs:
        batch.add(pg)
    batch.set_shape(bt.BT_SINGLE_GRAPH_SHAPE)
    batch.solve(4)
    for pg, P in zip(pgs, singles):
        assert np.array_equal(pg.get_poses(), P)


def test_bad_solver_config(bt):
    c = bt.config_default()
    c.solver = 7
    with pytest.raises(bt.BTError):
        bt.PoseGraph(c)
    c = _pcg_config(bt, iters=-1)
    with pytest.raises(bt.BTError):
        bt.PoseGraph(c)
