"""Coarse registration of Sec. IV-B on the GPU (bt_ransac, bt_ransac_init)
against the oracle (oracle/ransac.py): the same SplitMix64 samples, the same
single-precision inlier decisions, hence the same best sample and count; the
FP64 fits (quaternion form on the GPU, SVD form in the oracle) agree to
rounding."""
import numpy as np
import pytest

import oracle as O
import oracle.ransac as RO
import synthgen as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt as _bt
    _bt.load()
    return _bt


def _set(rng, n, outl=0.3):
    w = rng.normal(size=3)
    w *= 0.15 / np.linalg.norm(w)
    T = O.se3_exp(np.concatenate([rng.normal(size=3) * 0.02, w]))
    p = (rng.normal(size=(n, 3)) * [0.04, 0.04, 0.03] + [0, 0, 0.45]).astype(np.float32)
    q = p.astype(np.float64) @ T[:3, :3].T + T[:3, 3] + rng.normal(scale=0.001, size=(n, 3))
    k = int(outl * n)
    q[:k] = rng.normal(size=(k, 3)) * 0.05 + [0, 0, 0.45]
    return p, q.astype(np.float32), T


@pytest.mark.parametrize("n,refine", [(3, False), (10, False), (100, False), (400, False), (800, False),
                                      (400, True), (800, True)])
def test_matches_oracle(bt, n, refine):
    rng = np.random.default_rng(n + (1000 if refine else 0))
    p, q, T = _set(rng, n)
    for seed in (0, 12345):
        M, cnt = bt.ransac(p, q, hypotheses=128, seed=seed, refine=refine)
        Mo, cnt_o, best_o = RO.ransac(p, q, 128, seed, 0.005, refine)
        assert cnt == cnt_o
        assert np.abs(M - Mo).max() < 1e-9, (np.abs(M - Mo).max(), cnt, cnt_o)


def test_device_inputs_and_accuracy(bt):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    p, q, T = _set(rng, 500)
    M_h, c_h = bt.ransac(p, q, 256, 7, refine=True)
    M_d, c_d = bt.ransac(torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda(), 256, 7, refine=True)
    assert c_h == c_d and np.array_equal(M_h, M_d)
    assert S.rotation_angle(M_h[:3, :3] @ T[:3, :3].T) < np.radians(0.3)
    assert np.abs(M_h[:3, 3] - T[:3, 3]).max() < 0.002


def test_degenerate_inputs(bt):
    p = np.zeros((2, 3), np.float32)
    M, c = bt.ransac(p, p, 16, 0)
    assert np.array_equal(M, np.eye(4)) and c == 0
    line = np.c_[np.linspace(0, 0.1, 20), np.zeros(20), np.full(20, 0.5)].astype(np.float32)
    M, c = bt.ransac(line, line, 64, 0)
    assert np.array_equal(M, np.eye(4)) and c == 0
    M, c = bt.ransac(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), 16, 0)
    assert np.array_equal(M, np.eye(4)) and c == 0
    with pytest.raises(bt.BTError):
        bt.ransac(p, p, 0, 0)


@pytest.mark.parametrize("make", [lambda: S.tiny_graph(2), lambda: S.batched_graph(1003)])
def test_graph_init_matches_oracle(bt, make):
    g = make()
    pg = bt.graph_from_synth(g)
    pg.ransac_init(hypotheses=128, seed=3, refine=True)
    got = pg.get_poses()
    assert np.array_equal(got[0], g.pose_init[0])
    sets = {(i, j): (pi, pj) for (i, j, pi, pj) in g.matches}
    for j in range(1, g.n):
        pi, pj = sets[(0, j)]
        Mo, _, _ = RO.ransac(pi, pj, 128, 3, 0.005, True)
        want = Mo @ g.pose_init[0]
        assert np.abs(got[j] - want).max() < 1e-9
        # the coarse pose lands close to the truth
        assert S.rotation_angle(got[j][:3, :3] @ g.pose_true[j][:3, :3].T) < np.radians(1.0)
