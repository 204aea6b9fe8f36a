"""bt_select_keyframes / bt_is_novel_view (host code of libbt, Sec. IV-C/E)
against the oracle; no GPU work is involved."""
import numpy as np
import pytest

import oracle.keyframes as KO
import synthgen as S


@pytest.fixture(scope="module")
def bt():
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt as _bt
    _bt.load()
    return _bt


def _pose(R, rng):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = rng.normal(size=3)          # translations must not matter
    return T


@pytest.mark.parametrize("seed", range(8))
def test_selection_matches_oracle(bt, seed):
    rng = np.random.default_rng(seed)
    n, K = int(rng.integers(1, 60)), int(rng.integers(1, 16))
    pool = [S.random_rotation(rng) for _ in range(n)]
    R = S.random_rotation(rng)
    got = bt.select_keyframes(np.stack([_pose(P, rng) for P in pool]), _pose(R, rng), K)
    assert got == KO.select(pool, R, K)
    thr = float(rng.uniform(5, 60))
    assert bt.is_novel_view(np.stack(pool), R, thr) == KO.is_novel(pool, R, thr)


def test_sequence_plan_matches_oracle(bt):
    from paper_2108_00516_gb300 import keyframes as KF
    seq = S.paper_sequence(seed=2000, n_frames=120)
    R = seq.poses_true[:, :3, :3]
    graphs, history = KF.plan_sequence(R, max_nodes=10)
    pool = [0]
    for t in range(1, len(R)):
        sel = KO.select([R[f] for f in pool], R[t], 9)
        assert graphs[t - 1] == [pool[k] for k in sel] + [t]
        if KO.is_novel([R[f] for f in pool], R[t], 10.0):
            pool.append(t)
        assert history[t - 1] == pool
    assert len(pool) > 9                   # the pool outgrows K, so selection matters


def test_errors_and_edges(bt):
    rng = np.random.default_rng(3)
    pool = np.stack([_pose(S.random_rotation(rng), rng) for _ in range(5)])
    assert bt.select_keyframes(pool, pool[2], 0) == []
    assert bt.select_keyframes(pool, pool[2], 50)[0] == 0
    assert bt.is_novel_view(pool[:0], pool[0]) is True          # empty pool
    with pytest.raises(bt.BTError):
        bt.select_keyframes(pool, pool[0], -1)
    bad = pool.copy()
    bad[1, 0, 0] = np.nan
    with pytest.raises(bt.BTError):
        bt.select_keyframes(bad, pool[0], 3)
