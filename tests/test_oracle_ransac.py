"""Pins of the RANSAC + closed-form registration oracle (oracle/ransac.py,
Sec. IV-B) against published generator outputs, exact recovery and a known
outlier model."""
import numpy as np
import pytest

import oracle as O
import oracle.ransac as RO
import synthgen as S


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 seeded with 1234567, as published with
    # reference implementations of the generator
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [RO.splitmix64(1234567, c) for c in range(5)] == want


def _rigid(rng, ang=0.3, tr=0.05):
    w = rng.normal(size=3)
    w *= ang / np.linalg.norm(w)
    T = O.se3_exp(np.concatenate([rng.normal(size=3) * tr, w]))
    return T[:3, :3], T[:3, 3]


@pytest.mark.parametrize("seed", range(4))
def test_arun_recovers_exact_transform(seed):
    rng = np.random.default_rng(seed)
    R, t = _rigid(rng)
    p = rng.normal(size=(20, 3)) * 0.05 + [0, 0, 0.5]
    Rg, tg = RO.arun(p, p @ R.T + t)
    assert np.abs(Rg - R).max() < 1e-12 and np.abs(tg - t).max() < 1e-12


def test_arun_coplanar_points_give_a_rotation():
    rng = np.random.default_rng(5)
    R, t = _rigid(rng)
    p = np.c_[rng.normal(size=(10, 2)) * 0.05, np.full(10, 0.5)]      # one plane
    Rg, tg = RO.arun(p, p @ R.T + t)
    assert abs(np.linalg.det(Rg) - 1.0) < 1e-12 and np.abs(Rg - R).max() < 1e-10


def test_samples_are_distinct_and_in_range():
    for h in range(200):
        idx = RO.sample(99, h, 7)
        assert len(set(idx)) == 3 and all(0 <= k < 7 for k in idx)
    assert RO.sample(1, 0, 2) is None


def test_score_matches_fp64_away_from_threshold():
    rng = np.random.default_rng(6)
    R, t = _rigid(rng)
    p = (rng.normal(size=(500, 3)) * 0.05 + [0, 0, 0.5]).astype(np.float32)
    q = (p.astype(np.float64) @ R.T + t + rng.normal(scale=0.004, size=(500, 3))).astype(np.float32)
    d = np.linalg.norm(p.astype(np.float64) @ R.T + t - q.astype(np.float64), axis=1)
    far = np.abs(d - 0.005) > 1e-6
    assert np.array_equal(RO.score(R, t, p, q, 0.005)[far], (d < 0.005)[far])


def test_ransac_recovers_transform_through_outliers():
    rng = np.random.default_rng(7)
    R, t = _rigid(rng, 0.15, 0.02)
    n = 400
    p = (rng.normal(size=(n, 3)) * [0.04, 0.04, 0.03] + [0, 0, 0.45]).astype(np.float32)
    q = p.astype(np.float64) @ R.T + t + rng.normal(scale=0.001, size=(n, 3))
    out = rng.permutation(n)[:120]                                     # 30 % uniform outliers
    q[out] = rng.normal(size=(120, 3)) * 0.05 + [0, 0, 0.45]
    q = q.astype(np.float32)
    M, cnt, best = RO.ransac(p, q, 256, seed=11, delta=0.005)
    inl_true = np.setdiff1d(np.arange(n), out)
    assert best >= 0 and cnt >= 0.8 * len(inl_true)
    ang = S.rotation_angle(M[:3, :3] @ R.T)
    assert ang < np.radians(1.0) and np.abs(M[:3, 3] - t).max() < 0.005
    Mr, cnt_r, _ = RO.ransac(p, q, 256, seed=11, delta=0.005, refine=True)
    assert S.rotation_angle(Mr[:3, :3] @ R.T) < np.radians(0.2)
