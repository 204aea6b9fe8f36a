"""Pins of the keyframe-selection oracle (oracle/keyframes.py, Sec. IV-C/E)
against closed forms that bypass its trace/arccos formula."""
import math

import numpy as np
import pytest

import oracle.keyframes as KO
import synthgen as S


def rot(axis, ang):
    return S.axis_angle_matrix(np.asarray(axis, float) / np.linalg.norm(axis), ang)


def test_geodesic_is_the_rotation_angle():
    rng = np.random.default_rng(0)
    for _ in range(50):
        th = rng.uniform(0.0, math.pi * 0.999)
        axis = rng.normal(size=3)
        Q = S.random_rotation(rng)
        assert abs(KO.geodesic(np.eye(3), rot(axis, th)) - th) < 1e-7
        Ra, Rb = S.random_rotation(rng), S.random_rotation(rng)
        d = KO.geodesic(Ra, Rb)
        assert abs(d - KO.geodesic(Rb, Ra)) < 1e-12                  # symmetric
        assert abs(d - KO.geodesic(Q @ Ra, Q @ Rb)) < 1e-7           # left-invariant


@pytest.mark.parametrize("seed", range(5))
def test_greedy_selection_closed_form(seed):
    """Rotations about one axis, I_0 at angle 0, the current frame at 0 and
    the others at distinct positive angles: after round r every candidate's
    cost is (r + 1) theta_f - sum of the chosen angles, so greedy takes the
    frames in increasing angle."""
    rng = np.random.default_rng(seed)
    n, K = int(rng.integers(3, 25)), int(rng.integers(1, 16))
    thetas = [0.0] + list(rng.uniform(0.05, 1.5, n - 1))
    pool = [rot([0, 0, 1], t) for t in thetas]
    want = [0] + sorted(range(1, n), key=lambda f: thetas[f])[:max(0, min(K, n) - 1)]
    assert KO.select(pool, rot([0, 0, 1], 0.0), K) == want


def _angle_quat(Ra, Rb):
    """Rotation angle of Ra^T Rb from its unit quaternion, 2 atan2(|v|, w)."""
    R = Ra.T @ Rb
    w = 0.5 * math.sqrt(max(0.0, 1.0 + R[0, 0] + R[1, 1] + R[2, 2]))
    v = 0.5 * np.array([math.copysign(math.sqrt(max(0.0, 1 + R[0, 0] - R[1, 1] - R[2, 2])), R[2, 1] - R[1, 2]),
                        math.copysign(math.sqrt(max(0.0, 1 - R[0, 0] + R[1, 1] - R[2, 2])), R[0, 2] - R[2, 0]),
                        math.copysign(math.sqrt(max(0.0, 1 - R[0, 0] - R[1, 1] + R[2, 2])), R[1, 0] - R[0, 1])])
    return 2.0 * math.atan2(np.linalg.norm(v), w)


@pytest.mark.parametrize("seed", range(5))
def test_greedy_selection_generic(seed):
    """Random 3-D rotations (no ties), geodesics through quaternions."""
    rng = np.random.default_rng(100 + seed)
    n, K = int(rng.integers(3, 30)), int(rng.integers(1, 16))
    pool = [S.random_rotation(rng) for _ in range(n)]
    R = S.random_rotation(rng)
    chosen = [0]
    while len(chosen) < min(K, n):
        costs = [(_angle_quat(pool[f], R) + sum(_angle_quat(pool[f], pool[c]) for c in chosen), f)
                 for f in range(n) if f not in chosen]
        chosen.append(min(costs)[1])
    assert KO.select(pool, R, K) == chosen


def test_selection_edge_cases():
    rng = np.random.default_rng(9)
    pool = [S.random_rotation(rng) for _ in range(6)]
    R = S.random_rotation(rng)
    assert KO.select(pool, R, 100)[0] == 0 and sorted(KO.select(pool, R, 100)) == list(range(6))
    assert KO.select(pool, R, 1) == [0]
    assert KO.select([], R, 5) == [] and KO.select(pool, R, 0) == []


def test_novel_view_threshold():
    pool = [np.eye(3), rot([1, 0, 0], math.radians(40))]
    assert not KO.is_novel(pool, rot([0, 1, 0], math.radians(9.9)))
    assert KO.is_novel(pool, rot([0, 1, 0], math.radians(10.1)))
    assert not KO.is_novel(pool, rot([1, 0, 0], math.radians(45.0)))      # 5 deg from the second
