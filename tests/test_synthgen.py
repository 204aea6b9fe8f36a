"""Sanity of the seeded synthetic inputs (shapes, ranges, determinism)."""
import numpy as np

import synthgen as S


def test_tiny_graph_shapes_and_determinism():
    a = S.tiny_graph(5)
    b = S.tiny_graph(5)
    assert a.n == 4 and len(a.matches) == 6
    for k in range(4):
        assert a.depth(k).shape == (120, 160) and a.depth(k).dtype == np.float32
        assert a.normals(k).shape == (120, 160, 3)
        assert np.array_equal(a.depth(k), b.depth(k))
        assert np.array_equal(a.normals(k), b.normals(k), equal_nan=True)
        m = a.mask(k) > 0
        assert m.any() and np.all(a.depth(k)[~m] == 0) and np.all(a.depth(k)[m] > 0)
        n = a.normals(k)[np.isfinite(a.normals(k)[..., 0])]
        assert np.allclose(np.linalg.norm(n, axis=1), 1, atol=1e-5)
    for (i, j, pi, pj) in a.matches:
        assert i < j and len(pi) == len(pj) == 200
    assert np.array_equal(a.pose_init, b.pose_init)
    assert np.array_equal(a.pose_init[0], a.pose_true[0])


def test_init_perturbation_is_exact():
    g = S.tiny_graph(2)
    for k in range(1, g.n):
        dR = g.pose_init[k][:3, :3] @ g.pose_true[k][:3, :3].T
        assert abs(np.degrees(S.rotation_angle(dR)) - 5.0) < 1e-9
        assert abs(np.linalg.norm(g.pose_init[k][:3, 3] - g.pose_true[k][:3, 3]) - 0.01) < 1e-12


def test_trajectory_step_bounds():
    g = S.tiny_graph(9)
    for k in range(1, g.n):
        dR = g.pose_true[k][:3, :3] @ g.pose_true[k - 1][:3, :3].T
        assert np.degrees(S.rotation_angle(dR)) <= 10.0 + 1e-9
        assert np.linalg.norm(g.pose_true[k][:3, 3] - g.pose_true[k - 1][:3, 3]) <= 0.02 + 1e-12


def test_inlier_matches_are_consistent():
    g = S.random_graph(3, 2, S.TINY_CAMERA, 100, 0.0, depth_sigma=0.0)
    i, j, pi, pj = g.matches[0]
    Tji = g.pose_true[j] @ S.pose_inverse(g.pose_true[i])
    pred = pi.astype(float) @ Tji[:3, :3].T + Tji[:3, 3]
    assert np.abs(pred - pj).max() < 1e-6


def test_fd_normals_face_camera():
    g = S.tiny_graph(1)
    n = g.normals(0)
    ok = np.isfinite(n[..., 0])
    cam = g.cams[0]
    v, u = np.nonzero(ok)
    z = g.depth(0)[v, u]
    P = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], -1)
    assert np.all((n[v, u] * P).sum(-1) <= 0)
