"""Pins of the warm-start oracle (oracle/warmstart.py) against facts that do
not come from the oracle itself: a library rounding routine, finite
differences, symmetries, closed forms of Adam and of the increment, exact
recovery and gauge equivariance of the averaging solve."""
import numpy as np
import pytest

import oracle as O
import oracle.warmstart as W
import synthgen as S


def _rand_pose(rng, ang=0.3, tr=0.1):
    w = rng.normal(size=3)
    w *= ang * rng.uniform(0.2, 1.0) / np.linalg.norm(w)
    return O.se3_exp(np.concatenate([rng.normal(size=3) * tr, w]))


def _inv(T):
    out = np.eye(4)
    out[:3, :3] = T[:3, :3].T
    out[:3, 3] = -T[:3, :3].T @ T[:3, 3]
    return out


def test_bf16_matches_torch_rounding():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        # exact ties between two bf16 neighbours, both parities
                        (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32).astype(np.float64),
                        [0.0, -0.0, 1.0, -3.5, 65504.0]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(W.bf16(x), ref)


def _net_case(seed, n=40):
    rng = np.random.default_rng(seed)
    P = S.warmstart_init(seed).astype(np.float64)
    P = P + rng.normal(scale=0.02, size=P.shape)       # biases away from zero
    x = rng.normal(size=(n, 6))
    t = rng.normal(size=6)
    return P, x, t


@pytest.mark.parametrize("seed", [3, 4])
def test_gradient_matches_finite_differences(seed):
    """exact=True network: analytic gradient vs central differences."""
    P, x, t = _net_case(seed)
    _, g = W.loss_and_grad(P, [x], [t], exact=True)
    rng = np.random.default_rng(seed + 100)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in W.LAYERS])
    idx = np.concatenate([rng.integers(offs[k], offs[k + 1], 12) for k in range(len(W.LAYERS))])
    h = 1e-6
    worst = 0.0
    for k in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (W.loss_and_grad(Pp, [x], [t], exact=True)[0] - W.loss_and_grad(Pm, [x], [t], exact=True)[0]) / (2 * h)
        worst = max(worst, abs(fd - g[k]) / max(1e-3, abs(g[k])))
    assert worst < 1e-5, worst
    assert np.count_nonzero(g[idx]) > len(idx) // 2


def test_set_permutation_invariance():
    P, x, _ = _net_case(5, n=100)
    y0, _ = W.forward(P, x)
    y1, _ = W.forward(P, x[np.random.default_rng(0).permutation(len(x))])
    assert np.array_equal(y0, y1)


def test_max_pool_routes_to_one_row():
    """Only the rows that hold some channel's maximum receive gradient in W1:
    a set plus copies of a row that is nowhere the maximum has the same
    gradient."""
    P, x, t = _net_case(6, n=30)
    _, c = W.forward(P, x)
    rows = set(c["r"].tolist())
    loser = next(k for k in range(len(x)) if k not in rows)
    x2 = np.concatenate([x, np.repeat(x[loser:loser + 1], 5, axis=0)])
    g1 = W.loss_and_grad(P, [x], [t])[1]
    g2 = W.loss_and_grad(P, [x2], [t])[1]
    assert np.array_equal(g1, g2)


def test_adam_closed_forms():
    rng = np.random.default_rng(7)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    lr, eps = 1e-3, 1e-8
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    # with a constant gradient the bias-corrected moments are g and g^2 at
    # every step, so every step is -lr g / (|g| + eps)
    for t in range(1, 6):
        pn, m, v = W.adam(p, g, m, v, t, lr)
        assert np.allclose(pn - p, -lr * g / (np.abs(g) + eps), rtol=1e-9, atol=0)
        p = pn
    # first step with beta1 = 0: the same closed form
    pn, _, _ = W.adam(p0, g, np.zeros(50), np.zeros(50), 1, lr, beta1=0.0)
    assert np.allclose(pn - p0, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)


def test_features_closed_forms():
    rng = np.random.default_rng(8)
    p = rng.normal(size=(50, 3)) * 0.05 + [0, 0, 0.4]
    M0 = _rand_pose(rng)
    q = p @ M0[:3, :3].T + M0[:3, 3]
    x, c = W.features(p, q, M0)
    assert np.allclose(x[:, 3:], 0, atol=1e-12)                 # perfectly aligned pairs
    assert np.allclose(x[:, :3].mean(axis=0), 0, atol=1e-12)     # centred on q's mean
    # a common translation a of camera j's frame leaves the features unchanged
    a = np.array([0.03, -0.02, 0.05])
    Ta = np.eye(4)
    Ta[:3, 3] = a
    q2 = rng.normal(size=(50, 3)) * 0.01 + q
    x1, c1 = W.features(p, q2, M0)
    x2, c2 = W.features(p, q2 + a, Ta @ M0)
    assert np.allclose(x1, x2, atol=1e-12) and np.allclose(c2 - c1, a, atol=1e-15)


def test_increment_label_closed_forms():
    rng = np.random.default_rng(9)
    M0 = _rand_pose(rng)
    c = np.array([0.01, -0.02, 0.45])
    # pure translation a: omega = 0, u = a
    a = np.array([0.004, 0.01, -0.007])
    Ta = np.eye(4)
    Ta[:3, 3] = a
    y = W.label(M0, Ta @ M0, c)
    assert np.allclose(y, np.concatenate([np.zeros(3), a / W.S_U]), atol=1e-12)
    # pure rotation about the centre: u = 0, omega = axis * angle
    axis = np.array([1.0, 2.0, -2.0]) / 3.0
    R = O.se3_exp(np.concatenate([np.zeros(3), 0.15 * axis]))[:3, :3]
    Tc = np.eye(4)
    Tc[:3, :3] = R
    Tc[:3, 3] = c - R @ c
    y = W.label(M0, Tc @ M0, c)
    assert np.allclose(y, np.concatenate([0.15 * axis / W.S_W, np.zeros(3)]), atol=1e-12)
    # round trip
    M = _rand_pose(rng) @ M0
    assert np.allclose(W.increment(W.label(M0, M, c), c) @ M0, M, atol=1e-12)


def _graph(rng, N, fixed_node=0):
    T_true = [_rand_pose(rng, 0.5, 0.1) for _ in range(N)]
    T0 = [(_rand_pose(rng, 0.1, 0.01) @ T) if k != fixed_node else T.copy() for k, T in enumerate(T_true)]
    fixed = [k == fixed_node for k in range(N)]
    return T_true, T0, fixed


@pytest.mark.parametrize("N,fixed_node", [(2, 0), (5, 0), (6, 3)])
def test_average_recovers_consistent_increments(N, fixed_node):
    """Increments that all agree with one set of poses give those poses back
    (the anchor of both edge directions, then a zero right-hand side)."""
    rng = np.random.default_rng(10 + N)
    T_true, T0, fixed = _graph(rng, N, fixed_node)
    D = {(i, j): (T_true[j] @ _inv(T_true[i])) @ _inv(T0[j] @ _inv(T0[i]))
         for i in range(N) for j in range(i + 1, N)}
    T = W.average(T0, fixed, D)
    for k in range(N):
        assert np.allclose(T[k], T_true[k], atol=1e-12)


def test_average_is_gauge_equivariant():
    """Right-multiplying every pose by one object-frame transform G leaves
    every relative transform unchanged and so maps the result to T G."""
    rng = np.random.default_rng(11)
    N = 5
    T_true, T0, fixed = _graph(rng, N)
    D = {}
    for i in range(N):
        for j in range(i + 1, N):
            noise = _rand_pose(rng, 0.02, 0.003)                 # inconsistent edges
            D[(i, j)] = noise @ (T_true[j] @ _inv(T_true[i])) @ _inv(T0[j] @ _inv(T0[i]))
    G = _rand_pose(rng, 1.0, 0.2)
    A = W.average(T0, fixed, D)
    B = W.average([T @ G for T in T0], fixed, D)
    for k in range(N):
        assert np.allclose(B[k], A[k] @ G, atol=1e-10)
    # and it lands near the truth: within the edge noise
    assert max(S.rotation_angle(A[k][:3, :3] @ T_true[k][:3, :3].T) for k in range(N)) < 0.03


def test_average_two_nodes_closed_form():
    rng = np.random.default_rng(12)
    T0 = [_rand_pose(rng), _rand_pose(rng)]
    D = {(0, 1): _rand_pose(rng, 0.1, 0.01)}
    T = W.average(T0, [True, False], D)
    assert np.allclose(T[1], D[(0, 1)] @ T0[1], atol=1e-12) and np.array_equal(T[0], T0[0])
    T = W.average(T0, [False, True], D)         # the fixed node second
    M = D[(0, 1)] @ T0[1] @ _inv(T0[0])         # predicted T_1 T_0^-1
    assert np.allclose(T[1] @ _inv(T[0]), M, atol=1e-12) and np.array_equal(T[1], T0[1])
