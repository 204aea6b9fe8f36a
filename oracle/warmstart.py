"""FP64 oracle of the learned warm start.

Test infrastructure: only the tests, the package's smoke check and the
benchmark's CPU baseline leg import this module; the library never does.

The paper initialises the pose of each new frame from its sparse feature
matches with RANSAC and a closed-form least-squares fit (Sec. IV-B) and then
refines all poses of the retrieved keyframes with the pose-graph optimisation
(Sec. IV-D, Eq. 1-3).  The library replaces that initialisation, for every
node of a pose graph at once, by a small network on each edge's
correspondence set followed by a linear relative-pose averaging solve.  The
network is not in the paper; its definition is the library's own and is
written out here step by step in FP64, slowly and plainly:

  edge (i, j), i < j, with point pairs (p_k, q_k): p_k in camera i, q_k in
  camera j; M0 = T_j T_i^-1 at the initial poses (T maps object to camera).

  features   p'_k = M0 p_k,  c = mean_k q_k,
             x_k = ((p'_k - c) / S_P, (q_k - p'_k) / S_R)          (6 values)
  network    h1 = relu(W1 x + b1)       128   shared over the set
             h2 = relu(W2 h1 + b2)      256   shared over the set
             g  = max_k h2_k            256   (per channel; first index on ties)
             h3 = relu(W3 g + b3)       128
             y  = W4 h3 + b4            6     = (omega / S_W, u / S_U)
  increment  R = exp(omega) rotates about the set's centre c and u moves it:
             D(x) = R (x - c) + c + u,  M = D M0  (the edge's new relative pose)

Precision as run by the library: the weight matrices are BF16 copies of FP32
master weights, biases FP32, and the inputs of the 128 -> 256 contraction
(h1) are rounded to BF16; all sums are FP32 on the GPU (FP64 here).  The
rounding of h1 and of the weights is treated as the identity in the backward
pass (the gradient with respect to the master weights is that with respect
to their BF16 copies).  `exact=True` switches every rounding off; that
network is the one the finite-difference pins check.

Loss: mean over the edges of a minibatch of 1/2 |y - y*|^2, with the label
y* computed from the plain solver's converged poses.  Optimiser: Adam
(Kingma and Ba, 2015) on the FP32 master weights.

Relative-pose averaging (node initialisation from the edge increments):
  1. anchor: a free node j joined by an edge to a fixed node f (the lowest
     such f) takes the pose that edge predicts, T_j = D_fj T0_j for f < j and
     T_j = T0_j T0_f^-1 D_jf^-1 T0_f for j < f; other nodes keep T0;
  2. one linear least-squares solve for left increments d (T_i <- exp(d_i) T_i)
     over the free nodes: per edge the residual d_j - Ad(M_ij) d_i - e_ij with
     M_ij = T_j T_i^-1 at the anchored poses and e_ij = log(D_ij M0_ij M_ij^-1),
     weighted by diag(1/S_U^2 (x3), 1/S_W^2 (x3)) on (v, omega); normal
     equations solved by Cholesky;
  3. T_i <- exp(d_i) T_i.
"""
from __future__ import annotations

import numpy as np

from . import se3_exp, se3_log

S_P = 0.1      # m, scale of centred positions
S_R = 0.01     # m, scale of the pair offsets q - p'
S_W = 0.1      # rad, scale of the predicted rotation vector
S_U = 0.01     # m, scale of the predicted centre translation

LAYERS = [("W1", (128, 6)), ("b1", (128,)), ("W2", (256, 128)), ("b2", (256,)),
          ("W3", (128, 256)), ("b3", (128,)), ("W4", (6, 128)), ("b4", (6,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in LAYERS)


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), from the FP32 value: keep
    the upper 16 bits of the binary32 pattern after adding half an ulp of the
    kept part (0x7FFF plus the kept part's lowest bit)."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params) -> dict:
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (N_PARAMS,)
    out, o = {}, 0
    for name, shape in LAYERS:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).ravel() for name, _ in LAYERS])


def features(p, q, M0):
    """x (n, 6) and the centre c (3) of an edge's correspondence set."""
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    pp = p @ M0[:3, :3].T + M0[:3, 3]
    c = q.mean(axis=0)
    return np.concatenate([(pp - c) / S_P, (q - pp) / S_R], axis=1), c


def forward(params, x, exact: bool = False):
    """y (6) for one set x (n, 6), and what the backward pass needs."""
    L = unpack(params)
    rw = (lambda a: a) if exact else bf16
    W1, W2, W3, W4 = rw(L["W1"]), rw(L["W2"]), rw(L["W3"]), rw(L["W4"])
    x = np.asarray(x, np.float64)
    z1 = x @ W1.T + L["b1"]
    h1 = np.maximum(z1, 0.0)
    h1r = h1 if exact else bf16(h1)
    z2 = h1r @ W2.T + L["b2"]
    h2 = np.maximum(z2, 0.0)
    r = np.argmax(h2, axis=0)                     # first index of the maximum
    g = h2[r, np.arange(h2.shape[1])]
    z3 = W3 @ g + L["b3"]
    h3 = np.maximum(z3, 0.0)
    y = W4 @ h3 + L["b4"]
    cache = dict(x=x, z1=z1, h1r=h1r, r=r, g=g, z3=z3, h3=h3, W2=W2, W3=W3, W4=W4)
    return y, cache


def backward(params, cache, dy) -> np.ndarray:
    """Gradient of <dy, y> with respect to the flat parameter vector."""
    c = cache
    dy = np.asarray(dy, np.float64)
    G = {name: np.zeros(shape) for name, shape in LAYERS}
    G["W4"] = np.outer(dy, c["h3"])
    G["b4"] = dy.copy()
    dz3 = (c["W4"].T @ dy) * (c["z3"] > 0)
    G["W3"] = np.outer(dz3, c["g"])
    G["b3"] = dz3
    dg = c["W3"].T @ dz3
    dz2 = dg * (c["g"] > 0)                       # relu' at the selected row
    G["b2"] = dz2
    G["W2"] = dz2[:, None] * c["h1r"][c["r"], :]
    dh1 = np.zeros_like(c["h1r"])
    for ch in range(dz2.shape[0]):                # max-pool routes to row r[ch]
        if dz2[ch] != 0.0:
            dh1[c["r"][ch], :] += dz2[ch] * c["W2"][ch, :]
    dz1 = dh1 * (c["z1"] > 0)
    G["W1"] = dz1.T @ c["x"]
    G["b1"] = dz1.sum(axis=0)
    return pack(G)


def loss_and_grad(params, sets, targets, exact: bool = False):
    """Mean over the sets of 1/2 |y - y*|^2 and its gradient."""
    loss, grad = 0.0, np.zeros(N_PARAMS)
    for x, t in zip(sets, targets):
        y, cache = forward(params, x, exact)
        d = y - np.asarray(t, np.float64)
        loss += 0.5 * float(d @ d)
        grad += backward(params, cache, d)
    return loss / len(sets), grad / len(sets)


def adam(params, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """Step t (1-based) of Adam: returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def _inv(T):
    R, t = T[:3, :3], T[:3, 3]
    out = np.eye(4)
    out[:3, :3] = R.T
    out[:3, 3] = -R.T @ t
    return out


def rotation_exp(w):
    return se3_exp(np.concatenate([np.zeros(3), np.asarray(w, np.float64)]))[:3, :3]


def increment(y, c):
    """The edge's increment D (4x4) from a network output y and the centre c."""
    y = np.asarray(y, np.float64)
    R = rotation_exp(y[:3] * S_W)
    D = np.eye(4)
    D[:3, :3] = R
    D[:3, 3] = c + y[3:] * S_U - R @ c
    return D


def label(M0, M, c):
    """The output y* whose increment takes M0 to M (inverse of `increment`)."""
    D = M @ _inv(M0)
    w = se3_log(D)[3:]
    u = D[:3, 3] + D[:3, :3] @ c - c
    return np.concatenate([w / S_W, u / S_U])


def adjoint(T):
    """Ad_T for twists ordered (v, omega): [[R, [t]x R], [0, R]]."""
    R, t = T[:3, :3], T[:3, 3]
    tx = np.array([[0, -t[2], t[1]], [t[2], 0, -t[0]], [-t[1], t[0], 0]])
    A = np.zeros((6, 6))
    A[:3, :3] = R
    A[:3, 3:] = tx @ R
    A[3:, 3:] = R
    return A


def average(poses0, fixed, D):
    """Node poses from the edge increments D[(i, j)] (i < j) by anchoring and
    one FP64 linear least-squares solve (see the module docstring)."""
    T0 = [np.asarray(T, np.float64) for T in poses0]
    N = len(T0)
    fixed = [bool(f) for f in fixed]
    T = [t.copy() for t in T0]
    for j in range(N):
        if fixed[j]:
            continue
        for f in range(N):
            if not fixed[f]:
                continue
            if f < j and (f, j) in D:
                T[j] = D[(f, j)] @ T0[j]
                break
            if j < f and (j, f) in D:
                T[j] = T0[j] @ _inv(T0[f]) @ _inv(D[(j, f)]) @ T0[f]
                break
    free = [k for k in range(N) if not fixed[k]]
    if not free:
        return T
    col = {k: n for n, k in enumerate(free)}
    n = 6 * len(free)
    H = np.zeros((n, n))
    b = np.zeros(n)
    W = np.diag([1 / S_U ** 2] * 3 + [1 / S_W ** 2] * 3)
    for (i, j), Dij in D.items():
        M0 = T0[j] @ _inv(T0[i])
        M = T[j] @ _inv(T[i])
        e = se3_log(Dij @ M0 @ _inv(M))
        A = adjoint(M)
        J = {}
        if not fixed[j]:
            J[j] = np.eye(6)
        if not fixed[i]:
            J[i] = -A
        for a, Ja in J.items():
            b[6 * col[a]:6 * col[a] + 6] += Ja.T @ W @ e
            for bb, Jb in J.items():
                H[6 * col[a]:6 * col[a] + 6, 6 * col[bb]:6 * col[bb] + 6] += Ja.T @ W @ Jb
    L = np.linalg.cholesky(H)
    d = np.linalg.solve(L.T, np.linalg.solve(L, b))
    for k in free:
        T[k] = se3_exp(d[6 * col[k]:6 * col[k] + 6]) @ T[k]
    return T
