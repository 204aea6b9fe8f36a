"""Oracle of the coarse registration of Sec. IV-B: RANSAC over 3-point
samples of a correspondence set, each hypothesis fitted by the closed-form
least-squares method of Arun et al. (1987).

Test infrastructure: only the tests import this module; the library never
does.  Plain numpy, written from the paper's description:

  * a sample is 3 correspondences (p_k in camera i, q_k in camera j);
  * a hypothesis (R, t) minimises sum |R p_k + t - q_k|^2 over the sample:
    centroids, cross-covariance S = sum (p - p_c)(q - q_c)^T, S = U D V^T
    (a library SVD), R = V diag(1, 1, det(V U^T)) U^T, t = q_c - R p_c;
  * a correspondence is an inlier when |R p + t - q| < delta (5 mm in the
    paper; its normal-angle gate needs normals, which correspondence sets
    here do not carry);
  * the result is the hypothesis with the most inliers (ties: the earlier
    sample); optionally (refine) refitted on all its inliers.

Random numbers: sample indices come from the counter-based SplitMix64
generator (Steele, Lea, Flood 2014; constants as published by Vigna):
value(seed, c) = mix(seed + (c + 1) * 0x9E3779B97F4A7C15) with
mix(z) = z' ^ (z' >> 31), z' from two xorshift-multiply rounds.  Sample h
draws counters 16 h, 16 h + 1, ... and keeps the first three distinct
indices value % n.  Inlier tests are evaluated in IEEE single precision
with the operation order written in `score`, so that any implementation
of the same specification takes the same decisions.
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, counter: int) -> int:
    z = (seed + (counter + 1) * GOLDEN) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def sample(seed: int, h: int, n: int):
    """Indices of sample h (three distinct when n >= 3), or None."""
    if n < 3:
        return None
    out = []
    for c in range(16):
        k = splitmix64(seed, 16 * h + c) % n
        if k not in out:
            out.append(k)
            if len(out) == 3:
                return out
    return None


def arun(p, q):
    """(R, t) minimising sum |R p + t - q|^2 (FP64)."""
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    pc, qc = p.mean(axis=0), q.mean(axis=0)
    S = (p - pc).T @ (q - qc)
    U, _, Vt = np.linalg.svd(S)
    V = Vt.T
    d = np.sign(np.linalg.det(V @ U.T))
    R = V @ np.diag([1.0, 1.0, d if d != 0 else 1.0]) @ U.T
    return R, qc - R @ pc


def score(R, t, p, q, delta):
    """Inlier mask, single precision: u = ((R00 px + R01 py) + R02 pz) + tx
    (each product and sum rounded), e = u - q, inlier iff
    (ex ex + ey ey) + ez ez < fl(delta^2)."""
    f = np.float32
    R = np.asarray(R, np.float64).astype(f)
    t = np.asarray(t, np.float64).astype(f)
    p = np.asarray(p, f)
    q = np.asarray(q, f)
    u = [((R[r, 0] * p[:, 0] + R[r, 1] * p[:, 1]) + R[r, 2] * p[:, 2]) + t[r] for r in range(3)]
    e = [u[r] - q[:, r] for r in range(3)]
    d2 = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]
    return d2 < f(delta * delta)


def degenerate(p3, eps: float = 1e-12) -> bool:
    """Collinear (or coincident) sample: no unique rotation."""
    p3 = np.asarray(p3, np.float64)
    a, b = p3[1] - p3[0], p3[2] - p3[0]
    return float(np.linalg.norm(np.cross(a, b))) <= eps * max(1e-30, float(a @ a + b @ b))


def ransac(p, q, hypotheses: int, seed: int, delta: float = 0.005, refine: bool = False):
    """(M 4x4 with q ~ M p, inlier count, best sample index or -1)."""
    p = np.asarray(p, np.float32)
    q = np.asarray(q, np.float32)
    n = len(p)
    best, best_cnt, best_Rt = -1, -1, None
    for h in range(hypotheses):
        idx = sample(seed, h, n)
        if idx is None or degenerate(p[idx]):
            continue
        R, t = arun(p[idx], q[idx])
        cnt = int(score(R, t, p, q, delta).sum())
        if cnt > best_cnt:
            best, best_cnt, best_Rt = h, cnt, (R, t)
    M = np.eye(4)
    if best < 0:
        return M, 0, -1
    R, t = best_Rt
    if refine:
        inl = score(R, t, p, q, delta)
        if inl.sum() >= 3:
            R, t = arun(p[inl], q[inl])
    M[:3, :3] = R
    M[:3, 3] = t
    return M, best_cnt, best
