"""Helpers shared by the GPU parity tests (test infrastructure)."""
import numpy as np

import oracle as O
import synthgen as S


def pose_err(A, B):
    """Largest rotation angle (rad) and translation component (m) between two
    pose lists."""
    rot = max(S.rotation_angle(a[:3, :3] @ b[:3, :3].T) for a, b in zip(A, B))
    tr = max(np.abs(a[:3, 3] - b[:3, 3]).max() for a, b in zip(A, B))
    return rot, tr


def oracle_self_spread(g, iters, starts=3, scale=1e-7, seed=1):
    """How far the oracle's own free-running solve moves when its start is
    perturbed by ~`scale` rad and scale/10 m -- by default the size of
    rounding a transform to single precision (2^-24 ~ 6e-8 relative), which
    is what the GPU path does to every relative pose: (unperturbed result,
    rad, m, relative cost), maxima over `starts` perturbed starts.
    Projective re-association makes the Gauss-Newton map discontinuous, so a
    few decisions that flip at that scale move the end point; this measures
    that floor for the graph at hand."""
    base = O.solve(g, iters)
    rng = np.random.default_rng(seed)
    rot = tr = cost = 0.0
    for _ in range(starts):
        P = g.pose_init.copy()
        for n in range(1, len(P)):
            if g.fixed[n]:
                continue
            P[n] = O.se3_exp(np.r_[rng.normal(size=3) * 0.1 * scale, rng.normal(size=3) * scale]) @ P[n]
        r = O.solve(g, iters, poses=P)
        a, b = pose_err(r["poses"], base["poses"])
        rot, tr = max(rot, a), max(tr, b)
        cost = max(cost, abs(r["cost_final"] - base["cost_final"]) / base["cost_final"])
    return base, rot, tr, cost
