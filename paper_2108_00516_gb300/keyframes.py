"""Keyframe selection (Sec. IV-C) and memory-pool augmentation (Sec. IV-E).

Host-side logic that decides which stored frames form the pose graph of the
current frame; the graph itself is then solved by the CUDA library.
"""
from __future__ import annotations

import numpy as np


def rotation_geodesic(Ra: np.ndarray, Rb: np.ndarray) -> float:
    """Geodesic distance arccos((tr(Ra^T Rb) - 1) / 2) between rotations
    (the edge weight of the minimum H-subgraph problem, Sec. IV-C)."""
    c = (np.trace(Ra.T @ Rb) - 1.0) * 0.5
    return float(np.arccos(np.clip(c, -1.0, 1.0)))


def select_keyframes(pool: list[int], rotations, R_current: np.ndarray, K: int) -> list[int]:
    """Greedy selection of Sec. IV-C: start from the first frame I_0 (pool[0]),
    then repeatedly add the pool frame whose summed geodesic distance to the
    current frame and to every frame selected so far is smallest, until K
    frames are selected (or the pool is exhausted).  Ties go to the earlier
    pool entry."""
    if not pool:
        return []
    chosen = [pool[0]]
    rest = list(pool[1:])
    cost = {f: rotation_geodesic(rotations[f], R_current) + rotation_geodesic(rotations[f], rotations[pool[0]])
            for f in rest}
    while len(chosen) < K and rest:
        best = min(rest, key=lambda f: (cost[f], rest.index(f)))
        chosen.append(best)
        rest.remove(best)
        for f in rest:
            cost[f] += rotation_geodesic(rotations[f], rotations[best])
    return chosen


def is_novel_view(R_current: np.ndarray, pool: list[int], rotations, min_deg: float = 10.0) -> bool:
    """Pool augmentation rule of Sec. IV-E: the frame joins the pool when its
    rotation geodesic to every pool keyframe exceeds min_deg."""
    lim = np.deg2rad(min_deg)
    return all(rotation_geodesic(rotations[f], R_current) > lim for f in pool)


def plan_sequence(rotations: np.ndarray, max_nodes: int = 10, min_deg: float = 10.0):
    """Graph of every time step t >= 1 of a sequence: the keyframes selected
    for frame t (at most max_nodes - 1, I_0 first) followed by t itself; the
    pool is augmented after each step.  Returns (graphs, pool_history)."""
    pool = [0]
    graphs = []
    history = []
    for t in range(1, len(rotations)):
        kf = select_keyframes(pool, rotations, rotations[t], max_nodes - 1)
        graphs.append(kf + [t])
        if is_novel_view(rotations[t], pool, rotations, min_deg):
            pool.append(t)
        history.append(list(pool))
    return graphs, history
