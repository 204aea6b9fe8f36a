"""Oracle of the memory pool's keyframe selection (Sec. IV-C) and pool
augmentation (Sec. IV-E).

Test infrastructure: only the tests import this module; the library never
does.  Plain Python and numpy, FP64, written from the paper's description:

  * edge weight of two keyframes: the geodesic distance of their rotations,
    arccos((tr(R_i^T R_j) - 1) / 2) (the minimum H-subgraph objective);
  * greedy selection: start from {I_0} (the pool's first frame) and add, one
    at a time, the pool frame whose summed geodesic distance to the current
    frame I_t and to every frame selected so far is smallest, until K frames
    are selected or the pool is exhausted (ties: the earlier pool entry);
  * augmentation: the current frame joins the pool when its rotation
    geodesic to every pool frame exceeds the threshold (10 degrees; the text
    writes it as "arccos(10 deg)", read as 10 degrees).
"""
from __future__ import annotations

import math


def geodesic(Ra, Rb) -> float:
    tr = sum(Ra[k][0] * Rb[k][0] + Ra[k][1] * Rb[k][1] + Ra[k][2] * Rb[k][2] for k in range(3))
    c = (tr - 1.0) / 2.0
    return math.acos(max(-1.0, min(1.0, c)))


def select(pool_rot, R_cur, K: int) -> list[int]:
    """Indices into pool_rot of the selected keyframes, in selection order."""
    n = len(pool_rot)
    if n == 0 or K <= 0:
        return []
    chosen = [0]
    while len(chosen) < min(K, n):
        best, best_cost = -1, None
        for f in range(n):
            if f in chosen:
                continue
            cost = geodesic(pool_rot[f], R_cur) + sum(geodesic(pool_rot[f], pool_rot[c]) for c in chosen)
            if best_cost is None or cost < best_cost:
                best, best_cost = f, cost
        chosen.append(best)
    return chosen


def is_novel(pool_rot, R_cur, min_deg: float = 10.0) -> bool:
    lim = math.radians(min_deg)
    return all(geodesic(R, R_cur) > lim for R in pool_rot)
