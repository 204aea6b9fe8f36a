"""Keyframe selection (Sec. IV-C) and memory-pool augmentation (Sec. IV-E)
for a sequence: which stored frames form the pose graph of each frame.

The selection and the augmentation rule are library calls
(bt_select_keyframes, bt_is_novel_view: host code in libbt); this module
only walks a sequence with them.
"""
from __future__ import annotations

import numpy as np

from . import bt


def plan_sequence(rotations: np.ndarray, max_nodes: int = 10, min_deg: float = 10.0):
    """Graph of every time step t >= 1 of a sequence: the keyframes selected
    for frame t (at most max_nodes - 1, I_0 first) followed by t itself; the
    pool is augmented after each step.  Returns (graphs, pool_history)."""
    R = np.asarray(rotations, dtype=np.float64)
    pool = [0]
    graphs = []
    history = []
    for t in range(1, len(R)):
        sel = bt.select_keyframes(R[pool], R[t], max_nodes - 1)
        graphs.append([pool[k] for k in sel] + [t])
        if bt.is_novel_view(R[pool], R[t], min_deg):
            pool.append(t)
        history.append(list(pool))
    return graphs, history
