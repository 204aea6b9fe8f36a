"""Seeded training graphs for the learned warm start.

Same object, camera, noise, correspondence and initialisation model as the
batched workload (box-plus-ellipsoid object, mask coverage U[5, 40] % at the
first view, U{100..800} correspondences per pair with U[10, 30] % outliers,
1 mm depth noise, init perturbed by 5 deg / 1 cm, frame 0 fixed), with two
changes that make 100k graphs cheap to draw: 2 to 4 views at 160x120, and a
coarse coverage search.  Consecutive views are 1 to 6 trajectory steps apart,
so the pairs span the viewpoint changes of the short- and long-range edges of
larger graphs.  Holds no pose-graph arithmetic.
"""
from __future__ import annotations

import numpy as np

from .scene import (TINY_CAMERA, Shape, SynthGraph, _rng, distance_for_coverage, make_matches, make_pose,
                    perturb_pose, random_rotation, render, step_pose)

TRAIN_SEED = 6000
HELDOUT_SEED = 7000


def training_graph(graph_id: int, seed_base: int = TRAIN_SEED) -> SynthGraph:
    rng = _rng(seed_base, 99, graph_id)
    n = int(rng.integers(2, 5))
    cov = float(rng.uniform(0.05, 0.40))
    n_m = int(rng.integers(100, 801))
    outl = float(rng.uniform(0.10, 0.30))
    skips = rng.integers(1, 7, n - 1)
    cam = TINY_CAMERA
    g_rng = _rng(seed_base, graph_id)
    shape = Shape.random(g_rng)
    R0 = random_rotation(g_rng)
    d = distance_for_coverage(shape, cam, R0, cov, probe_width=40, steps=14)
    t0 = np.array([0.0, 0.0, d])
    T = make_pose(R0, t0)
    poses = [T]
    for k in range(n - 1):
        for _ in range(int(skips[k])):
            T = step_pose(T, t0, g_rng)
        poses.append(T)
    pose_true = np.stack(poses)
    renders = [render(shape, cam, pose_true[k], _rng(seed_base, graph_id, 1, k)) for k in range(n)]
    matches = []
    for i in range(n):
        for j in range(i + 1, n):
            pi, pj, _ = make_matches(shape, cam, cam, pose_true[i], pose_true[j], renders[i], renders[j],
                                     n_m, outl, _rng(seed_base, graph_id, 2, i, j))
            matches.append((i, j, pi, pj))
    prng = _rng(seed_base, graph_id, 3)
    pose_init = pose_true.copy()
    for k in range(1, n):
        pose_init[k] = perturb_pose(pose_true[k], 5.0, 0.01, prng)
    fixed = np.zeros(n, np.int32)
    fixed[0] = 1
    for r in renders:
        r.depth_clean = None
        r.normals_true = None
    return SynthGraph([cam] * n, renders, pose_true, pose_init, fixed, matches, shape,
                      dict(seed=(seed_base, graph_id), n_frames=n, coverage=cov, matches=n_m, outliers=outl))


def _job(args):
    return training_graph(*args)


def training_graphs(ids, seed_base: int = TRAIN_SEED, workers: int | None = None, chunksize: int = 64):
    """Yields training graphs in id order, made in forked worker processes
    (the pool is created by the caller's first call; create it before CUDA
    is initialised, see TrainingPool)."""
    return [training_graph(k, seed_base) for k in ids] if workers == 1 else \
        TrainingPool(workers).map(ids, seed_base, chunksize)


class TrainingPool:
    """A fork-based process pool for training graphs.  Create it before the
    calling process initialises CUDA; it can be used afterwards."""

    def __init__(self, workers: int | None = None):
        import multiprocessing as mp
        import os
        import sys
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_initialized():
            raise RuntimeError("TrainingPool forks worker processes; create it before CUDA is initialised")
        self.workers = workers or max(1, min(64, os.cpu_count() or 1))
        self.pool = mp.get_context("fork").Pool(self.workers)

    def map(self, ids, seed_base: int = TRAIN_SEED, chunksize: int = 64):
        return self.pool.imap(_job, [(k, seed_base) for k in ids], chunksize)

    def close(self):
        self.pool.terminate()
        self.pool.join()


# flat parameter layout of the warm-start network (input layout only: the
# library and the oracle each unpack it themselves)
WARMSTART_LAYERS = [("W1", (128, 6)), ("b1", (128,)), ("W2", (256, 128)), ("b2", (256,)),
                    ("W3", (128, 256)), ("b3", (128,)), ("W4", (6, 128)), ("b4", (6,))]


def warmstart_init(seed: int) -> np.ndarray:
    """Seeded FP32 initial parameters: weights U(-sqrt(6/fan_in), +sqrt(6/fan_in))
    (He uniform), last layer scaled by 0.1, biases U(-0.01, 0.01)."""
    rng = _rng(8000, seed)
    out = []
    for name, shape in WARMSTART_LAYERS:
        if name.startswith("W"):
            a = np.sqrt(6.0 / shape[1]) * (0.1 if name == "W4" else 1.0)
            out.append(rng.uniform(-a, a, shape).ravel())
        else:
            out.append(rng.uniform(-0.01, 0.01, shape))
    return np.concatenate(out).astype(np.float32)
