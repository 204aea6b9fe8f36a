"""Seeded synthetic RGB-D sequences (the paper-shaped workload: 640x480,
fx = fy = 600, mask coverage 15-30 %, 500 correspondences per frame pair with
20 % outliers, camera steps of up to 10 deg and 2 cm).

Frames and correspondence sets are produced on demand and cached; `prefetch`
renders many of them in a pool of forked worker processes, which must happen
before the calling process initialises CUDA."""
from __future__ import annotations

import os
from concurrent.futures import ProcessPoolExecutor
from dataclasses import dataclass, field
import multiprocessing as mp

import numpy as np

from .scene import (VGA_CAMERA, Camera, Shape, _rng, distance_for_coverage, make_matches,
                    make_pose, perturb_pose, random_rotation, render, step_pose)


@dataclass
class Sequence:
    seed: int
    cam: Camera
    shape: Shape
    poses_true: np.ndarray                 # (T, 4, 4)
    n_matches: int = 500
    outlier_frac: float = 0.2
    depth_sigma: float = 0.001
    _frames: dict = field(default_factory=dict)
    _matches: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.poses_true)

    def frame(self, t: int):
        r = self._frames.get(t)
        if r is None:
            r = _render_frame(self.shape, self.cam, self.poses_true[t], self.seed, t, self.depth_sigma)
            self._frames[t] = r
        return r

    def matches(self, i: int, j: int):
        """(pts_i, pts_j) for frames i < j."""
        assert i < j
        m = self._matches.get((i, j))
        if m is None:
            m = _pair_matches(self, i, j)
            self._matches[(i, j)] = m
        return m

    def init_pose(self, t: int, graph_key: int, rot_deg: float = 5.0, trans_m: float = 0.01) -> np.ndarray:
        """Initial pose of frame t in the graph solved at time `graph_key`:
        the true pose perturbed by exactly rot_deg / trans_m (frame 0 exact)."""
        if t == 0:
            return self.poses_true[0].copy()
        return perturb_pose(self.poses_true[t], rot_deg, trans_m, _rng(self.seed, 4, graph_key, t))

    def prefetch(self, frames=(), pairs=(), workers: int | None = None):
        """Render `frames` and draw the correspondence sets `pairs` in a pool
        of forked worker processes.  Forking is only safe before the calling
        process has initialised CUDA, which is checked."""
        frames = sorted({t for t in frames if t not in self._frames} |
                        {t for p in pairs for t in p if t not in self._frames})
        pairs = [p for p in pairs if p not in self._matches]
        if not frames and not pairs:
            return
        _check_no_cuda()
        workers = workers or max(1, min(32, os.cpu_count() or 1))
        ctx = mp.get_context("fork")
        global _SEQ
        _SEQ = self
        try:
            if frames:
                with ProcessPoolExecutor(workers, mp_context=ctx) as ex:
                    for t, r in zip(frames, ex.map(_render_job, frames, chunksize=4)):
                        self._frames[t] = r
            if pairs:
                # workers forked now inherit every rendered frame; only the
                # correspondence arrays travel back
                with ProcessPoolExecutor(workers, mp_context=ctx) as ex:
                    for p, m in zip(pairs, ex.map(_pair_job, pairs, chunksize=16)):
                        self._matches[p] = m
        finally:
            _SEQ = None


_SEQ = None


def _check_no_cuda():
    import sys
    torch = sys.modules.get("torch")
    if torch is not None and torch.cuda.is_initialized():
        raise RuntimeError("Sequence.prefetch forks worker processes; call it before CUDA is initialised")


def _render_job(t):
    s = _SEQ
    r = _render_frame(s.shape, s.cam, s.poses_true[t], s.seed, t, s.depth_sigma)
    r.normals_true = None
    return r


def _pair_job(p):
    return _pair_matches(_SEQ, p[0], p[1])


def _render_frame(shape, cam, T, seed, t, depth_sigma):
    return render(shape, cam, T, _rng(seed, 1, t), depth_sigma)


def _pair_matches(seq: Sequence, i: int, j: int):
    ri, rj = seq.frame(i), seq.frame(j)
    pi, pj, _ = make_matches(seq.shape, seq.cam, seq.cam, seq.poses_true[i], seq.poses_true[j], ri, rj,
                             seq.n_matches, seq.outlier_frac, _rng(seq.seed, 2, i, j), noise=seq.depth_sigma)
    return pi, pj


def paper_sequence(seed: int = 2000, n_frames: int = 300, cam: Camera = VGA_CAMERA,
                   coverage_range=(0.15, 0.30)) -> Sequence:
    """300-frame sequence of one random object; the first view's distance is
    set so that the mask covers U[15, 30] % of the image."""
    rng = _rng(seed)
    shape = Shape.random(rng)
    R0 = random_rotation(rng)
    d = distance_for_coverage(shape, cam, R0, float(rng.uniform(*coverage_range)))
    t0 = np.array([0.0, 0.0, d])
    poses = [make_pose(R0, t0)]
    for _ in range(1, n_frames):
        poses.append(step_pose(poses[-1], t0, rng))
    return Sequence(seed, cam, shape, np.stack(poses))
