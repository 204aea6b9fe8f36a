"""Seeded synthetic RGB-D scenes for the pose-graph workloads.

This module makes inputs only: it ray-casts an analytic box-plus-ellipsoid
object, adds depth noise, estimates normals by finite differences, draws
sparse correspondences with outliers, walks a camera trajectory and perturbs
initial poses.  It contains none of the pose-graph arithmetic (no residuals,
Jacobians, association, reduction or solver); both the CPU oracle and the
CUDA library consume what it produces.

Conventions shared with the library interface:
  * pose T (4x4, float64, row-major) maps object coordinates to camera
    coordinates, X_c = R X_o + t (the paper's object pose in the camera
    frame, Sec. III);
  * pixel (u, v) has its centre at integer coordinates; the pinhole model is
    u = fx X/Z + cx, v = fy Y/Z + cy;
  * depth is metres along the optical axis, 0 where nothing was hit;
  * normals are unit vectors in the camera frame pointing toward the camera,
    NaN where they cannot be estimated.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# small rotation helpers (quaternion based; used only to synthesise poses)
# --------------------------------------------------------------------------

def quat_to_matrix(q: np.ndarray) -> np.ndarray:
    """Unit quaternion (w, x, y, z) -> 3x3 rotation matrix."""
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def axis_angle_matrix(axis: np.ndarray, angle: float) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    h = 0.5 * angle
    return quat_to_matrix(np.concatenate([[np.cos(h)], np.sin(h) * axis]))


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    return quat_to_matrix(rng.normal(size=4))


def make_pose(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def pose_inverse(T: np.ndarray) -> np.ndarray:
    R, t = T[:3, :3], T[:3, 3]
    return make_pose(R.T, -R.T @ t)


def rotation_angle(R: np.ndarray) -> float:
    """Geodesic angle of a rotation matrix (radians)."""
    c = (np.trace(R) - 1.0) * 0.5
    return float(np.arccos(np.clip(c, -1.0, 1.0)))


# --------------------------------------------------------------------------
# camera and object
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_tuple(self):
        return (self.fx, self.fy, self.cx, self.cy, self.width, self.height)


TINY_CAMERA = Camera(140.0, 140.0, 80.0, 60.0, 160, 120)
VGA_CAMERA = Camera(600.0, 600.0, 320.0, 240.0, 640, 480)
QVGA_CAMERA = Camera(300.0, 300.0, 160.0, 120.0, 320, 240)


@dataclass(frozen=True)
class Shape:
    """Union of an axis-aligned box (centred at the object origin) and an
    axis-aligned ellipsoid (centre offset), both in object coordinates."""
    box_half: np.ndarray
    ell_axes: np.ndarray
    ell_center: np.ndarray
    with_ellipsoid: bool = True

    @staticmethod
    def random(rng: np.random.Generator, with_ellipsoid: bool = True) -> "Shape":
        return Shape(box_half=rng.uniform(0.03, 0.08, 3),
                     ell_axes=rng.uniform(0.02, 0.06, 3),
                     ell_center=rng.uniform(-0.04, 0.04, 3),
                     with_ellipsoid=with_ellipsoid)


def cast_rays(shape: Shape, T: np.ndarray, dirs_cam: np.ndarray):
    """Intersect camera rays X = s * d (d with d_z = 1) with the object.

    Returns (s, normal_cam) with s = inf where the ray misses; since d_z = 1
    the hit depth Z equals s.  normal_cam is the analytic outward normal in
    the camera frame.
    """
    R, t = T[:3, :3], T[:3, 3]
    o = -R.T @ t                       # camera centre in object frame
    d = dirs_cam @ R                   # rows: R^T d
    shp = d.shape[:-1]
    best = np.full(shp, np.inf)
    nrm = np.zeros(shp + (3,))

    hb = shape.box_half
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (-hb - o) * inv
        t2 = (hb - o) * inv
    t1 = np.nan_to_num(t1, nan=-np.inf)
    t2 = np.nan_to_num(t2, nan=np.inf)
    tn = np.minimum(t1, t2)
    tf = np.maximum(t1, t2)
    tnear = tn.max(-1)
    tfar = tf.min(-1)
    hit = (tfar >= tnear) & (tnear > 0)
    ax = tn.argmax(-1)
    n_obj = np.zeros(shp + (3,))
    sgn = -np.sign(np.take_along_axis(d, ax[..., None], -1)[..., 0])
    np.put_along_axis(n_obj, ax[..., None], sgn[..., None], -1)
    best = np.where(hit, tnear, best)
    nrm = np.where(hit[..., None], n_obj, nrm)

    if shape.with_ellipsoid:
        ea, ec = shape.ell_axes, shape.ell_center
        o2 = (o - ec) / ea
        d2 = d / ea
        a = (d2 * d2).sum(-1)
        b = 2.0 * (d2 * o2).sum(-1)
        c = (o2 * o2).sum() - 1.0
        disc = b * b - 4 * a * c
        ok = disc >= 0
        s = np.where(ok, (-b - np.sqrt(np.where(ok, disc, 0.0))) / (2 * a), np.inf)
        hit_e = ok & (s > 0) & (s < best)
        with np.errstate(invalid="ignore"):
            x = o + np.where(hit_e, s, 0.0)[..., None] * d
        ne = (x - ec) / (ea * ea)
        ne = ne / np.linalg.norm(ne, axis=-1, keepdims=True).clip(1e-30)
        best = np.where(hit_e, s, best)
        nrm = np.where(hit_e[..., None], ne, nrm)

    normal_cam = nrm @ R.T
    return best, normal_cam


def pixel_rays(cam: Camera) -> np.ndarray:
    v, u = np.mgrid[0:cam.height, 0:cam.width].astype(np.float64)
    return np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy,
                     np.ones_like(u)], -1)


def backproject(depth: np.ndarray, cam: Camera) -> np.ndarray:
    v, u = np.mgrid[0:cam.height, 0:cam.width].astype(np.float64)
    z = depth.astype(np.float64)
    return np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], -1)


def masked_box_smooth(depth: np.ndarray, s: int) -> np.ndarray:
    """Mean of the valid (> 0) depths in a (2s+1)^2 window, at valid pixels
    only (normalised box filter; background stays 0)."""
    d = np.where(depth > 0, depth, 0.0).astype(np.float64)
    if s <= 0:
        return d
    v = (depth > 0).astype(np.float64)

    def box(a):
        c = np.pad(a, s).cumsum(0).cumsum(1)
        c = np.pad(c, ((1, 0), (1, 0)))
        w = 2 * s + 1
        return c[w:, w:] - c[:-w, w:] - c[w:, :-w] + c[:-w, :-w]

    num, den = box(d), box(v)
    return np.where((depth > 0) & (den > 0), num / np.maximum(den, 1.0), 0.0)


def fd_normals(depth: np.ndarray, cam: Camera, k: int = 1) -> np.ndarray:
    """Normals from central differences of back-projected depth, half-width
    k pixels; NaN where any of the four neighbours has no depth."""
    H, W = depth.shape
    P = backproject(depth, cam)
    valid = depth > 0
    out = np.full((H, W, 3), np.nan)
    if H <= 2 * k or W <= 2 * k:
        return out
    dPu = P[k:H - k, 2 * k:] - P[k:H - k, :W - 2 * k]
    dPv = P[2 * k:, k:W - k] - P[:H - 2 * k, k:W - k]
    n = np.cross(dPv, dPu)
    ok = (valid[k:H - k, k:W - k] & valid[k:H - k, 2 * k:] & valid[k:H - k, :W - 2 * k]
          & valid[2 * k:, k:W - k] & valid[:H - 2 * k, k:W - k])
    nn = np.linalg.norm(n, axis=-1, keepdims=True)
    ok &= nn[..., 0] > 0
    n = n / np.where(nn > 0, nn, 1.0)
    flip = (n * P[k:H - k, k:W - k]).sum(-1) > 0
    n = np.where(flip[..., None], -n, n)
    n = np.where(ok[..., None], n, np.nan)
    out[k:H - k, k:W - k] = n
    return out


@dataclass
class Render:
    depth: np.ndarray          # float32 HxW, noisy, 0 = background
    normals: np.ndarray        # float32 HxWx3
    mask: np.ndarray           # uint8 HxW
    depth_clean: np.ndarray    # float64 HxW (inf-free, 0 = background)
    normals_true: np.ndarray   # float64 HxWx3 analytic (0 on background)


def bounding_radius(shape: Shape) -> float:
    r = float(np.linalg.norm(shape.box_half))
    if shape.with_ellipsoid:
        r = max(r, float(np.linalg.norm(shape.ell_center) + shape.ell_axes.max()))
    return r


def image_bbox(shape: Shape, cam: Camera, T: np.ndarray):
    """Conservative pixel box (u0, u1, v0, v1), end-exclusive, that contains
    the projection of the object's bounding sphere; None = whole image."""
    c, rad = T[:3, 3], bounding_radius(shape) * 1.01
    if c[2] - rad <= 1e-3:
        return None
    zs = (c[2] - rad, c[2] + rad)
    xs = [(c[0] + a) / z for a in (-rad, rad) for z in zs]
    ys = [(c[1] + a) / z for a in (-rad, rad) for z in zs]
    u0 = int(np.floor(cam.fx * min(xs) + cam.cx)) - 1
    u1 = int(np.ceil(cam.fx * max(xs) + cam.cx)) + 2
    v0 = int(np.floor(cam.fy * min(ys) + cam.cy)) - 1
    v1 = int(np.ceil(cam.fy * max(ys) + cam.cy)) + 2
    return (max(u0, 0), min(u1, cam.width), max(v0, 0), min(v1, cam.height))


def cast_image(shape: Shape, cam: Camera, T: np.ndarray):
    """Ray-cast every pixel centre; only rays inside the object's projected
    bounding box are traced (the rest miss by construction)."""
    s = np.full((cam.height, cam.width), np.inf)
    n = np.zeros((cam.height, cam.width, 3))
    bb = image_bbox(shape, cam, T)
    if bb is None:
        return cast_rays(shape, T, pixel_rays(cam))
    u0, u1, v0, v1 = bb
    if u0 >= u1 or v0 >= v1:
        return s, n
    v, u = np.mgrid[v0:v1, u0:u1].astype(np.float64)
    dirs = np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, np.ones_like(u)], -1)
    ss, nn = cast_rays(shape, T, dirs)
    s[v0:v1, u0:u1] = ss
    n[v0:v1, u0:u1] = nn
    return s, n


def render(shape: Shape, cam: Camera, T: np.ndarray, rng: np.random.Generator | None,
           depth_sigma: float = 0.001, fd_halfwidth: int | None = None,
           analytic_normals: bool = False) -> Render:
    s, n_true = cast_image(shape, cam, T)
    hit = np.isfinite(s)
    clean = np.where(hit, s, 0.0)
    depth = clean.copy()
    if depth_sigma > 0 and rng is not None:
        depth = np.where(hit, clean + rng.normal(0.0, depth_sigma, clean.shape), 0.0)
        depth = np.where(hit, np.maximum(depth, 1e-3), 0.0)
    if analytic_normals:
        normals = np.where(hit[..., None], n_true, np.nan)
    else:
        # central differences over +-k pixels with k = W/160 (the same angular
        # stencil at every resolution), on the depth pre-smoothed by a masked
        # (2k-1)^2 box filter; at 160x120 this is plain +-1 pixel differences
        k = fd_halfwidth if fd_halfwidth is not None else max(1, cam.width // 160)
        normals = fd_normals(masked_box_smooth(depth, k - 1), cam, k)
    return Render(depth=depth.astype(np.float32), normals=normals.astype(np.float32),
                  mask=hit.astype(np.uint8), depth_clean=clean,
                  normals_true=np.where(hit[..., None], n_true, 0.0))


def coverage(shape: Shape, cam: Camera, T: np.ndarray) -> float:
    s, _ = cast_image(shape, cam, T)
    return float(np.isfinite(s).mean())


def distance_for_coverage(shape: Shape, cam: Camera, R: np.ndarray, target: float,
                          lateral: np.ndarray | None = None, probe_width: int = 160,
                          steps: int = 22) -> float:
    """Bisect the object distance so that the mask covers `target` of the image."""
    lo, hi = 0.08, 3.0
    lat = np.zeros(2) if lateral is None else lateral
    # coverage is (nearly) resolution independent: bisect on a camera of at
    # most probe_width pixels across
    f = max(1, cam.width // probe_width)
    small = Camera(cam.fx / f, cam.fy / f, (cam.cx + 0.5) / f - 0.5, (cam.cy + 0.5) / f - 0.5,
                   cam.width // f, cam.height // f)
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        c = coverage(shape, small, make_pose(R, np.array([lat[0], lat[1], mid])))
        if c > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# --------------------------------------------------------------------------
# sparse correspondences
# --------------------------------------------------------------------------

def make_matches(shape: Shape, cam_i: Camera, cam_j: Camera, T_i: np.ndarray, T_j: np.ndarray,
                 r_i: Render, r_j: Render, n: int, outlier_frac: float,
                 rng: np.random.Generator, noise: float = 0.001):
    """Correspondences between frames i and j: (pts_i, pts_j, is_inlier).

    An inlier is a surface point seen (unoccluded, inside the mask) by both
    cameras, expressed in each camera frame plus N(0, noise) per axis.  An
    outlier replaces the frame-j point by the back-projection of a uniformly
    drawn masked pixel of frame j.
    """
    if n <= 0:
        e = np.zeros((0, 3), np.float32)
        return e, e.copy(), np.zeros(0, bool)
    cand = np.flatnonzero(r_i.mask.ravel())
    if cand.size == 0 or not r_j.mask.any():
        e = np.zeros((0, 3), np.float32)
        return e, e.copy(), np.zeros(0, bool)
    cand = rng.permutation(cand)
    Pc_i = backproject(r_i.depth_clean, cam_i).reshape(-1, 3)
    T_ji = T_j @ pose_inverse(T_i)
    got_i, got_j = [], []
    need = n
    for start in range(0, cand.size, 4 * n + 64):
        idx = cand[start:start + 4 * n + 64]
        Xi = Pc_i[idx]
        Xj = Xi @ T_ji[:3, :3].T + T_ji[:3, 3]
        z = Xj[:, 2]
        good = z > 1e-6
        zs = np.where(good, z, 1.0)
        uj = cam_j.fx * Xj[:, 0] / zs + cam_j.cx
        vj = cam_j.fy * Xj[:, 1] / zs + cam_j.cy
        iu = np.floor(uj + 0.5).astype(np.int64)
        iv = np.floor(vj + 0.5).astype(np.int64)
        good &= (iu >= 0) & (iu < cam_j.width) & (iv >= 0) & (iv < cam_j.height)
        iu_c = np.clip(iu, 0, cam_j.width - 1)
        iv_c = np.clip(iv, 0, cam_j.height - 1)
        good &= r_j.mask[iv_c, iu_c] > 0
        # visibility: the first hit along the ray through Xj is Xj itself
        dirs = Xj / zs[:, None]
        s, _ = cast_rays(shape, T_j, dirs)
        good &= np.abs(s - z) < 1e-6
        got_i.append(Xi[good])
        got_j.append(Xj[good])
        need -= int(good.sum())
        if need <= 0:
            break
    Xi = np.concatenate(got_i)[:n]
    Xj = np.concatenate(got_j)[:n]
    m = Xi.shape[0]
    pi = Xi + rng.normal(0.0, noise, Xi.shape)
    pj = Xj + rng.normal(0.0, noise, Xj.shape)
    inl = np.ones(m, bool)
    n_out = int(round(outlier_frac * m))
    if n_out > 0:
        which = rng.choice(m, n_out, replace=False)
        pix = rng.choice(np.flatnonzero(r_j.mask.ravel()), n_out)
        Pn_j = backproject(r_j.depth, cam_j).reshape(-1, 3)
        pj[which] = Pn_j[pix]
        inl[which] = False
    return pi.astype(np.float32), pj.astype(np.float32), inl


# --------------------------------------------------------------------------
# graphs
# --------------------------------------------------------------------------

def perturb_pose(T: np.ndarray, rot_deg: float, trans_m: float, rng: np.random.Generator) -> np.ndarray:
    """Rotate the object about its own origin by exactly rot_deg (random axis)
    and shift it by exactly trans_m (random direction), in the camera frame."""
    dR = axis_angle_matrix(random_unit(rng), np.deg2rad(rot_deg))
    return make_pose(dR @ T[:3, :3], T[:3, 3] + trans_m * random_unit(rng))


def step_pose(T: np.ndarray, t_home: np.ndarray, rng: np.random.Generator,
              max_deg: float = 10.0, max_trans: float = 0.02, radius: float = 0.03) -> np.ndarray:
    """One trajectory step: rotation U[0, max_deg] about a random axis through
    the object origin, translation U[0, max_trans] in a random direction,
    reversed when it would leave a ball of `radius` around t_home."""
    dR = axis_angle_matrix(random_unit(rng), np.deg2rad(rng.uniform(0.0, max_deg)))
    dt = rng.uniform(0.0, max_trans) * random_unit(rng)
    t = T[:3, 3] + dt
    if np.linalg.norm(t - t_home) > radius:
        t = T[:3, 3] - dt
    return make_pose(dR @ T[:3, :3], t)


@dataclass
class SynthGraph:
    cams: list
    renders: list
    pose_true: np.ndarray          # (N,4,4)
    pose_init: np.ndarray          # (N,4,4)
    fixed: np.ndarray              # (N,) int32
    matches: list                  # [(i, j, pts_i f32 (n,3), pts_j f32 (n,3))], i < j
    shape: Shape | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.renders)

    def depth(self, i):
        return self.renders[i].depth

    def normals(self, i):
        return self.renders[i].normals

    def mask(self, i):
        return self.renders[i].mask


def _rng(*seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(seed))))


def random_graph(seed: int, n_frames: int, cam: Camera, n_matches: int, outlier_frac: float,
                 dist_range=(0.35, 0.6), coverage_target: float | None = None,
                 init_rot_deg: float = 5.0, init_trans_m: float = 0.01,
                 depth_sigma: float = 0.001, with_ellipsoid: bool = True,
                 analytic_normals: bool = False, perturb: bool = True) -> SynthGraph:
    """A fully connected graph of n_frames views of one random object.
    Frame 0 is the fixed reference (gauge) and keeps its true pose."""
    rng = _rng(seed)
    shape = Shape.random(rng, with_ellipsoid)
    R0 = random_rotation(rng)
    if coverage_target is not None:
        d = distance_for_coverage(shape, cam, R0, coverage_target)
    else:
        d = rng.uniform(*dist_range)
    t0 = np.array([0.0, 0.0, d])
    poses = [make_pose(R0, t0)]
    for _ in range(1, n_frames):
        poses.append(step_pose(poses[-1], t0, rng))
    pose_true = np.stack(poses)
    renders = [render(shape, cam, pose_true[k], _rng(seed, 1, k), depth_sigma,
                      analytic_normals=analytic_normals) for k in range(n_frames)]
    matches = []
    for i in range(n_frames):
        for j in range(i + 1, n_frames):
            pi, pj, _ = make_matches(shape, cam, cam, pose_true[i], pose_true[j],
                                     renders[i], renders[j], n_matches, outlier_frac,
                                     _rng(seed, 2, i, j), noise=depth_sigma)
            matches.append((i, j, pi, pj))
    prng = _rng(seed, 3)
    pose_init = pose_true.copy()
    if perturb:
        for k in range(1, n_frames):
            pose_init[k] = perturb_pose(pose_true[k], init_rot_deg, init_trans_m, prng)
    fixed = np.zeros(n_frames, np.int32)
    fixed[0] = 1
    return SynthGraph([cam] * n_frames, renders, pose_true, pose_init, fixed, matches, shape,
                      dict(seed=seed))


def tiny_graph(graph_id: int = 0, **kw) -> SynthGraph:
    """Tiny workload: N=4 views at 160x120 (fx=fy=140), 200 matches per edge
    with 20% outliers, depth noise 1 mm, init perturbed by 5 deg / 1 cm."""
    args = dict(n_frames=4, cam=TINY_CAMERA, n_matches=200, outlier_frac=0.2)
    args.update(kw)
    return random_graph(1000 + graph_id, **args)


def paper_graph(graph_id: int = 0, n_frames: int = 10, **kw) -> SynthGraph:
    """Paper-shaped single graph: N=10 views at 640x480 (fx=fy=600), mask
    coverage U[15,30]% at the first view, 500 matches with 20% outliers."""
    rng = _rng(2000, 99, graph_id)
    args = dict(n_frames=n_frames, cam=VGA_CAMERA, n_matches=500, outlier_frac=0.2,
                coverage_target=float(rng.uniform(0.15, 0.30)))
    args.update(kw)
    return random_graph(2000 + graph_id, **args)


def batched_graph(graph_id: int, strip: bool = True) -> SynthGraph:
    """One graph of the batched workload (seed 4000 + graph_id): N uniform in
    3..20 views, all 320x240 (fx=fy=300) or all 640x480 (fx=fy=600) with equal
    probability, mask coverage U[5, 40] % at the first view, U{100..800}
    correspondences per pair with U[10, 30] % outliers, init 5 deg / 1 cm.
    strip drops the renderer-only arrays (clean depth, analytic normals)."""
    rng = _rng(4000, 99, graph_id)
    n = int(rng.integers(3, 21))
    cam = VGA_CAMERA if rng.random() < 0.5 else QVGA_CAMERA
    cov = float(rng.uniform(0.05, 0.40))
    n_m = int(rng.integers(100, 801))
    outl = float(rng.uniform(0.10, 0.30))
    g = random_graph(4000 + graph_id, n, cam, n_m, outl, coverage_target=cov)
    if strip:
        for r in g.renders:
            r.depth_clean = None
            r.normals_true = None
    g.meta.update(n_frames=n, width=cam.width, coverage=cov, matches=n_m, outliers=outl)
    return g


def _batched_job(k):
    return batched_graph(k)


def batched_graphs(ids, workers: int | None = None) -> list:
    """Graphs of the batched workload, made in forked worker processes (call
    before the calling process initialises CUDA)."""
    import multiprocessing as mp
    import os
    import sys
    from concurrent.futures import ProcessPoolExecutor
    torch = sys.modules.get("torch")
    if torch is not None and torch.cuda.is_initialized():
        raise RuntimeError("batched_graphs forks worker processes; call it before CUDA is initialised")
    ids = list(ids)
    workers = workers or max(1, min(32, os.cpu_count() or 1))
    if workers == 1 or len(ids) == 1:
        return [batched_graph(k) for k in ids]
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("fork")) as ex:
        return list(ex.map(_batched_job, ids))
