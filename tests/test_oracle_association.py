"""Pins of the oracle's projective association (Eq. 3 and the gating sentence
after it, Sec. IV-D) and of its rounding classification.

The association keeps a source pixel x of frame i when its point, seen from
camera j, projects to a valid target pixel u' (nearest pixel) whose point
lies within d_max of it and whose normal is within theta_max of the source
normal.  The scenes below fix every one of these quantities in closed form:
camera j is camera i rolled by 90 degrees about the optical axis (so pixel
offsets rotate exactly and every projection lands on a pixel centre), target
depths are placed on the source pixel's ray at a chosen distance, and target
normals are the source normal turned by a chosen angle and then rolled with
the camera.  A distance gate compared against d_max^2 as if it were d_max,
an unrotated target normal, truncation instead of the nearest pixel or a
missed validity test each changes a decision below.
"""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle as O
import synthgen as S

PRM = O.Params()
DMAX = PRM.dense_max_dist
TMAX = PRM.dense_max_normal_deg

W, H, FX, CX, CY = 41, 31, 40.0, 20.0, 15.0
CAM = S.Camera(FX, FX, CX, CY, W, H)
Z = 0.5
ROLL = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])   # 90 deg about the optical axis


def _graph(depth_i, normals_i, mask_i, depth_j, normals_j, mask_j, t_j=(0.0, 0.0, 0.0)):
    """Two frames; T_0 = I, T_1 = [ROLL | t_j] (object -> camera)."""
    def rend(d, n, m):
        return SimpleNamespace(depth=np.ascontiguousarray(d, np.float32),
                               normals=np.ascontiguousarray(n, np.float32),
                               mask=np.ascontiguousarray(m, np.uint8))
    T1 = np.eye(4)
    T1[:3, :3] = ROLL
    T1[:3, 3] = t_j
    P = np.stack([np.eye(4), T1])
    return SimpleNamespace(renders=[rend(depth_i, normals_i, mask_i), rend(depth_j, normals_j, mask_j)],
                           cams=[CAM, CAM], matches=[], pose_init=P, fixed=np.array([1, 0], np.int32))


def _target_of(u, v):
    """Pixel of camera j that source pixel (u, v) projects to under the roll:
    (x, y) -> (-y, x) in camera coordinates, so (u - cx, v - cy) ->
    (-(v - cy), u - cx)."""
    return int(CX - (v - CY)), int(CY + (u - CX))


def _ray_norm(u, v):
    return np.sqrt(1.0 + ((u - CX) / FX) ** 2 + ((v - CY) / FX) ** 2)


def _turn(n, axis, deg):
    return S.axis_angle_matrix(np.asarray(axis, float), np.deg2rad(deg)) @ n


class _Scene:
    """Source frame: a fronto-parallel plane at Z with per-pixel normals;
    target frame: filled per case."""

    def __init__(self):
        self.di = np.full((H, W), Z, np.float32)
        self.ni = np.zeros((H, W, 3), np.float32)
        self.mi = np.zeros((H, W), np.uint8)
        self.dj = np.zeros((H, W), np.float32)
        self.nj = np.full((H, W, 3), np.nan, np.float32)
        self.mj = np.zeros((H, W), np.uint8)
        self.expect = {}     # source pixel index -> target pixel index or -1

    def case(self, u, v, dist, angle_deg, n_src=(1.0, 0.0, -1.0), keep=None, tgt_mask=1, tgt_depth_ok=True,
             tgt_normal_ok=True):
        n = np.asarray(n_src, float)
        n /= np.linalg.norm(n)
        self.mi[v, u] = 1
        self.ni[v, u] = n
        tu, tv = _target_of(u, v)
        # the target point on the source point's ray at `dist` beyond it
        self.dj[tv, tu] = (Z + dist / _ray_norm(u, v)) if tgt_depth_ok else 0.0
        axis = np.cross(n, [0.0, 1.0, 0.0]) if abs(n[1]) < 0.9 else np.cross(n, [1.0, 0.0, 0.0])
        nt = ROLL @ _turn(n, axis / np.linalg.norm(axis), angle_deg)
        self.nj[tv, tu] = nt if tgt_normal_ok else np.nan
        self.mj[tv, tu] = tgt_mask
        self.expect[v * W + u] = tv * W + tu if keep else -1

    def graph(self, t_j=(0.0, 0.0, 0.0)):
        return _graph(self.di, self.ni, self.mi, self.dj, self.nj, self.mj, t_j)


def _run(g):
    sp, tp = O.associate(g, 0, 1, g.pose_init, PRM)
    return dict(zip(sp.tolist(), tp.tolist()))


def test_distance_gate():
    """|T_i T_j^-1 t - p| <= d_max: kept at 0.999 d_max, dropped at 1.001 d_max,
    on rays of every direction in the image (the distance is measured along
    the ray, not in depth)."""
    s = _Scene()
    for k, (u, v) in enumerate([(20, 15), (8, 3), (33, 27), (12, 22), (30, 6)]):
        s.case(u, v, 0.999 * DMAX, 0.0, keep=True)
        s.case(u + 1, v, 1.001 * DMAX, 0.0, keep=False)
        s.case(u, v + 1, -0.999 * DMAX, 0.0, keep=True)     # target in front of the source point
        s.case(u + 1, v + 1, -1.001 * DMAX, 0.0, keep=False)
    kept = _run(s.graph())
    for sp, tp in s.expect.items():
        assert kept.get(sp, -1) == tp, (divmod(sp, W), tp)


def test_angle_gate():
    """The angle between n_i and the target normal brought into camera i is
    at most theta_max: kept at theta_max - 0.05 deg, dropped at +0.05 deg.  The
    roll moves the target normal by ~60 deg, so comparing it unrotated fails."""
    s = _Scene()
    cases = [((20, 15), (1.0, 0.0, -1.0)), ((9, 9), (0.2, 0.5, -1.0)), ((28, 20), (-0.7, 0.3, -1.0))]
    for (u, v), n in cases:
        s.case(u, v, 0.3 * DMAX, TMAX - 0.05, n_src=n, keep=True)
        s.case(u + 1, v, 0.3 * DMAX, TMAX + 0.05, n_src=n, keep=False)
        s.case(u, v + 1, 0.3 * DMAX, 1.0, n_src=n, keep=True)
        # the pin discriminates: unrotated, these normals are far from the rotated ones
        nn = np.asarray(n) / np.linalg.norm(n)
        assert np.degrees(np.arccos(np.clip(nn @ (ROLL @ nn), -1, 1))) > 20.0
    kept = _run(s.graph())
    for sp, tp in s.expect.items():
        assert kept.get(sp, -1) == tp, (divmod(sp, W), tp)


def test_target_validity_and_image_bounds():
    """The target pixel must be masked, have a depth and a normal; a
    projection outside the image is dropped (with W > H, source columns
    u < cx - cy or u > cx + cy land outside rows 0..H-1)."""
    s = _Scene()
    s.case(20, 10, 0.0, 0.0, keep=True)
    s.case(21, 10, 0.0, 0.0, keep=False, tgt_mask=0)
    s.case(22, 10, 0.0, 0.0, keep=False, tgt_depth_ok=False)
    s.case(23, 10, 0.0, 0.0, keep=False, tgt_normal_ok=False)
    for u in (0, 4, 36, 40):            # v' = u - 5 outside 0..30
        s.mi[12, u] = 1
        s.ni[12, u] = (0.0, 0.0, -1.0)
        s.expect[12 * W + u] = -1
    for u in (5, 35):                   # the first and last columns that land inside
        s.case(u, 12, 0.0, 0.0, keep=True)
    kept = _run(s.graph())
    for sp, tp in s.expect.items():
        assert kept.get(sp, -1) == tp, (divmod(sp, W), tp)
    # invalid source pixels are not sources at all
    s.di[3, 3] = 0.0
    s.mi[3, 3] = 1
    s.ni[3, 3] = (0.0, 0.0, -1.0)
    c = O.associate_classified(s.graph(), 0, 1, s.graph().pose_init, PRM)
    assert 3 * W + 3 not in set(c.src.tolist())


@pytest.mark.parametrize("shift,step", [(0.3, 0), (0.7, 1), (-0.3, 0), (-0.7, -1)])
def test_nearest_pixel(shift, step):
    """u' = floor(u + 1/2): a projection 0.3 px past a pixel centre stays on
    it, 0.7 px past moves to the next pixel (truncation would keep it)."""
    s = _Scene()
    u, v = 20, 15
    s.mi[v, u] = 1
    s.ni[v, u] = (0.0, 0.0, -1.0)
    # camera-j translation along x shifts the projection by FX * dx / Z pixels
    dx = shift * Z / FX
    tu, tv = _target_of(u, v)
    for du in (-1, 0, 1):
        s.dj[tv, tu + du] = Z
        s.nj[tv, tu + du] = (0.0, 0.0, -1.0)
        s.mj[tv, tu + du] = 1
    kept = _run(s.graph(t_j=(dx, 0.0, 0.0)))
    assert kept[v * W + u] == tv * W + tu + step


# ---------------------------------------------------------------------------
# classification of decisions against single-precision rounding
# ---------------------------------------------------------------------------

def _decide(g, i, j, P, src, dtype, order):
    """Association decisions of the given source pixels, written out again
    with numpy: dtype float64 (the exact result up to FP64 rounding), or
    float32 with the operations in another order than the oracle's (the
    source normal rotated into camera j instead of the target normal into
    camera i, a reciprocal multiplied instead of a divide, sums
    reassociated)."""
    f = np.dtype(dtype).type
    ci, cj = g.cams[i], g.cams[j]
    B = P[j] @ np.linalg.inv(P[i])
    Bf = B[:3].astype(dtype)
    v, u = np.divmod(src, ci.width)
    z = g.renders[i].depth.ravel()[src].astype(dtype)
    if order == "alt":
        p = np.stack([(u - f(ci.cx)).astype(dtype) * (z * (f(1) / f(ci.fx))),
                      (v - f(ci.cy)).astype(dtype) * (z * (f(1) / f(ci.fy))), z], -1)
        q = np.stack([((Bf[r, 2] * p[:, 2] + Bf[r, 3]) + Bf[r, 1] * p[:, 1]) + Bf[r, 0] * p[:, 0]
                      for r in range(3)], -1)
        rz = f(1) / q[:, 2]
        uh = (f(cj.fx) * q[:, 0]) * rz + (f(cj.cx) + f(0.5))
        vh = (f(cj.fy) * q[:, 1]) * rz + (f(cj.cy) + f(0.5))
    else:
        p = np.stack([(u - f(ci.cx)) * z / f(ci.fx), (v - f(ci.cy)) * z / f(ci.fy), z], -1).astype(dtype)
        q = p @ Bf[:, :3].T + Bf[:, 3]
        uh = f(cj.fx) * q[:, 0] / q[:, 2] + f(cj.cx) + f(0.5)
        vh = f(cj.fy) * q[:, 1] / q[:, 2] + f(cj.cy) + f(0.5)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        fu, fv = np.floor(uh), np.floor(vh)
        ok = (q[:, 2] > 0) & (fu >= 0) & (fu < cj.width) & (fv >= 0) & (fv < cj.height)
    iu = np.where(ok, fu, 0).astype(np.int64)
    iv = np.where(ok, fv, 0).astype(np.int64)
    tp = iv * cj.width + iu
    rj = g.renders[j]
    zt = rj.depth.ravel()[tp].astype(dtype)
    nt = rj.normals.reshape(-1, 3)[tp].astype(dtype)
    ok &= (rj.mask.ravel()[tp] > 0) & (zt > 0) & np.isfinite(zt) & np.isfinite(nt).all(-1)
    t = np.stack([(iu - f(cj.cx)) * zt / f(cj.fx), (iv - f(cj.cy)) * zt / f(cj.fy), zt], -1).astype(dtype)
    d = t - q
    ns = g.renders[i].normals.reshape(-1, 3)[src].astype(dtype)
    with np.errstate(invalid="ignore", over="ignore"):
        if order == "alt":
            ok &= ((d[:, 2] * d[:, 2] + d[:, 1] * d[:, 1]) + d[:, 0] * d[:, 0]) <= f(DMAX * DMAX)
            m = ns @ Bf[:, :3].T                       # R_B n_i, in camera j
            cs = (m[:, 2] * nt[:, 2] + m[:, 1] * nt[:, 1]) + m[:, 0] * nt[:, 0]
        else:
            ok &= np.sqrt((d * d).sum(-1)) <= f(DMAX)
            cs = (ns * (nt @ Bf[:, :3])).sum(-1)       # n_i . R_B^T n_j
        ok &= cs >= f(np.cos(np.deg2rad(TMAX)))
    return np.where(ok, tp, -1)


@pytest.fixture(scope="module")
def tiny():
    return S.tiny_graph(3)


@pytest.fixture(scope="module")
def paper_pair():
    return S.paper_graph(0, n_frames=3)


def _check_admitted(g, i, j, P):
    c = O.associate_classified(g, i, j, P, PRM)
    assert np.all(np.isfinite(c.slack)), "single-precision decision outside the admissible set"
    for dtype, order in [(np.float64, "plain"), (np.float32, "alt"), (np.float32, "plain")]:
        dec = _decide(g, i, j, P, c.src, dtype, order)
        bad = ~c.admits(dec)
        assert not bad.any(), (dtype.__name__, order, int(bad.sum()), c.src[bad][:5])
    # the oracle's own list agrees with the classification's nominal decisions
    sp, tp = O.associate(g, i, j, P, PRM)
    acc = c.nominal >= 0
    assert np.array_equal(sp, c.src[acc]) and np.array_equal(tp, c.nominal[acc])
    return c


def test_classification_admits_exact_and_reordered(tiny, paper_pair):
    """The exact (FP64) decision and an independently ordered single-precision
    evaluation both fall inside the admissible set of every pixel, at the
    initial and at the true poses."""
    n_amb = n_all = 0
    for g in (tiny, paper_pair):
        for P in (g.pose_init, g.pose_true):
            for (i, j) in [(0, 1), (1, 0), (2, 1)]:
                c = _check_admitted(g, i, j, P)
                n_amb += int(c.ambiguous.sum())
                n_all += len(c.src)
    assert n_all > 100_000
    # the band is narrow: few decisions are left open
    assert n_amb < 5e-3 * n_all, (n_amb, n_all)


def test_classification_rejects_real_mistakes(paper_pair):
    """A neighbouring pixel, or a dropped pixel, where the decision is not
    near any boundary is not admitted."""
    g = paper_pair
    c = O.associate_classified(g, 0, 1, g.pose_init, PRM)
    clear = (~c.ambiguous) & (c.nominal >= 0)
    idx = np.flatnonzero(clear)[:: max(1, clear.sum() // 500)]
    assert len(idx) > 100
    for wrong in (c.nominal + 1, c.nominal + g.cams[1].width, np.full(len(c.src), -1)):
        assert not c.admits(wrong)[idx].any()


def test_classification_opens_gate_edges():
    """Decisions placed on a gate (distance d_max (1 +- 1e-9), angle
    theta_max +- 1e-7 deg) are ambiguous and admit both outcomes, with a slack
    equal to the Huber cost of the kept pixel; pixels well inside are
    not ambiguous."""
    s = _Scene()
    s.case(20, 15, DMAX * (1 - 1e-9), 0.0, keep=True)
    s.case(21, 15, DMAX * (1 + 1e-9), 0.0, keep=False)
    s.case(22, 15, 0.3 * DMAX, TMAX - 1e-7, keep=True)
    s.case(23, 15, 0.3 * DMAX, TMAX + 1e-7, keep=False)
    s.case(24, 15, 0.5 * DMAX, 10.0, keep=True)
    g = s.graph()
    c = O.associate_classified(g, 0, 1, g.pose_init, PRM)
    amb = dict(zip(c.src.tolist(), c.ambiguous.tolist()))
    for u in (20, 21, 22, 23):
        sp = 15 * W + u
        assert amb[sp], u
        k = int(np.flatnonzero(c.src == sp)[0])
        tu, tv = _target_of(u, 15)
        assert c.admits(np.where(c.src == sp, tv * W + tu, c.nominal))[k]
        assert c.admits(np.where(c.src == sp, -1, c.nominal))[k]
        assert c.slack[k] > 0
    assert not amb[15 * W + 24]
