"""Index-level and element-wise parity of one Gauss-Newton iteration (Eq. 3,
Sec. IV-D) between the GPU kernels and the FP64 oracle.

Association (integers).  bt_debug_associate exports, for every valid source
pixel of an ordered pair, the target pixel the residual kernel associates it
with (or -1).  The oracle classifies the same pixel in FP64: the outcome it
computes in single precision from the definition, and the other outcomes
that single-precision rounding admits (a neighbouring pixel within rounding
of a half-pixel edge, dropped within rounding of a gate or the image edge).
Every GPU decision must be admitted; decisions left open must stay rare.

Normal equations (frozen association).  bt_debug_normal_equations exports
H and g as the solve assembles them: right perturbations of the free nodes,
T <- T exp(d).  The oracle evaluates its left-perturbation system on the
GPU's association (orc_normal_equations_frozen) and it is brought to the
same coordinates by d_left = Ad_T d_right:  H_r = A^T H_l A,  g_r = A^T g_l
with A = blockdiag(Ad_{T_i}) over the free nodes.  Tolerances:
  H    : |dH|_F <= 1e-6 |H|_F, and every entry |dH_ab| <= 4e-6 sqrt(H_aa H_bb)
         (|H_ab| <= sqrt(H_aa H_bb); each FP32 term carries ~5 roundings and
         a lane sums up to 16 of them before the warp reduction, ~25 roundings
         of 2^-24 in all: 1.5e-6, doubled)
  g_a  : sqrt(H_aa) (1e-6 sqrt(2E) + EPS_R sqrt(n))
         where |g_a| <= sqrt(H_aa) sqrt(2E) (Cauchy-Schwarz, Huber weights)
         and EPS_R bounds the FP32 rounding of one residual at ~1 m
         (the transform rounded to single, a few operations: 2^-24 x 1 m x a
         few), n the number of terms; g vanishes at the optimum, so its
         error floor is that of the residuals, not relative to g
  E    : 1e-6 E + EPS_R sqrt(2 E n)
  count: exact (the same association on both sides).
"""
import numpy as np
import pytest

import oracle as O
import synthgen as S

pytestmark = pytest.mark.gpu

EPS_R = 2e-7
H_RTOL_NORM = 1e-6
H_RTOL_ENTRY = 4e-6
AMBIGUOUS_MAX = 5e-3


@pytest.fixture(scope="module")
def bt():
    import torch
    from paper_2108_00516_gb300 import build as lbuild
    lbuild.build()
    from paper_2108_00516_gb300 import bt as _bt
    _bt.load()
    torch.cuda.init()
    return _bt


@pytest.fixture(scope="module")
def paper():
    return S.paper_graph(0)


def _skew(x):
    return np.array([[0, -x[2], x[1]], [x[2], 0, -x[0]], [-x[1], x[0], 0]])


def adjoint(T):
    """Ad_T for d = (v, w): exp(Ad_T d) T = T exp(d)."""
    R, t = T[:3, :3], T[:3, 3]
    A = np.zeros((6, 6))
    A[:3, :3] = R
    A[:3, 3:] = _skew(t) @ R
    A[3:, 3:] = R
    return A


def gpu_association(pg, g):
    """{(i, j): (source pixels, target pixels)} of the GPU for every ordered
    pair, and the raw per-source-pixel outcomes."""
    N = len(g.renders)
    assoc, raw = {}, {}
    for i in range(N):
        src = np.flatnonzero(((g.mask(i) > 0) & (g.depth(i) > 0) & np.isfinite(g.depth(i)) &
                              np.isfinite(g.normals(i)).all(-1)).ravel())
        for j in range(N):
            if i == j:
                continue
            out = pg.debug_associate(i, j)
            assert len(out) == len(src)
            raw[(i, j)] = out
            acc = out >= 0
            assoc[(i, j)] = (src[acc].astype(np.int32), out[acc].astype(np.int32))
    return assoc, raw


def check_association(g, P, raw):
    """Every GPU decision admitted by the oracle's classification; returns
    (decisions, ambiguous, GPU decisions that differ from the oracle's)."""
    total = amb = diff = 0
    for (i, j), out in raw.items():
        c = O.associate_classified(g, i, j, P)
        assert len(c.src) == len(out)
        ok = c.admits(out)
        assert ok.all(), ((i, j), int((~ok).sum()), c.src[~ok][:8], out[~ok][:8], c.nominal[~ok][:8],
                          c.alt[~ok][:8])
        total += len(out)
        amb += int(c.ambiguous.sum())
        diff += int((out != c.nominal).sum())
    return total, amb, diff


CASES = [("tiny", 0, "init"), ("tiny", 1, "true"), ("tiny", 2, "init"), ("paper", 0, "init"),
         ("paper", 0, "solved")]


def _graph(kind, gid, paper):
    return paper if kind == "paper" else S.tiny_graph(gid)


@pytest.mark.parametrize("kind,gid,where", CASES)
def test_association_index_parity(bt, paper, kind, gid, where):
    """Pixel by pixel: every GPU association decision is the oracle's or one
    that single-precision rounding admits; open decisions are rare."""
    g = _graph(kind, gid, paper)
    pg = bt.graph_from_synth(g)
    if where == "true":
        pg.set_poses(g.pose_true)
    elif where == "solved":
        pg.solve(3)
    P = pg.get_poses()
    _, raw = gpu_association(pg, g)
    total, amb, diff = check_association(g, P, raw)
    print(f"\n{kind}-{gid} {where}: {total} decisions, {amb} open ({amb / total:.2e}), {diff} differ")
    assert total > 1000
    assert amb <= AMBIGUOUS_MAX * total
    assert diff <= amb


@pytest.mark.parametrize("kind,gid,where", CASES)
def test_normal_equations_frozen_association(bt, paper, kind, gid, where):
    """H, g and E of one iteration element by element against the oracle
    evaluated on the GPU's association (right-perturbation coordinates)."""
    g = _graph(kind, gid, paper)
    pg = bt.graph_from_synth(g)
    if where == "true":
        pg.set_poses(g.pose_true)
    elif where == "solved":
        pg.solve(3)
    P = pg.get_poses()
    Hg, gg, cg = pg.debug_normal_equations()
    assoc, _ = gpu_association(pg, g)
    Hl, gl, El, cnt = O.normal_equations_frozen(g, P, assoc)
    assert cg["dense_inliers"] == cnt
    free = [k for k in range(len(g.renders)) if not g.fixed[k]]
    idx = np.concatenate([np.arange(6 * k, 6 * k + 6) for k in free])
    A = np.zeros((len(idx), len(idx)))
    for a, k in enumerate(free):
        A[6 * a:6 * a + 6, 6 * a:6 * a + 6] = adjoint(P[k])
    Hr = A.T @ Hl[np.ix_(idx, idx)] @ A
    gr = A.T @ gl[idx]
    assert Hg.shape == Hr.shape
    d = np.sqrt(np.diag(Hr))
    n_terms = cnt + sum(len(m[2]) for m in g.matches)
    errH = np.abs(Hg - Hr) / np.outer(d, d)
    tol_g = d * (1e-6 * np.sqrt(2 * El) + EPS_R * np.sqrt(n_terms))
    errg = np.abs(gg - gr) / tol_g
    print(f"\n{kind}-{gid} {where}: |dH|/|H| {np.linalg.norm(Hg - Hr) / np.linalg.norm(Hr):.2e}, "
          f"max |dH|/sqrt(HaaHbb) {errH.max():.2e}, max |dg|/tol {errg.max():.2e}, "
          f"|g| / (sqrt(Haa) sqrt(2E)) max {np.max(np.abs(gr) / (d * np.sqrt(2 * El))):.2e}, "
          f"E {cg['total']:.9g} vs {El:.9g}")
    assert np.linalg.norm(Hg - Hr) <= H_RTOL_NORM * np.linalg.norm(Hr)
    assert errH.max() <= H_RTOL_ENTRY, errH.max()
    assert errg.max() <= 1.0, errg.max()
    assert abs(cg["total"] - El) <= 1e-6 * El + EPS_R * np.sqrt(2 * El * n_terms)
    # the same E as the solve reports through bt_eval_cost
    assert abs(pg.eval_cost()["total"] - cg["total"]) <= 1e-6 * cg["total"]


def test_debug_calls_reject_bad_arguments(bt):
    g = S.tiny_graph(0)
    pg = bt.graph_from_synth(g)
    for (i, j) in [(0, 0), (-1, 1), (0, 4)]:
        with pytest.raises(bt.BTError):
            pg.debug_associate(i, j)
    pg.set_active([pg.frame_ids[0]])       # only the fixed node: no unknowns
    with pytest.raises(bt.BTError):
        pg.debug_normal_equations()
