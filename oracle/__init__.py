"""ctypes front-end of the FP64 CPU oracle (oracle/bt_oracle.c).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product path (the
CUDA library and its binding) never touches it.

A "graph" here is anything with the attributes ``renders`` (objects with
``depth`` float32 HxW, ``normals`` float32 HxWx3, ``mask`` uint8 HxW),
``cams`` (objects with ``fx, fy, cx, cy, width, height``), ``matches``
(list of ``(i, j, pts_i, pts_j)``), ``pose_init`` (N,4,4) and ``fixed`` (N,).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class _Frame(C.Structure):
    _fields_ = [("depth", C.POINTER(C.c_float)), ("normals", C.POINTER(C.c_float)),
                ("mask", C.POINTER(C.c_uint8)), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class _MatchSet(C.Structure):
    _fields_ = [("i", C.c_int32), ("j", C.c_int32), ("count", C.c_int32),
                ("pts_i", C.POINTER(C.c_float)), ("pts_j", C.POINTER(C.c_float))]


class _Params(C.Structure):
    _fields_ = [("huber_sparse", C.c_double), ("huber_dense", C.c_double),
                ("dense_max_dist", C.c_double), ("dense_max_normal_deg", C.c_double),
                ("lambda_sparse", C.c_double), ("lambda_dense", C.c_double),
                ("solver", C.c_int32), ("pcg_max_iters", C.c_int32), ("pcg_tol", C.c_double)]


@dataclass
class Params:
    """Method constants.  Defaults: Huber thresholds 5 mm and normal gate
    45 deg (the paper's only distance and angle constants, Sec. IV-B),
    distance gate 2 cm, lambda_1 = lambda_2 = 1 (Sec. IV-D)."""
    huber_sparse: float = 0.005
    huber_dense: float = 0.005
    dense_max_dist: float = 0.02
    dense_max_normal_deg: float = 45.0
    lambda_sparse: float = 1.0
    lambda_dense: float = 1.0
    solver: int = 0               # 0: Cholesky, 1: PCG with Jacobi preconditioner (Sec. IV-D)
    pcg_max_iters: int = 500
    pcg_tol: float = 1e-10

    def c(self) -> _Params:
        return _Params(self.huber_sparse, self.huber_dense, self.dense_max_dist,
                       self.dense_max_normal_deg, self.lambda_sparse, self.lambda_dense,
                       self.solver, self.pcg_max_iters, self.pcg_tol)


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(str(path))
        L.orc_huber_rho.restype = C.c_double
        L.orc_huber_rho.argtypes = [C.c_double, C.c_double]
        L.orc_huber_weight.restype = C.c_double
        L.orc_huber_weight.argtypes = [C.c_double, C.c_double]
        L.orc_se3_exp.argtypes = [_dp, _dp]
        L.orc_se3_log.argtypes = [_dp, _dp]
        L.orc_cholesky_solve.restype = C.c_int
        L.orc_cholesky_solve.argtypes = [C.c_int, _dp, _dp]
        L.orc_pcg_solve.restype = C.c_int
        L.orc_pcg_solve.argtypes = [C.c_int, _dp, _dp, C.c_int, C.c_double, C.POINTER(C.c_int)]
        L.orc_associate.restype = C.c_int
        L.orc_associate.argtypes = [C.POINTER(_Frame), C.POINTER(_Frame), _dp, _dp,
                                    C.POINTER(_Params), _ip, _ip, C.c_int]
        L.orc_associate_classify.restype = C.c_int
        L.orc_associate_classify.argtypes = [C.POINTER(_Frame), C.POINTER(_Frame), _dp, _dp,
                                             C.POINTER(_Params), _ip, _ip, _ip, _dp, C.c_int]
        L.orc_normal_equations_frozen.restype = C.c_long
        L.orc_normal_equations_frozen.argtypes = [C.POINTER(_Frame), C.c_int, _dp, C.POINTER(_MatchSet),
                                                  C.c_int, C.POINTER(_Params), C.POINTER(_ip),
                                                  C.POINTER(_ip), _ip, C.c_int, _dp, _dp, _dp]
        L.orc_dense_terms.argtypes = [C.POINTER(_Frame), C.POINTER(_Frame), _dp, _dp, _ip, _ip,
                                      C.c_int, _dp, _dp]
        L.orc_sparse_terms.argtypes = [C.POINTER(_MatchSet), _dp, _dp, _dp, _dp]
        L.orc_energy.argtypes = [C.POINTER(_Frame), C.c_int, _dp, C.POINTER(_MatchSet), C.c_int,
                                 C.POINTER(_Params), C.c_int, _dp]
        L.orc_normal_equations.restype = C.c_long
        L.orc_normal_equations.argtypes = [C.POINTER(_Frame), C.c_int, _dp, C.POINTER(_MatchSet),
                                           C.c_int, C.POINTER(_Params), C.c_int, _dp, _dp, _dp]
        L.orc_solve.restype = C.c_int
        L.orc_solve.argtypes = [C.POINTER(_Frame), C.c_int, _dp, _ip, C.POINTER(_MatchSet), C.c_int,
                                C.POINTER(_Params), C.c_int, C.c_int, _dp, _dp]
        _LIB = L
    return _LIB


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class Problem:
    """Marshals a graph into the oracle's C structures (kept alive here)."""

    def __init__(self, graph, nodes=None):
        nodes = list(range(len(graph.renders))) if nodes is None else list(nodes)
        pos = {f: k for k, f in enumerate(nodes)}
        self.keep = []
        self.frames = (_Frame * max(1, len(nodes)))()
        for k, f in enumerate(nodes):
            r, cam = graph.renders[f], graph.cams[f]
            d = np.ascontiguousarray(r.depth, np.float32)
            n = np.ascontiguousarray(r.normals, np.float32)
            m = np.ascontiguousarray(r.mask, np.uint8)
            self.keep += [d, n, m]
            self.frames[k] = _Frame(_ptr(d, C.c_float), _ptr(n, C.c_float), _ptr(m, C.c_uint8),
                                    cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        sets = []
        for (i, j, pi, pj) in graph.matches:
            if i in pos and j in pos and len(pi) > 0:
                a = np.ascontiguousarray(pi, np.float32)
                b = np.ascontiguousarray(pj, np.float32)
                self.keep += [a, b]
                sets.append(_MatchSet(pos[i], pos[j], len(a), _ptr(a, C.c_float), _ptr(b, C.c_float)))
        self.n_sets = len(sets)
        self.sets = (_MatchSet * max(1, len(sets)))(*sets)
        self.n = len(nodes)
        self.nodes = nodes
        self.fixed = np.ascontiguousarray(np.asarray(graph.fixed)[nodes], np.int32)
        self.pose_init = np.ascontiguousarray(np.asarray(graph.pose_init)[nodes], np.float64)


def solve(graph, iters: int, params: Params | None = None, poses=None, n_threads: int | None = None,
          nodes=None):
    """Run the FP64 Gauss-Newton solve.  Returns dict(poses, cost_per_iter,
    cost_final, status)."""
    P = Problem(graph, nodes)
    prm = (params or Params()).c()
    X = np.ascontiguousarray(P.pose_init if poses is None else poses, np.float64).copy()
    cpi = np.zeros(max(1, iters))
    cf = np.zeros(1)
    st = lib().orc_solve(P.frames, P.n, _ptr(X, C.c_double), _ptr(P.fixed, C.c_int32), P.sets, P.n_sets,
                         C.byref(prm), iters, n_threads or default_threads(),
                         _ptr(cpi, C.c_double), _ptr(cf, C.c_double))
    return dict(poses=X, cost_per_iter=cpi[:iters], cost_final=float(cf[0]), status=int(st))


def energy(graph, poses, params: Params | None = None, n_threads: int | None = None, nodes=None):
    """Eq. 1 at `poses`: dict(total, dense, sparse, dense_count, sparse_count)."""
    P = Problem(graph, nodes)
    prm = (params or Params()).c()
    X = np.ascontiguousarray(poses, np.float64)
    out = np.zeros(5)
    lib().orc_energy(P.frames, P.n, _ptr(X, C.c_double), P.sets, P.n_sets, C.byref(prm),
                     n_threads or default_threads(), _ptr(out, C.c_double))
    return dict(total=out[0], dense=out[1], sparse=out[2], dense_count=int(out[3]),
                sparse_count=int(out[4]))


def normal_equations(graph, poses, params: Params | None = None, n_threads: int | None = None,
                     nodes=None):
    """Full 6N x 6N H, 6N g and the energy at `poses` (no gauge applied)."""
    P = Problem(graph, nodes)
    prm = (params or Params()).c()
    X = np.ascontiguousarray(poses, np.float64)
    H = np.zeros((6 * P.n, 6 * P.n))
    g = np.zeros(6 * P.n)
    E = np.zeros(1)
    cnt = lib().orc_normal_equations(P.frames, P.n, _ptr(X, C.c_double), P.sets, P.n_sets,
                                     C.byref(prm), n_threads or default_threads(),
                                     _ptr(H, C.c_double), _ptr(g, C.c_double), _ptr(E, C.c_double))
    return H, g, float(E[0]), int(cnt)


def associate(graph, i: int, j: int, poses, params: Params | None = None):
    """Accepted (source pixel, target pixel) pairs of the ordered pair i -> j."""
    P = Problem(graph)
    prm = (params or Params()).c()
    X = np.ascontiguousarray(poses, np.float64)
    cap = graph.cams[i].width * graph.cams[i].height
    sp = np.zeros(cap, np.int32)
    tp = np.zeros(cap, np.int32)
    n = lib().orc_associate(C.byref(P.frames[i]), C.byref(P.frames[j]), _ptr(X[i], C.c_double),
                            _ptr(X[j], C.c_double), C.byref(prm), _ptr(sp, C.c_int32),
                            _ptr(tp, C.c_int32), cap)
    return sp[:n].copy(), tp[:n].copy()


@dataclass
class Classified:
    """Association decisions of one ordered pair, one entry per valid masked
    source pixel (increasing pixel order): ``src`` the pixel, ``nominal`` the
    oracle's single-precision decision (target pixel or -1), ``alt`` (n, 4)
    the other outcomes single-precision rounding admits (-1 = dropped, -2 =
    none), ``slack`` the largest change of that pixel's Huber cost (Eq. 3,
    before lambda_2) over them."""
    src: np.ndarray
    nominal: np.ndarray
    alt: np.ndarray
    slack: np.ndarray

    @property
    def ambiguous(self) -> np.ndarray:
        return (self.alt != -2).any(axis=1)

    def admits(self, outcome: np.ndarray) -> np.ndarray:
        """Per entry: is `outcome` (target pixel or -1) the nominal decision
        or one of the admissible alternatives?"""
        outcome = np.asarray(outcome)
        return (outcome == self.nominal) | (self.alt == outcome[:, None]).any(axis=1)

    def count_range(self):
        """(fewest, most) accepted associations over the admissible outcomes."""
        acc_nom = self.nominal >= 0
        acc_alt = (self.alt >= 0).any(axis=1)
        rej_alt = (self.alt == -1).any(axis=1)
        lo = int(np.sum(acc_nom & ~rej_alt))
        hi = int(np.sum(acc_nom | acc_alt))
        return lo, hi


def associate_classified(graph, i: int, j: int, poses, params: Params | None = None) -> Classified:
    """Every association decision of the ordered pair i -> j with the outcomes
    that single-precision rounding admits (FP64 classification)."""
    P = Problem(graph)
    prm = (params or Params()).c()
    X = np.ascontiguousarray(poses, np.float64)
    cap = graph.cams[i].width * graph.cams[i].height
    sp = np.zeros(cap, np.int32)
    nom = np.zeros(cap, np.int32)
    alt = np.zeros((cap, 4), np.int32)
    sl = np.zeros(cap)
    n = lib().orc_associate_classify(C.byref(P.frames[i]), C.byref(P.frames[j]), _ptr(X[i], C.c_double),
                                     _ptr(X[j], C.c_double), C.byref(prm), _ptr(sp, C.c_int32),
                                     _ptr(nom, C.c_int32), _ptr(alt, C.c_int32), _ptr(sl, C.c_double), cap)
    return Classified(sp[:n].copy(), nom[:n].copy(), alt[:n].copy(), sl[:n].copy())


def energy_bounds(graph, poses, params: Params | None = None, nodes=None):
    """Over every ordered pair of the graph (or of `nodes`): the fewest and
    most dense associations single-precision rounding admits, the largest
    change of the dense energy (lambda_2 included) that the admissible
    alternatives can make, and the number of ambiguous pixels."""
    prm = params or Params()
    nodes = list(range(len(graph.renders))) if nodes is None else list(nodes)
    lo = hi = 0
    slack = 0.0
    amb = 0
    total = 0
    for a in nodes:
        for b in nodes:
            if a == b:
                continue
            c = associate_classified(graph, a, b, poses if len(poses) == len(graph.renders)
                                     else _expand(poses, nodes, len(graph.renders)), prm)
            l, h = c.count_range()
            lo += l
            hi += h
            slack += prm.lambda_dense * float(np.sum(c.slack))
            amb += int(c.ambiguous.sum())
            total += len(c.src)
    return dict(count_lo=lo, count_hi=hi, slack=slack, ambiguous=amb, pixels=total)


def _expand(poses, nodes, n_all):
    X = np.tile(np.eye(4), (n_all, 1, 1))
    for k, f in enumerate(nodes):
        X[f] = poses[k]
    return X


def normal_equations_frozen(graph, poses, assoc, params: Params | None = None, n_threads: int | None = None):
    """orc_normal_equations with the association given instead of computed:
    assoc[(i, j)] = (source pixels, target pixels) of every ordered pair.
    Returns the full 6N x 6N H, 6N g, the energy and the dense term count."""
    P = Problem(graph)
    prm = (params or Params()).c()
    N = P.n
    X = np.ascontiguousarray(poses, np.float64)
    keep = []
    srcs = (_ip * max(1, N * (N - 1)))()
    tgts = (_ip * max(1, N * (N - 1)))()
    cnt = np.zeros(max(1, N * (N - 1)), np.int32)
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            k = i * (N - 1) + (j if j < i else j - 1)
            s, t = assoc[(i, j)]
            s = np.ascontiguousarray(s, np.int32)
            t = np.ascontiguousarray(t, np.int32)
            if len(s) != len(t):
                raise ValueError("source and target lists differ in length")
            keep += [s, t]
            srcs[k] = _ptr(s, C.c_int32)
            tgts[k] = _ptr(t, C.c_int32)
            cnt[k] = len(s)
    H = np.zeros((6 * N, 6 * N))
    g = np.zeros(6 * N)
    E = np.zeros(1)
    n = lib().orc_normal_equations_frozen(P.frames, N, _ptr(X, C.c_double), P.sets, P.n_sets, C.byref(prm),
                                          srcs, tgts, _ptr(cnt, C.c_int32), n_threads or default_threads(),
                                          _ptr(H, C.c_double), _ptr(g, C.c_double), _ptr(E, C.c_double))
    if n < 0:
        raise ValueError("association holds a pixel index out of range")
    return H, g, float(E[0]), int(n)


def dense_terms(graph, i: int, j: int, poses, src, tgt):
    """Residuals (n,) and 12-column Jacobians (n,12) for a frozen association."""
    P = Problem(graph)
    X = np.ascontiguousarray(poses, np.float64)
    src = np.ascontiguousarray(src, np.int32)
    tgt = np.ascontiguousarray(tgt, np.int32)
    n = len(src)
    r = np.zeros(max(1, n))
    J = np.zeros((max(1, n), 12))
    lib().orc_dense_terms(C.byref(P.frames[i]), C.byref(P.frames[j]), _ptr(X[i], C.c_double),
                          _ptr(X[j], C.c_double), _ptr(src, C.c_int32), _ptr(tgt, C.c_int32), n,
                          _ptr(r, C.c_double), _ptr(J, C.c_double))
    return r[:n].copy(), J[:n].copy()


def sparse_terms(pts_i, pts_j, Ti, Tj):
    """Residuals e (n,3) and Jacobians (n,3,12) of one correspondence set."""
    a = np.ascontiguousarray(pts_i, np.float32)
    b = np.ascontiguousarray(pts_j, np.float32)
    n = len(a)
    ms = _MatchSet(0, 1, n, _ptr(a, C.c_float), _ptr(b, C.c_float))
    e = np.zeros((max(1, n), 3))
    J = np.zeros((max(1, n), 3, 12))
    Ti = np.ascontiguousarray(Ti, np.float64)
    Tj = np.ascontiguousarray(Tj, np.float64)
    lib().orc_sparse_terms(C.byref(ms), _ptr(Ti, C.c_double), _ptr(Tj, C.c_double),
                           _ptr(e, C.c_double), _ptr(J, C.c_double))
    return e[:n].copy(), J[:n].copy()


def se3_exp(xi) -> np.ndarray:
    xi = np.ascontiguousarray(xi, np.float64)
    T = np.zeros(16)
    lib().orc_se3_exp(_ptr(xi, C.c_double), _ptr(T, C.c_double))
    return T.reshape(4, 4)


def se3_log(T) -> np.ndarray:
    T = np.ascontiguousarray(T, np.float64).reshape(16)
    xi = np.zeros(6)
    lib().orc_se3_log(_ptr(T, C.c_double), _ptr(xi, C.c_double))
    return xi


def cholesky_solve(A, b):
    A = np.ascontiguousarray(A, np.float64).copy()
    b = np.ascontiguousarray(b, np.float64).copy()
    st = lib().orc_cholesky_solve(len(b), _ptr(A, C.c_double), _ptr(b, C.c_double))
    return b, st



def pcg_solve(A, b, max_iters: int = 500, tol: float = 1e-10):
    """x of A x = b by Jacobi-preconditioned conjugate gradients, and the
    iteration count (raises ValueError if A is not positive definite)."""
    A = np.ascontiguousarray(A, np.float64)
    x = np.ascontiguousarray(b, np.float64).copy()
    it = C.c_int()
    if lib().orc_pcg_solve(len(x), _ptr(A, C.c_double), _ptr(x, C.c_double), int(max_iters), float(tol),
                           C.byref(it)) != 0:
        raise ValueError("matrix not positive definite")
    return x, it.value

def huber_rho(r, delta):
    return lib().orc_huber_rho(float(r), float(delta))


def huber_weight(r, delta):
    return lib().orc_huber_weight(float(r), float(delta))
