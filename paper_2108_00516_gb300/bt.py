"""Python binding of libbt (include/bt.h): argument marshalling only.

Every step of the pose-graph solve runs in the library's CUDA kernels; this
module converts numpy arrays (host memory) or CUDA tensors (device memory) to
pointers, calls the C functions of the same name, and turns status codes into
exceptions.  Importing it loads the compiled library and fails loudly if it
has not been built or cannot be loaded; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

BT_OK = 0
BT_ERR_INVALID = -1
BT_ERR_CUDA = -2
BT_ERR_OOM = -3
BT_ERR_SINGULAR = -4
BT_ERR_TIMEOUT = -5
BT_ERR_STATE = -6
BT_HOST = 0
BT_DEVICE = 1
BT_FP32 = 0
BT_BF16 = 1
BT_FP16 = 2
BT_MAX_NODES = 24
BT_MAX_REPORT_ITERS = 64
BT_NUM_SHAPES = 6
BT_SINGLE_GRAPH_SHAPE = 2
BT_SOLVER_CHOLESKY = 0
BT_SOLVER_PCG = 1

LIB_PATH = Path(__file__).resolve().parent / "_build" / "libbt.so"


class bt_intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class bt_config(C.Structure):
    _fields_ = [("huber_sparse", C.c_double), ("huber_dense", C.c_double),
                ("dense_max_dist", C.c_double), ("dense_max_normal_deg", C.c_double),
                ("lambda_sparse", C.c_double), ("lambda_dense", C.c_double),
                ("precision", C.c_int32), ("max_frames", C.c_int32),
                ("solver", C.c_int32), ("pcg_max_iters", C.c_int32), ("pcg_tol", C.c_double)]


class bt_matches(C.Structure):
    _fields_ = [("other_frame", C.c_int32), ("count", C.c_int32),
                ("pts_self", C.c_void_p), ("pts_other", C.c_void_p)]


class bt_solve_report(C.Structure):
    _fields_ = [("iters_run", C.c_int32), ("status", C.c_int32), ("used_warmstart", C.c_int32),
                ("fell_back", C.c_int32), ("cost_init", C.c_double), ("cost_final", C.c_double),
                ("dense_cost_final", C.c_double), ("sparse_cost_final", C.c_double),
                ("cost_per_iter", C.c_double * BT_MAX_REPORT_ITERS), ("dense_inliers", C.c_int64),
                ("dense_pixel_pairs", C.c_int64)]


class bt_profile(C.Structure):
    _fields_ = [("prep_launches", C.c_int64), ("xform_launches", C.c_int64),
                ("residual_launches", C.c_int64), ("reduce_launches", C.c_int64),
                ("residual_ms", C.c_double), ("reduce_ms", C.c_double),
                ("timed_residual_launches", C.c_int64), ("timed_reduce_launches", C.c_int64),
                ("dense_pixel_pairs", C.c_int64), ("sparse_pairs", C.c_int64),
                ("solve_phase_cycles", C.c_int64 * 4)]


# name -> (restype, argtypes); every symbol include/bt.h declares
SIGNATURES = {
    "bt_config_default": (None, [C.POINTER(bt_config)]),
    "bt_graph_create": (C.c_int, [C.POINTER(bt_config), C.c_void_p, C.POINTER(C.c_void_p)]),
    "bt_graph_destroy": (None, [C.c_void_p]),
    "bt_add_frame": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(bt_intrinsics),
                               C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                               C.POINTER(C.c_int32)]),
    "bt_set_matches": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_int32]),
    "bt_remove_frame": (C.c_int, [C.c_void_p, C.c_int32]),
    # the per-solve calls take raw addresses (c_void_p also accepts ctypes
    # pointers): converting an array with data_as costs more than the call
    "bt_set_active": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "bt_num_active": (C.c_int, [C.c_void_p]),
    "bt_set_poses": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bt_get_poses": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "bt_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "bt_eval_cost": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "bt_batch_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "bt_batch_destroy": (None, [C.c_void_p]),
    "bt_batch_add": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bt_batch_size": (C.c_int, [C.c_void_p]),
    "bt_batch_set_shape": (C.c_int, [C.c_void_p, C.c_int32]),
    "bt_batch_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "bt_batch_solve": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(bt_solve_report)]),
    "bt_warmstart_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "bt_warmstart_destroy": (None, [C.c_void_p]),
    "bt_warmstart_num_params": (C.c_int32, []),
    "bt_warmstart_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "bt_warmstart_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "bt_warmstart_get_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_int32]),
    "bt_warmstart_set_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "bt_warmstart_add_set": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.c_int32]),
    "bt_warmstart_add_graph": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "bt_warmstart_num_samples": (C.c_int32, [C.c_void_p]),
    "bt_warmstart_clear_samples": (C.c_int, [C.c_void_p]),
    "bt_warmstart_get_sample": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "bt_warmstart_predict": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_float)]),
    "bt_warmstart_gradient": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_float),
                                        C.POINTER(C.c_double)]),
    "bt_warmstart_train_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_float,
                                          C.POINTER(C.c_double)]),
    "bt_warmstart_apply": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bt_warmstart_apply_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "bt_batch_solve_warm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                      C.c_double, C.POINTER(bt_solve_report)]),
    "bt_ransac": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_double,
                            C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_void_p]),
    "bt_ransac_init": (C.c_int, [C.c_void_p, C.c_int32, C.c_uint64, C.c_double, C.c_int32]),
    "bt_select_keyframes": (C.c_int32, [C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double), C.c_int32,
                                        C.POINTER(C.c_int32)]),
    "bt_is_novel_view": (C.c_int32, [C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double), C.c_double]),
    "bt_debug_associate": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.c_int32,
                                     C.POINTER(C.c_int32)]),
    "bt_debug_normal_equations": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32,
                                            C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "bt_debug_fail_allocations": (C.c_int32, [C.c_int32]),
    "bt_debug_tensor_wait_ns": (C.c_int64, [C.c_int64]),
    "bt_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "bt_profile_read": (C.c_int, [C.c_void_p, C.POINTER(bt_profile)]),
    "bt_device_cache_bytes": (C.c_int64, []),
    "bt_device_cache_trim": (C.c_int64, []),
    "bt_pair_dense_energy_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(bt_intrinsics),
                                               C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_void_p,
                                               C.POINTER(bt_intrinsics), C.POINTER(C.c_double),
                                               C.POINTER(bt_config), C.c_void_p, C.c_void_p]),
    "bt_noalloc_last_error": (C.c_char_p, []),
    "bt_status_str": (C.c_char_p, [C.c_int]),
    "bt_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: Path | str | None = None):
    """Load libbt.so (once): `path`, else $BT_LIB, else the in-tree build.
    Raises RuntimeError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    import os
    p = Path(path) if path else Path(os.environ.get("BT_LIB") or LIB_PATH)
    if not p.exists():
        raise RuntimeError(f"libbt.so not found at {p}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class BTError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = load()
        msg = L.bt_last_error().decode() or L.bt_status_str(status).decode()
        super().__init__(f"{where}: {L.bt_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def _check(st: int, where: str):
    if st != BT_OK:
        raise BTError(st, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _addr(a) -> int:
    """Address of the first element of a C-contiguous numpy array.  Through
    the buffer protocol when the array is writable (~0.35 us), else numpy's
    ctypes interface (~0.9 us): the per-frame calls pass up to ~20 arrays."""
    try:
        return C.addressof(C.c_char.from_buffer(a))
    except (TypeError, ValueError, BufferError):
        return a.ctypes.data


def _ptr(x, dtype, shape_check=None):
    """(pointer, keepalive, mem_kind) for a numpy array or a CUDA tensor."""
    if type(x) is np.ndarray and x.dtype == dtype and x.flags.c_contiguous:
        return _addr(x), x, BT_HOST
    if _is_torch(x):
        if not x.is_cuda:
            x = x.contiguous().numpy()
        else:
            x = x.contiguous()
            return C.c_void_p(x.data_ptr()), x, BT_DEVICE
    a = np.ascontiguousarray(x, dtype=dtype)
    return _addr(a), a, BT_HOST


# numpy image of bt_matches (int32, int32, void*, void*): a frame's
# correspondence sets are passed as one array built column by column
_MATCHES_DT = np.dtype([("other_frame", "<i4"), ("count", "<i4"), ("pts_self", "<u8"), ("pts_other", "<u8")])
assert _MATCHES_DT.itemsize == C.sizeof(bt_matches)


def config_default() -> bt_config:
    c = bt_config()
    load().bt_config_default(C.byref(c))
    return c


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)      # torch.cuda.Stream


class PoseGraph:
    """Owns one bt_graph.  Frames are numpy arrays (copied from host) or CUDA
    tensors (read on the device); poses are 4x4 float64 object->camera."""

    def __init__(self, config: bt_config | dict | None = None, stream=None):
        L = load()
        cfg = config_default()
        if isinstance(config, dict):
            for k, v in config.items():
                setattr(cfg, k, v)
        elif config is not None:
            cfg = config
        self._h = C.c_void_p()
        self._stream = stream
        _check(L.bt_graph_create(C.byref(cfg), _stream_handle(stream), C.byref(self._h)), "bt_graph_create")
        self.config = cfg
        # per-solve buffers reused across calls (their addresses taken once)
        self._lib = L
        self._rep = bt_solve_report()
        self._rep_addr = C.addressof(self._rep)
        self._cpi = np.ctypeslib.as_array(self._rep.cost_per_iter)
        self._pout = np.zeros(16 * BT_MAX_NODES)
        self._pout_addr = self._pout.ctypes.data
        self._n_active = None   # cached count; every method that changes the active set resets it

    def close(self):
        if self._h:
            load().bt_graph_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_frame(self, depth, normals, mask, intrinsics, pose, fixed=False, matches=()):
        """matches: iterable of (other_frame_id, pts_self (n,3), pts_other (n,3))."""
        self._n_active = None
        L = load()
        d, kd, mk = _ptr(depth, np.float32)
        n, kn, mk2 = _ptr(normals, np.float32)
        m, km, mk3 = _ptr(mask, np.uint8)
        if not (mk == mk2 == mk3):
            raise ValueError("depth, normals and mask must all be host arrays or all CUDA tensors")
        fx, fy, cx, cy, w, h = intrinsics
        K = bt_intrinsics(fx, fy, cx, cy, w, h)
        P = np.ascontiguousarray(pose, np.float64).reshape(16)
        keep = [kd, kn, km]
        nm = len(matches)
        ms = np.zeros(max(1, nm), _MATCHES_DT)
        if nm:
            others, counts, pa, pb = [], [], [], []
            for other, ps, po in matches:
                a, ka, mka = _ptr(ps, np.float32)
                b, kb, mkb = _ptr(po, np.float32)
                if not (mka == mkb == mk):
                    raise ValueError("matches must use the same memory kind as the frame")
                keep += [ka, kb]
                others.append(int(other))
                counts.append(len(ps))
                pa.append(a.value if isinstance(a, C.c_void_p) else a)
                pb.append(b.value if isinstance(b, C.c_void_p) else b)
            ms["other_frame"][:nm] = others
            ms["count"][:nm] = counts
            ms["pts_self"][:nm] = pa
            ms["pts_other"][:nm] = pb
        fid = C.c_int32(-1)
        _check(L.bt_add_frame(self._h, d, n, m, C.byref(K), _addr(P), int(bool(fixed)), ms.ctypes.data, nm, mk,
                              C.byref(fid)), "bt_add_frame")
        return fid.value

    def set_matches(self, frame_a, frame_b, pts_a, pts_b):
        a, ka, mka = _ptr(pts_a, np.float32)
        b, kb, mkb = _ptr(pts_b, np.float32)
        if mka != mkb:
            raise ValueError("pts_a and pts_b must share a memory kind")
        _check(load().bt_set_matches(self._h, int(frame_a), int(frame_b), int(len(pts_a)), a, b, mka),
               "bt_set_matches")

    def remove_frame(self, frame_id):
        self._n_active = None
        _check(load().bt_remove_frame(self._h, int(frame_id)), "bt_remove_frame")

    def set_active(self, ids):
        arr = np.ascontiguousarray(ids, np.int32)
        self._n_active = None
        _check(self._lib.bt_set_active(self._h, _addr(arr), len(arr)), "bt_set_active")
        self._n_active = len(arr)

    @property
    def num_active(self) -> int:
        if self._n_active is not None:
            return self._n_active
        n = self._lib.bt_num_active(self._h)
        _check(min(n, 0), "bt_num_active")
        self._n_active = n
        return n

    def set_poses(self, poses):
        P = np.ascontiguousarray(poses, np.float64).reshape(-1)
        if P.size != 16 * self.num_active:
            raise ValueError("poses must be (n_active, 4, 4)")
        _check(self._lib.bt_set_poses(self._h, _addr(P)), "bt_set_poses")

    def get_poses(self) -> np.ndarray:
        out = np.zeros((self.num_active, 4, 4))
        _check(load().bt_get_poses(self._h, out.ctypes.data_as(C.POINTER(C.c_double))), "bt_get_poses")
        return out

    def solve(self, iters: int, raise_on_error: bool = True):
        """Returns (poses (N,4,4), report dict)."""
        n = self.num_active
        C.memset(self._rep_addr, 0, C.sizeof(bt_solve_report))
        st = self._lib.bt_solve(self._h, int(iters), self._pout_addr, self._rep_addr)
        if raise_on_error:
            _check(st, "bt_solve")
        if st != BT_OK:
            self._pout[:16 * n] = 0.0    # the poses are not written on failure
        rep = self._rep
        k = rep.iters_run
        r = dict(status=st, iters_run=k, cost_init=rep.cost_init, cost_final=rep.cost_final,
                 dense_cost_final=rep.dense_cost_final, sparse_cost_final=rep.sparse_cost_final,
                 cost_per_iter=self._cpi[:k].copy(), dense_inliers=rep.dense_inliers,
                 dense_pixel_pairs=rep.dense_pixel_pairs)
        return self._pout[:16 * n].reshape(n, 4, 4).copy(), r

    def ransac_init(self, hypotheses: int = 256, seed: int = 0, inlier_dist: float = 0.005, refine: bool = False):
        """bt_ransac_init: the paper's coarse initialisation of the free nodes."""
        _check(load().bt_ransac_init(self._h, int(hypotheses), int(seed) & ((1 << 64) - 1), float(inlier_dist),
                                     1 if refine else 0), "bt_ransac_init")

    def profile_enable(self, on=True):
        """on: False/0 off, True/1 time every solve, k > 1 every k-th solve."""
        _check(load().bt_profile_enable(self._h, int(on)), "bt_profile_enable")

    def profile_read(self) -> dict:
        p = bt_profile()
        _check(load().bt_profile_read(self._h, C.byref(p)), "bt_profile_read")
        out = {k: getattr(p, k) for k, _ in bt_profile._fields_}
        out["solve_phase_cycles"] = list(p.solve_phase_cycles)
        return out

    def debug_associate(self, src_node: int, dst_node: int) -> np.ndarray:
        """bt_debug_associate: target pixel (or -1) of every valid source
        pixel of active node src_node (increasing pixel order) against
        dst_node, at the stored poses."""
        L = load()
        cnt = C.c_int32(0)
        _check(L.bt_debug_associate(self._h, int(src_node), int(dst_node), None, 0, C.byref(cnt)),
               "bt_debug_associate")
        out = np.zeros(max(1, cnt.value), np.int32)
        _check(L.bt_debug_associate(self._h, int(src_node), int(dst_node),
                                    out.ctypes.data_as(C.POINTER(C.c_int32)), len(out), C.byref(cnt)),
               "bt_debug_associate")
        return out[:cnt.value].copy()

    def debug_normal_equations(self):
        """bt_debug_normal_equations: (H (n,n), g (n,), costs dict) of one
        Gauss-Newton iteration at the stored poses, right perturbations of the
        free nodes in active order; the poses are not changed."""
        L = load()
        n = C.c_int32(0)
        cap = 6 * BT_MAX_NODES
        H = np.zeros((cap, cap))
        g = np.zeros(cap)
        c = (C.c_double * 4)()
        _check(L.bt_debug_normal_equations(self._h, H.ctypes.data_as(C.POINTER(C.c_double)),
                                           g.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(n), c),
               "bt_debug_normal_equations")
        m = n.value
        Hm = H.reshape(-1)[:m * m].reshape(m, m).copy()
        return Hm, g[:m].copy(), dict(total=c[0], dense=c[1], sparse=c[2], dense_inliers=int(round(c[3])))

    def eval_cost(self):
        c = (C.c_double * 3)()
        n = C.c_int64()
        _check(load().bt_eval_cost(self._h, c, C.byref(n)), "bt_eval_cost")
        return dict(total=c[0], dense=c[1], sparse=c[2], dense_inliers=n.value)


def _report_dict(rep, st):
    return dict(status=st, iters_run=rep.iters_run, cost_init=rep.cost_init, cost_final=rep.cost_final,
                dense_cost_final=rep.dense_cost_final, sparse_cost_final=rep.sparse_cost_final,
                cost_per_iter=np.array(rep.cost_per_iter[:rep.iters_run]),
                dense_inliers=rep.dense_inliers, dense_pixel_pairs=rep.dense_pixel_pairs)


class Batch:
    """bt_batch: solves many PoseGraphs together (CUDA-graph replay of the
    Gauss-Newton loop, autotuned residual CTA shape)."""

    def __init__(self, stream=None):
        self._h = C.c_void_p()
        self.graphs = []
        _check(load().bt_batch_create(_stream_handle(stream), C.byref(self._h)), "bt_batch_create")

    def add(self, graph: "PoseGraph"):
        _check(load().bt_batch_add(self._h, graph._h), "bt_batch_add")
        self.graphs.append(graph)

    def set_shape(self, shape: int):
        _check(load().bt_batch_set_shape(self._h, int(shape)), "bt_batch_set_shape")

    def tuning(self):
        sh = C.c_int32()
        us = (C.c_double * BT_NUM_SHAPES)()
        _check(load().bt_batch_tuning(self._h, C.byref(sh), us), "bt_batch_tuning")
        return sh.value, list(us)

    def solve(self, iters: int, raise_on_error: bool = True):
        """Returns a list of report dicts (poses are written into the graphs)."""
        n = len(self.graphs)
        reps = (bt_solve_report * max(1, n))()
        st = load().bt_batch_solve(self._h, int(iters), reps)
        if raise_on_error:
            _check(st, "bt_batch_solve")
        return [_report_dict(reps[k], reps[k].status) for k in range(n)]

    def solve_warm(self, warmstart: "WarmStart", iters: int, fallback_iters: int, ref_costs=None,
                   tol: float = 0.01, raise_on_error: bool = True):
        """bt_batch_solve_warm: warm start + `iters` iterations, plain
        `fallback_iters`-iteration solve where the final cost exceeds
        (1 + tol) * ref_costs[k].  Returns report dicts with used_warmstart
        and fell_back."""
        n = len(self.graphs)
        reps = (bt_solve_report * max(1, n))()
        ref = None
        if ref_costs is not None:
            ref = np.ascontiguousarray(ref_costs, np.float64)
            if ref.size != n:
                raise ValueError("one reference cost per graph")
        st = load().bt_batch_solve_warm(self._h, warmstart._h, int(iters), int(fallback_iters),
                                        None if ref is None else ref.ctypes.data_as(C.POINTER(C.c_double)),
                                        float(tol), reps)
        if raise_on_error:
            _check(st, "bt_batch_solve_warm")
        out = []
        for k in range(n):
            d = _report_dict(reps[k], reps[k].status)
            d.update(used_warmstart=reps[k].used_warmstart, fell_back=reps[k].fell_back)
            out.append(d)
        return out

    def close(self):
        if self._h:
            load().bt_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _poses16(poses) -> np.ndarray:
    a = np.asarray(poses, dtype=np.float64)
    if a.shape[-2:] == (3, 3):                     # rotations only: embed in 4x4 poses
        T = np.zeros(a.shape[:-2] + (4, 4))
        T[..., :3, :3] = a
        T[..., 3, 3] = 1.0
        a = T
    return np.ascontiguousarray(a.reshape(-1, 16))


def ransac(pts_i, pts_j, hypotheses: int = 256, seed: int = 0, inlier_dist: float = 0.005, refine: bool = False,
           stream=None):
    """bt_ransac: (4x4 relative pose q ~ M p, inlier count) of one
    correspondence set (numpy arrays or CUDA tensors)."""
    pi, ki, kind = _ptr(pts_i, np.float32)
    pj, kj, kind2 = _ptr(pts_j, np.float32)
    if kind != kind2:
        raise ValueError("both point arrays must live in the same memory")
    M = np.zeros(16)
    cnt = C.c_int32()
    _check(load().bt_ransac(pi, pj, int(ki.shape[0]), kind, int(hypotheses), int(seed) & ((1 << 64) - 1),
                            float(inlier_dist), 1 if refine else 0, M.ctypes.data_as(C.POINTER(C.c_double)),
                            C.byref(cnt), _stream_handle(stream)), "bt_ransac")
    return M.reshape(4, 4), cnt.value


def debug_fail_allocations(n: int) -> int:
    """bt_debug_fail_allocations: the library's next n device or pinned host
    allocations fail as out of memory (0 cancels); returns the pending count."""
    return int(load().bt_debug_fail_allocations(int(n)))


def debug_tensor_wait_ns(ns: int) -> int:
    """bt_debug_tensor_wait_ns: bound of the warm-start forward pass's waits on
    the tensor cores for the launches that follow (ns < 0: default 1 s, 0:
    give up at once); returns the previous bound."""
    return int(load().bt_debug_tensor_wait_ns(int(ns)))


def device_cache_bytes() -> int:
    """Bytes of idle device blocks in the process-wide cache (bt_device_cache_bytes)."""
    return int(load().bt_device_cache_bytes())


def device_cache_trim() -> int:
    """Frees the idle cached blocks above 64 KiB; returns the bytes freed."""
    return int(load().bt_device_cache_trim())


def select_keyframes(pool_poses, pose_current, K: int) -> list:
    """bt_select_keyframes: pool indices (selection order) of the greedy
    keyframe selection of Sec. IV-C.  Poses as (n, 4, 4) or rotations (n, 3, 3)."""
    P = _poses16(pool_poses)
    cur = _poses16(pose_current)
    out = np.zeros(max(1, int(K)), np.int32)
    n = load().bt_select_keyframes(P.ctypes.data_as(C.POINTER(C.c_double)), len(P),
                                   cur.ctypes.data_as(C.POINTER(C.c_double)), int(K),
                                   out.ctypes.data_as(C.POINTER(C.c_int32)))
    _check(min(n, 0), "bt_select_keyframes")
    return out[:n].tolist()


def is_novel_view(pool_poses, pose_current, min_deg: float = 10.0) -> bool:
    """bt_is_novel_view: the pool augmentation rule of Sec. IV-E."""
    P = _poses16(pool_poses)
    cur = _poses16(pose_current)
    r = load().bt_is_novel_view(P.ctypes.data_as(C.POINTER(C.c_double)), len(P),
                                cur.ctypes.data_as(C.POINTER(C.c_double)), float(min_deg))
    _check(min(r, 0), "bt_is_novel_view")
    return bool(r)


WS_NUM_PARAMS = 67590


def _ids(ids) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(ids, dtype=np.int32).ravel())


class WarmStart:
    """bt_warmstart: the learned warm start (set network + FP64 relative-pose
    averaging), its device-resident training set and its training step."""

    def __init__(self, params=None, stream=None):
        self._h = C.c_void_p()
        _check(load().bt_warmstart_create(_stream_handle(stream), C.byref(self._h)), "bt_warmstart_create")
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        if _is_torch(params) and params.is_cuda:
            if params.dtype.itemsize != 4 or params.numel() != WS_NUM_PARAMS or not params.is_contiguous():
                raise ValueError("parameters: contiguous float32 tensor of %d" % WS_NUM_PARAMS)
            _check(load().bt_warmstart_set_params(self._h, C.c_void_p(params.data_ptr()), BT_DEVICE),
                   "bt_warmstart_set_params")
            return
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
        if a.size != WS_NUM_PARAMS:
            raise ValueError("parameters: %d floats expected, got %d" % (WS_NUM_PARAMS, a.size))
        _check(load().bt_warmstart_set_params(self._h, C.c_void_p(a.ctypes.data), BT_HOST),
               "bt_warmstart_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(WS_NUM_PARAMS, np.float32)
        _check(load().bt_warmstart_get_params(self._h, C.c_void_p(out.ctypes.data), BT_HOST),
               "bt_warmstart_get_params")
        return out

    def get_adam(self):
        """(first moments, second moments, step) of the Adam optimiser."""
        m = np.empty(WS_NUM_PARAMS, np.float32)
        v = np.empty(WS_NUM_PARAMS, np.float32)
        t = C.c_int32()
        _check(load().bt_warmstart_get_adam(self._h, C.c_void_p(m.ctypes.data), C.c_void_p(v.ctypes.data),
                                            C.byref(t), BT_HOST), "bt_warmstart_get_adam")
        return m, v, t.value

    def set_adam(self, m, v, step: int):
        m = np.ascontiguousarray(np.asarray(m, np.float32).ravel())
        v = np.ascontiguousarray(np.asarray(v, np.float32).ravel())
        if m.size != WS_NUM_PARAMS or v.size != WS_NUM_PARAMS:
            raise ValueError("moments: %d floats each" % WS_NUM_PARAMS)
        _check(load().bt_warmstart_set_adam(self._h, C.c_void_p(m.ctypes.data), C.c_void_p(v.ctypes.data),
                                            int(step), BT_HOST), "bt_warmstart_set_adam")

    def add_set(self, pts_i, pts_j, pose_i, pose_j, label_i=None, label_j=None):
        """One training sample: point pairs and the two frames' initial poses
        (and, optionally, the poses a solve converged to)."""
        pi, ki, kind = _ptr(pts_i, np.float32)
        pj, kj, kind2 = _ptr(pts_j, np.float32)
        if kind != kind2:
            raise ValueError("both point arrays must live in the same memory")
        n = int(ki.shape[0])
        poses = [None if T is None else np.ascontiguousarray(T, np.float64).reshape(16)
                 for T in (pose_i, pose_j, label_i, label_j)]
        ptrs = [None if T is None else T.ctypes.data_as(C.POINTER(C.c_double)) for T in poses]
        _check(load().bt_warmstart_add_set(self._h, pi, pj, n, *ptrs, kind), "bt_warmstart_add_set")

    def add_graph(self, graph: "PoseGraph", poses_init, poses_label=None):
        P0 = np.ascontiguousarray(poses_init, np.float64)
        PL = None if poses_label is None else np.ascontiguousarray(poses_label, np.float64)
        _check(load().bt_warmstart_add_graph(self._h, graph._h, P0.ctypes.data_as(C.POINTER(C.c_double)),
                                             None if PL is None else PL.ctypes.data_as(C.POINTER(C.c_double))),
               "bt_warmstart_add_graph")

    def num_samples(self) -> int:
        n = load().bt_warmstart_num_samples(self._h)
        _check(min(n, 0), "bt_warmstart_num_samples")
        return n

    def clear_samples(self):
        _check(load().bt_warmstart_clear_samples(self._h), "bt_warmstart_clear_samples")

    def sample(self, k: int):
        c = (C.c_float * 3)()
        y = (C.c_float * 6)()
        _check(load().bt_warmstart_get_sample(self._h, int(k), c, y), "bt_warmstart_get_sample")
        return np.array(c[:], np.float32), np.array(y[:], np.float32)

    def predict(self, ids) -> np.ndarray:
        a = _ids(ids)
        out = np.empty((a.size, 6), np.float32)
        _check(load().bt_warmstart_predict(self._h, a.ctypes.data_as(C.POINTER(C.c_int32)), a.size,
                                           out.ctypes.data_as(C.POINTER(C.c_float))), "bt_warmstart_predict")
        return out

    def gradient(self, ids):
        a = _ids(ids)
        g = np.empty(WS_NUM_PARAMS, np.float32)
        loss = C.c_double()
        _check(load().bt_warmstart_gradient(self._h, a.ctypes.data_as(C.POINTER(C.c_int32)), a.size,
                                            g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)),
               "bt_warmstart_gradient")
        return loss.value, g

    def train_step(self, ids, lr: float, want_loss: bool = False):
        a = _ids(ids)
        loss = C.c_double()
        _check(load().bt_warmstart_train_step(self._h, a.ctypes.data_as(C.POINTER(C.c_int32)), a.size, float(lr),
                                              C.byref(loss) if want_loss else None), "bt_warmstart_train_step")
        return loss.value if want_loss else None

    def apply(self, graph: "PoseGraph"):
        _check(load().bt_warmstart_apply(self._h, graph._h), "bt_warmstart_apply")

    def apply_batch(self, batch: "Batch", raise_on_error: bool = True):
        n = len(batch.graphs)
        st_arr = (C.c_int32 * max(1, n))()
        st = load().bt_warmstart_apply_batch(self._h, batch._h, st_arr)
        if raise_on_error:
            _check(st, "bt_warmstart_apply_batch")
        return list(st_arr[:n])

    def close(self):
        if self._h:
            load().bt_warmstart_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def noalloc_argument_error(torch, device: int, size_a, size_b, depth_a, normals_a, mask_a, depth_b, normals_b,
                           mask_b, out) -> str:
    """What is wrong with the buffers of a bt_pair_dense_energy_noalloc call
    ("" if nothing): each must be a contiguous CUDA tensor on `device`; depth
    float32 with W*H elements, normals float32 with 3*W*H, mask uint8 or bool
    with W*H, out float64 with at least 2.  The C call reads and writes them by
    pointer and cannot check any of this itself."""
    named = (("depth_a", depth_a), ("normals_a", normals_a), ("mask_a", mask_a), ("depth_b", depth_b),
             ("normals_b", normals_b), ("mask_b", mask_b), ("out", out))
    for name, x in named:
        if not (getattr(x, "is_cuda", False) and x.is_contiguous()):
            return f"{name} must be a contiguous CUDA tensor"
        if x.device.index != device:
            return f"{name} is on {x.device}, not cuda:{device}"
    for tag, (w, h), d, n, m in (("a", size_a, depth_a, normals_a, mask_a), ("b", size_b, depth_b, normals_b,
                                                                               mask_b)):
        hw = int(w) * int(h)
        if d.dtype != torch.float32 or d.numel() != hw:
            return f"depth_{tag} must be float32 with W*H = {hw} elements"
        if n.dtype != torch.float32 or n.numel() != 3 * hw:
            return f"normals_{tag} must be float32 with 3*W*H = {3 * hw} elements"
        if m.dtype not in (torch.uint8, torch.bool) or m.numel() != hw:
            return f"mask_{tag} must be uint8 or bool with W*H = {hw} elements"
    if out.dtype != torch.float64 or out.numel() < 2:
        return "out must be float64 with at least 2 elements"
    return ""


def pair_dense_energy_noalloc(depth_a, normals_a, mask_a, intr_a, pose_a, depth_b, normals_b, mask_b, intr_b,
                              pose_b, out, config: bt_config | None = None, stream=None):
    """bt_pair_dense_energy_noalloc: all image buffers and `out` (2 float64)
    must be contiguous CUDA tensors on the current device -- depth float32
    with W*H elements, normals float32 with 3*W*H, mask uint8 or bool with
    W*H, out float64 with at least 2 -- since the C call reads and writes
    them by pointer; enqueues on `stream` and returns immediately."""
    import torch
    Ka = bt_intrinsics(*intr_a)
    Kb = bt_intrinsics(*intr_b)
    err = noalloc_argument_error(torch, torch.cuda.current_device(), (Ka.width, Ka.height), (Kb.width, Kb.height),
                                 depth_a, normals_a, mask_a, depth_b, normals_b, mask_b, out)
    if err:
        raise ValueError("bt_pair_dense_energy_noalloc: " + err)
    Pa = np.ascontiguousarray(pose_a, np.float64).reshape(16)
    Pb = np.ascontiguousarray(pose_b, np.float64).reshape(16)
    cfg = config if config is not None else config_default()
    L = load()
    st = L.bt_pair_dense_energy_noalloc(
        C.c_void_p(depth_a.data_ptr()), C.c_void_p(normals_a.data_ptr()), C.c_void_p(mask_a.data_ptr()),
        C.byref(Ka), Pa.ctypes.data_as(C.POINTER(C.c_double)),
        C.c_void_p(depth_b.data_ptr()), C.c_void_p(normals_b.data_ptr()), C.c_void_p(mask_b.data_ptr()),
        C.byref(Kb), Pb.ctypes.data_as(C.POINTER(C.c_double)), C.byref(cfg),
        C.c_void_p(out.data_ptr()), _stream_handle(stream))
    if st != BT_OK:
        raise RuntimeError(f"bt_pair_dense_energy_noalloc: {L.bt_status_str(st).decode()} ({st}): "
                           f"{L.bt_noalloc_last_error().decode()}")


def graph_from_synth(sg, config=None, stream=None, device=None) -> PoseGraph:
    """Loads a synthetic graph (attributes renders, cams, matches, pose_init,
    fixed) into a PoseGraph; device = 'cuda' passes CUDA tensors instead of
    host arrays."""
    pg = PoseGraph(config, stream)
    ids = []
    if device is not None:
        import torch

        def conv(x):
            return torch.as_tensor(np.ascontiguousarray(x), device=device)
    else:
        def conv(x):
            return x
    by_new = {}
    for (i, j, pi, pj) in sg.matches:
        by_new.setdefault(j, []).append((i, pj, pi))
    for k in range(len(sg.renders)):
        r, cam = sg.renders[k], sg.cams[k]
        ms = [(ids[i], conv(ps), conv(po)) for (i, ps, po) in by_new.get(k, [])]
        ids.append(pg.add_frame(conv(r.depth), conv(r.normals), conv(r.mask), cam.as_tuple(),
                                sg.pose_init[k], bool(sg.fixed[k]), ms))
    pg.frame_ids = ids
    return pg
