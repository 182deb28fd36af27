"""ctypes binding of libba.so (the C ABI declared in include/ba.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  The functions keep the C names (ba_create, ba_set_problem,
ba_solve, ba_get_state, ba_set_state, ba_solve_batch, ba_create_server,
ba_submit, ba_poll, ba_destroy, ba_last_error).  PyTorch, when asked for,
supplies the device memory (its caching allocator) and the CUDA stream.

Importing this module does not need a GPU; loading the library does not
either; creating a handle does.  If libba.so has not been built the first
call raises an error; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, c_char_p, c_double, c_int, c_int32,
                    c_int64, c_size_t, c_uint8, c_uint64, c_void_p)
from typing import Optional, Sequence

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libba.so")

BA_OK, BA_ERR_INVALID_ARG, BA_ERR_OOM, BA_ERR_CUDA, BA_ERR_NOT_READY = 0, 1, 2, 3, 4
BA_ERR_TIMEOUT, BA_ERR_BUSY, BA_ERR_STATE, BA_ERR_NUMERIC = 5, 6, 7, 8
BA_FP64, BA_FP32 = 0, 1
BA_SOLVER_AUTO, BA_SOLVER_DENSE, BA_SOLVER_PCG = 0, 1, 2
BA_MEM_HOST, BA_MEM_DEVICE = 0, 1
BA_MAX_ITERS = 256

STATUS_NAMES = {0: "BA_OK", 1: "BA_ERR_INVALID_ARG", 2: "BA_ERR_OOM", 3: "BA_ERR_CUDA",
                4: "BA_ERR_NOT_READY", 5: "BA_ERR_TIMEOUT", 6: "BA_ERR_BUSY",
                7: "BA_ERR_STATE", 8: "BA_ERR_NUMERIC"}

ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p)


class Options(Structure):
    _fields_ = [("precision", c_int), ("solver", c_int), ("max_lm_iters", c_int),
                ("huber_delta", c_double), ("pcg_tol", c_double), ("pcg_max_iters", c_int),
                ("refine", c_int), ("refine_max", c_int), ("refine_tol", c_double),
                ("mu0", c_double), ("dense_max_dim", c_int), ("device", c_int),
                ("cuda_stream", c_void_p), ("use_graph", c_int), ("alloc", ALLOC_FN),
                ("free_fn", FREE_FN), ("alloc_ctx", c_void_p), ("serve_arena_bytes", c_size_t),
                ("serve_slots", c_int), ("serve_queue", c_int), ("profile", c_int),
                ("pcg_variant", c_int), ("mu_min", c_double),
                ("serve_tick_ms", c_double),
                ("serve_split_ms", c_double),
                ("prior_seq_weight", c_double),
                ("prior_abs_weight", c_double),
                ("pcg_resident_cap", c_int)]


class Intrinsics(Structure):
    _fields_ = [("fx", c_double), ("fy", c_double), ("cx", c_double), ("cy", c_double)]


class Report(Structure):
    _fields_ = [("status", c_int32), ("n_iters", c_int32), ("n_accepted", c_int32),
                ("solver", c_int32), ("cost", c_double * (BA_MAX_ITERS + 1)),
                ("accepted", c_uint8 * BA_MAX_ITERS), ("mu", c_double * BA_MAX_ITERS),
                ("pcg_iters", c_int32 * BA_MAX_ITERS),
                ("pcg_rel_residual", c_double * BA_MAX_ITERS),
                ("gain", c_double * BA_MAX_ITERS), ("rmse_px", c_double),
                ("n_valid_obs", c_int64), ("solve_ms", c_double), ("setup_ms", c_double),
                ("n_kernels", c_int32), ("pcg_variant", c_int32)]

    def as_dict(self):
        n = self.n_iters
        return dict(status=self.status, n_iters=n, n_accepted=self.n_accepted,
                    solver=self.solver, costs=np.array(self.cost[:n + 1]),
                    accepted=np.array(self.accepted[:n], dtype=bool),
                    mu=np.array(self.mu[:n]), pcg_iters=np.array(self.pcg_iters[:n]),
                    pcg_rel_residual=np.array(self.pcg_rel_residual[:n]),
                    gain=np.array(self.gain[:n]), rmse_px=self.rmse_px,
                    n_valid_obs=self.n_valid_obs, solve_ms=self.solve_ms,
                    setup_ms=self.setup_ms, n_kernels=self.n_kernels,
                    pcg_variant=self.pcg_variant)


class KernelStat(Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", c_int32), ("pad", c_int32),
                ("total_ms", c_double)]


class Problem(Structure):
    _fields_ = [("n_cams", c_int32), ("n_pts", c_int32), ("n_obs", c_int64),
                ("cam_qt", c_void_p), ("pts", c_void_p), ("obs_cam", c_void_p),
                ("obs_pt", c_void_p), ("obs_uv", c_void_p), ("cam_fixed", c_void_p),
                ("K", Intrinsics), ("cam_qt_out", c_void_p), ("pts_out", c_void_p)]


class Result(Structure):
    _fields_ = [("status", c_int32), ("n_iters", c_int32), ("n_accepted", c_int32),
                ("pad", c_int32), ("initial_cost", c_double), ("final_cost", c_double),
                ("rmse_px", c_double), ("latency_ms", c_double),
                ("cost", c_double * (BA_MAX_ITERS + 1))]

    def costs(self):
        return np.array(self.cost[:self.n_iters + 1])


class BAError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_LIB = None

_SIGNATURES = {
    "ba_options_default": (None, [POINTER(Options)]),
    "ba_create": (c_int, [POINTER(Options), POINTER(c_void_p)]),
    "ba_set_problem": (c_int, [c_void_p, c_int32, c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, POINTER(Intrinsics), c_void_p, c_int]),
    "ba_solve": (c_int, [c_void_p, POINTER(Report)]),
    "ba_get_state": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "ba_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "ba_get_reduced_system": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "ba_destroy": (None, [c_void_p]),
    "ba_kernel_stats": (c_int, [c_void_p, c_void_p, c_int32, POINTER(c_int32)]),
    "ba_last_error": (c_char_p, [c_void_p]),
    "ba_solve_batch": (c_int, [c_void_p, c_int32, POINTER(Problem), POINTER(Result)]),
    "ba_get_batch_schedule": (c_int, [c_void_p, POINTER(c_int32), POINTER(c_int32)]),
    "ba_set_batch_schedule": (c_int, [c_void_p, c_int32, c_int32]),
    "ba_tune_batch": (c_int, [c_void_p, c_int32, POINTER(Problem), POINTER(c_int32),
                              POINTER(c_int32)]),
    "ba_create_server": (c_int, [POINTER(Options), POINTER(c_void_p)]),
    "ba_submit": (c_int, [c_void_p, POINTER(Problem), POINTER(c_uint64)]),
    "ba_poll": (c_int, [c_void_p, c_uint64, POINTER(Result)]),
    "ba_cost_noalloc": (c_int, [c_int, c_void_p, c_int32, c_int32, c_int64, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p, POINTER(Intrinsics), c_double,
                                c_void_p]),
    "ba_selftest_barrier": (c_int, [c_int32, c_int32, c_int32, c_double, POINTER(c_int32),
                                    POINTER(c_double)]),
    "ba_reprojection_errors": (c_int, [c_int32, c_void_p, c_int32, c_int32, c_int64, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_void_p,
                                       POINTER(Intrinsics), c_double, c_void_p, c_void_p,
                                       POINTER(c_int64), c_int32]),
    "ba_triangulate": (c_int, [c_int32, c_void_p, c_int32, c_int32, c_int64, c_void_p, c_void_p,
                               c_void_p, c_void_p, POINTER(Intrinsics), c_void_p, c_void_p,
                               c_void_p, c_int32]),
    # pose-graph optimisation (ba_pose_graph.h)
    "ba_pg_create": (c_int, [POINTER(Options), POINTER(c_void_p)]),
    "ba_pg_set_graph": (c_int, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_int]),
    "ba_pg_solve": (c_int, [c_void_p, POINTER(Report)]),
    "ba_pg_get_state": (c_int, [c_void_p, c_void_p, c_int]),
    "ba_pg_last_error": (c_char_p, [c_void_p]),
    "ba_pg_destroy": (None, [c_void_p]),
    # rig BA with extrinsic refinement (ba_rig.h)
    "ba_rig_create": (c_int, [POINTER(Options), POINTER(c_void_p)]),
    "ba_rig_set_problem": (c_int, [c_void_p, c_int32, c_int32, c_int32, c_int64, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   POINTER(Intrinsics), c_void_p, c_void_p]),
    "ba_rig_solve": (c_int, [c_void_p, POINTER(Report)]),
    "ba_rig_get_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ba_rig_last_error": (c_char_p, [c_void_p]),
    "ba_rig_destroy": (None, [c_void_p]),
}

EXPORTS = tuple(_SIGNATURES)


def lib():
    """The loaded libba.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -m "
                               "paper_2510_15271_b300.build` (or __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def ba_last_error(h=None) -> str:
    msg = lib().ba_last_error(h)
    return msg.decode() if msg else ""


def _check(status, h=None):
    if status != BA_OK:
        raise BAError(status, ba_last_error(h))


def ba_options_default(**kw) -> Options:
    o = Options()
    lib().ba_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class _TorchMemory:
    """PyTorch caching-allocator callbacks (kept alive with the handle)."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class Handle:
    """Owns one ba_handle (solver or server)."""

    def __init__(self, ptr, keep=()):
        self.ptr = ptr
        self._keep = keep

    def close(self):
        if self.ptr:
            lib().ba_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def ba_create(opts: Optional[Options] = None, use_torch: bool = False, server: bool = False,
              **kw) -> Handle:
    """Create a solver (or, with server=True, a serving) handle.  use_torch
    hands the library PyTorch's current CUDA stream and caching allocator."""
    o = opts if opts is not None else ba_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    keep = ()
    if use_torch:
        import torch
        mem = _TorchMemory(o.device)
        o.alloc = mem.alloc
        o.free_fn = mem.free
        o.cuda_stream = torch.cuda.current_stream(o.device).cuda_stream
        keep = (mem,)
    h = c_void_p()
    fn = lib().ba_create_server if server else lib().ba_create
    _check(fn(ctypes.byref(o), ctypes.byref(h)), None)
    return Handle(h, keep)


def _host(a, dtype, shape=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if shape is not None:
        arr = arr.reshape(shape)
    return arr


def _is_torch_cuda(a):
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def ba_set_problem(h: Handle, cam_qt, pts, obs_cam, obs_pt, obs_uv, intrinsics,
                   cam_fixed=None):
    """Load a problem.  Arrays are numpy/host arrays or CUDA torch tensors
    (all of one kind).  intrinsics = (fx, fy, cx, cy)."""
    K = Intrinsics(*[float(v) for v in intrinsics])
    if _is_torch_cuda(obs_uv):
        import torch
        ts = [cam_qt.contiguous().to(torch.float64), pts.contiguous().to(torch.float64),
              obs_cam.contiguous().to(torch.int32), obs_pt.contiguous().to(torch.int32),
              obs_uv.contiguous().to(torch.float64)]
        fx = None if cam_fixed is None else cam_fixed.contiguous().to(torch.uint8)
        st = lib().ba_set_problem(h.ptr, ts[0].shape[0], ts[1].shape[0], ts[2].shape[0],
                                  ts[0].data_ptr(), ts[1].data_ptr(), ts[2].data_ptr(),
                                  ts[3].data_ptr(), ts[4].data_ptr(), ctypes.byref(K),
                                  None if fx is None else fx.data_ptr(), BA_MEM_DEVICE)
        torch.cuda.current_stream().synchronize()
        _check(st, h.ptr)
        return
    q = _host(cam_qt, np.float64).reshape(-1, 7)
    p = _host(pts, np.float64).reshape(-1, 3)
    c = _host(obs_cam, np.int32)
    j = _host(obs_pt, np.int32)
    uv = _host(obs_uv, np.float64).reshape(-1, 2)
    fx = None if cam_fixed is None else _host(cam_fixed, np.uint8)
    st = lib().ba_set_problem(h.ptr, q.shape[0], p.shape[0], c.shape[0], q.ctypes.data,
                              p.ctypes.data, c.ctypes.data, j.ctypes.data, uv.ctypes.data,
                              ctypes.byref(K), None if fx is None else fx.ctypes.data,
                              BA_MEM_HOST)
    _check(st, h.ptr)


def ba_solve(h: Handle) -> dict:
    r = Report()
    st = lib().ba_solve(h.ptr, ctypes.byref(r))
    _check(st, h.ptr)
    return r.as_dict()


def ba_get_state(h: Handle, n_cams: int, n_pts: int):
    q = np.empty((n_cams, 7))
    p = np.empty((n_pts, 3))
    _check(lib().ba_get_state(h.ptr, q.ctypes.data, p.ctypes.data, BA_MEM_HOST), h.ptr)
    return q, p


def ba_set_state(h: Handle, cam_qt, pts):
    q = _host(cam_qt, np.float64)
    p = _host(pts, np.float64)
    _check(lib().ba_set_state(h.ptr, q.ctypes.data, p.ctypes.data, BA_MEM_HOST), h.ptr)


def ba_get_reduced_system(h: Handle, n_cams: int):
    """(S, b, x) of the last linear solve as the device holds them (dense
    FP64 copies; see ba.h)."""
    n = 6 * n_cams
    S = np.empty((n, n))
    b = np.empty(n)
    x = np.empty(n)
    _check(lib().ba_get_reduced_system(h.ptr, n, S.ctypes.data, b.ctypes.data, x.ctypes.data),
           h.ptr)
    return S, b, x


def ba_destroy(h: Handle):
    h.close()


def ba_kernel_stats(h: Handle) -> dict:
    """{kernel name: (launches, total device ms)} of the last solve
    (handle created with profile=1)."""
    arr = (KernelStat * 32)()
    n = c_int32()
    _check(lib().ba_kernel_stats(h.ptr, arr, 32, ctypes.byref(n)), h.ptr)
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}


# --------------------------------------------------------------------------- pose graphs

class PoseGraphHandle:
    """Owns one ba_pose_graph."""

    def __init__(self, ptr, keep=()):
        self.ptr = ptr
        self._keep = keep

    def close(self):
        if self.ptr:
            lib().ba_pg_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _pg_check(status, g):
    if status != BA_OK:
        msg = lib().ba_pg_last_error(g)
        raise BAError(status, msg.decode() if msg else "")


def ba_pg_create(opts: Optional[Options] = None, use_torch: bool = False,
                 **kw) -> PoseGraphHandle:
    """Create a pose-graph solver; use_torch as for ba_create."""
    o = opts if opts is not None else ba_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    keep = ()
    if use_torch:
        import torch
        mem = _TorchMemory(o.device)
        o.alloc = mem.alloc
        o.free_fn = mem.free
        o.cuda_stream = torch.cuda.current_stream(o.device).cuda_stream
        keep = (mem,)
    g = c_void_p()
    _pg_check(lib().ba_pg_create(ctypes.byref(o), ctypes.byref(g)), None)
    return PoseGraphHandle(g, keep)


def ba_pg_set_graph(g: PoseGraphHandle, node_qt, edge_ij, edge_qt, edge_w, node_fixed=None):
    """Load a graph from host arrays: node_qt (n, 7), edge_ij (E, 2), edge_qt
    (E, 7) measured pose of node i in node j, edge_w (E,), node_fixed (n,)."""
    q = _host(node_qt, np.float64).reshape(-1, 7)
    ij = _host(edge_ij, np.int32).reshape(-1, 2)
    eq = _host(edge_qt, np.float64).reshape(-1, 7)
    w = _host(edge_w, np.float64).reshape(-1)
    fx = None if node_fixed is None else _host(node_fixed, np.uint8)
    st = lib().ba_pg_set_graph(g.ptr, q.shape[0], q.ctypes.data, ij.shape[0], ij.ctypes.data,
                               eq.ctypes.data, w.ctypes.data,
                               None if fx is None else fx.ctypes.data, BA_MEM_HOST)
    _pg_check(st, g.ptr)


def ba_pg_solve(g: PoseGraphHandle) -> dict:
    r = Report()
    st = lib().ba_pg_solve(g.ptr, ctypes.byref(r))
    _pg_check(st, g.ptr)
    return r.as_dict()


def ba_pg_get_state(g: PoseGraphHandle, n_nodes: int) -> np.ndarray:
    q = np.empty((n_nodes, 7))
    _pg_check(lib().ba_pg_get_state(g.ptr, q.ctypes.data, BA_MEM_HOST), g.ptr)
    return q


def ba_pg_destroy(g: PoseGraphHandle):
    g.close()


# --------------------------------------------------------------------------- rig BA

class RigHandle:
    """Owns one ba_rig."""

    def __init__(self, ptr):
        self.ptr = ptr
        self.sizes = None

    def close(self):
        if self.ptr:
            lib().ba_rig_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _rig_check(status, g):
    if status != BA_OK:
        msg = lib().ba_rig_last_error(g)
        raise BAError(status, msg.decode() if msg else "")


def ba_rig_create(opts: Optional[Options] = None, **kw) -> RigHandle:
    o = opts if opts is not None else ba_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    g = c_void_p()
    _rig_check(lib().ba_rig_create(ctypes.byref(o), ctypes.byref(g)), None)
    return RigHandle(g)


def ba_rig_set_problem(g: RigHandle, vehicle_qt, extr_qt, pts, obs_frame, obs_rc, obs_pt, obs_uv,
                       intrinsics, frame_fixed=None, rc_fixed=None):
    """Host arrays: vehicle_qt (F, 7) world -> vehicle, extr_qt (R, 7)
    vehicle -> camera, pts (P, 3), observations, intrinsics (fx, fy, cx, cy)."""
    vq = _host(vehicle_qt, np.float64).reshape(-1, 7)
    eq = _host(extr_qt, np.float64).reshape(-1, 7)
    p = _host(pts, np.float64).reshape(-1, 3)
    f = _host(obs_frame, np.int32)
    c = _host(obs_rc, np.int32)
    j = _host(obs_pt, np.int32)
    uv = _host(obs_uv, np.float64).reshape(-1, 2)
    K = Intrinsics(*[float(v) for v in intrinsics])
    ff = None if frame_fixed is None else _host(frame_fixed, np.uint8)
    rf = None if rc_fixed is None else _host(rc_fixed, np.uint8)
    st = lib().ba_rig_set_problem(g.ptr, vq.shape[0], eq.shape[0], p.shape[0], f.shape[0],
                                  vq.ctypes.data, eq.ctypes.data, p.ctypes.data, f.ctypes.data,
                                  c.ctypes.data, j.ctypes.data, uv.ctypes.data, ctypes.byref(K),
                                  None if ff is None else ff.ctypes.data,
                                  None if rf is None else rf.ctypes.data)
    _rig_check(st, g.ptr)
    g.sizes = (vq.shape[0], eq.shape[0], p.shape[0])


def ba_rig_solve(g: RigHandle) -> dict:
    r = Report()
    _rig_check(lib().ba_rig_solve(g.ptr, ctypes.byref(r)), g.ptr)
    return r.as_dict()


def ba_rig_get_state(g: RigHandle):
    F, R, P = g.sizes
    vq, eq, p = np.empty((F, 7)), np.empty((R, 7)), np.empty((P, 3))
    _rig_check(lib().ba_rig_get_state(g.ptr, vq.ctypes.data, eq.ctypes.data, p.ctypes.data),
               g.ptr)
    return vq, eq, p


# --------------------------------------------------------------------------- batch / serve

class _ProblemArrays:
    """Host arrays of one ba_problem kept alive for the call."""

    def __init__(self, cam_qt, pts, obs_cam, obs_pt, obs_uv, intrinsics, cam_fixed=None,
                 want_state=False):
        self.q = _host(cam_qt, np.float64).reshape(-1, 7)
        self.p = _host(pts, np.float64).reshape(-1, 3)
        self.c = _host(obs_cam, np.int32)
        self.j = _host(obs_pt, np.int32)
        self.uv = _host(obs_uv, np.float64).reshape(-1, 2)
        self.fx = None if cam_fixed is None else _host(cam_fixed, np.uint8)
        self.q_out = np.empty_like(self.q) if want_state else None
        self.p_out = np.empty_like(self.p) if want_state else None
        self.st = Problem()
        self.st.n_cams, self.st.n_pts, self.st.n_obs = self.q.shape[0], self.p.shape[0], self.c.shape[0]
        self.st.cam_qt, self.st.pts = self.q.ctypes.data, self.p.ctypes.data
        self.st.obs_cam, self.st.obs_pt = self.c.ctypes.data, self.j.ctypes.data
        self.st.obs_uv = self.uv.ctypes.data
        self.st.cam_fixed = None if self.fx is None else self.fx.ctypes.data
        self.st.K = Intrinsics(*[float(v) for v in intrinsics])
        self.st.cam_qt_out = None if self.q_out is None else self.q_out.ctypes.data
        self.st.pts_out = None if self.p_out is None else self.p_out.ctypes.data

    @classmethod
    def from_scene(cls, s, want_state=False):
        return cls(s.cam_qt, s.pts, s.obs_cam, s.obs_pt, s.obs_uv, s.intrinsics(), s.cam_fixed,
                   want_state)


def ba_solve_batch(h: Handle, problems: Sequence[_ProblemArrays]):
    n = len(problems)
    arr = (Problem * n)(*[p.st for p in problems])
    res = (Result * n)()
    st = lib().ba_solve_batch(h.ptr, n, arr, res)
    _check(st, h.ptr)
    return list(res)


def ba_tune_batch(h: Handle, problems: Sequence[_ProblemArrays]):
    n = len(problems)
    arr = (Problem * n)(*[p.st for p in problems])
    t, c = c_int32(), c_int32()
    _check(lib().ba_tune_batch(h.ptr, n, arr, ctypes.byref(t), ctypes.byref(c)), h.ptr)
    return t.value, c.value


def ba_get_batch_schedule(h: Handle):
    t, c = c_int32(), c_int32()
    _check(lib().ba_get_batch_schedule(h.ptr, ctypes.byref(t), ctypes.byref(c)), h.ptr)
    return t.value, c.value


def ba_set_batch_schedule(h: Handle, threads: int, ctas_per_sm: int):
    _check(lib().ba_set_batch_schedule(h.ptr, threads, ctas_per_sm), h.ptr)


def ba_create_server(opts: Optional[Options] = None, **kw) -> Handle:
    return ba_create(opts, server=True, **kw)


def ba_submit(h: Handle, prob: _ProblemArrays) -> int:
    rid = c_uint64()
    _check(lib().ba_submit(h.ptr, ctypes.byref(prob.st), ctypes.byref(rid)), h.ptr)
    return rid.value


def ba_poll(h: Handle, req_id: int):
    """Result of a request, or None while it is not done."""
    r = Result()
    st = lib().ba_poll(h.ptr, req_id, ctypes.byref(r))
    if st == BA_ERR_NOT_READY:
        return None
    _check(st, h.ptr)
    return r


# --------------------------------------------------------------------------- convenience

def ba_selftest_barrier(device: int = 0, blocks: int = 8, expected: int = 8,
                        limit_ms: float = 50.0):
    """(timed_out, waited_ms) of one grid barrier of `blocks` CTAs expecting
    `expected` arrivals (ba_selftest_barrier)."""
    t = c_int32()
    w = c_double()
    _check(lib().ba_selftest_barrier(device, blocks, expected, limit_ms, ctypes.byref(t),
                                     ctypes.byref(w)))
    return bool(t.value), w.value


def _ptr(a):
    return None if a is None else a.ctypes.data_as(c_void_p)


def ba_reprojection_errors(cam_qt, pts, obs_cam, obs_pt, obs_uv, intrinsics, threshold_px,
                           device: int = 0, want_err2: bool = True):
    """(err2 or None, inlier mask (bool), inlier count) of every observation
    (ba_reprojection_errors, host arrays)."""
    q = _host(cam_qt, np.float64, (-1, 7))
    X = _host(pts, np.float64, (-1, 3))
    oc = _host(obs_cam, np.int32)
    op = _host(obs_pt, np.int32)
    uv = _host(obs_uv, np.float64, (-1, 2))
    n = oc.shape[0]
    err2 = np.empty(n) if want_err2 else None
    inl = np.empty(n, dtype=np.uint8)
    cnt = c_int64()
    K = Intrinsics(*intrinsics)
    _check(lib().ba_reprojection_errors(device, None, q.shape[0], X.shape[0], n, _ptr(q), _ptr(X),
                                        _ptr(oc), _ptr(op), _ptr(uv), ctypes.byref(K),
                                        float(threshold_px), _ptr(err2), _ptr(inl),
                                        ctypes.byref(cnt), BA_MEM_HOST))
    return err2, inl.astype(bool), int(cnt.value)


def ba_triangulate(cam_qt, obs_cam, obs_pt, obs_uv, intrinsics, n_pts: int, mask=None,
                   device: int = 0):
    """(points (n_pts, 3), status (n_pts,) int8) by DLT (ba_triangulate, host
    arrays)."""
    q = _host(cam_qt, np.float64, (-1, 7))
    oc = _host(obs_cam, np.int32)
    op = _host(obs_pt, np.int32)
    uv = _host(obs_uv, np.float64, (-1, 2))
    m = None if mask is None else _host(np.asarray(mask).astype(np.uint8), np.uint8)
    X = np.empty((n_pts, 3))
    status = np.empty(n_pts, dtype=np.int8)
    K = Intrinsics(*intrinsics)
    _check(lib().ba_triangulate(device, None, q.shape[0], n_pts, oc.shape[0], _ptr(q), _ptr(oc),
                                _ptr(op), _ptr(uv), ctypes.byref(K), _ptr(m), _ptr(X),
                                _ptr(status), BA_MEM_HOST))
    return X, status


def options_for_scene(scene, precision: Optional[str] = None, **kw) -> Options:
    """Solver options from a scene's solve settings."""
    prec = precision or scene.precision
    o = ba_options_default()
    o.precision = BA_FP32 if prec == "fp32" else BA_FP64
    o.solver = {"dense": BA_SOLVER_DENSE, "pcg": BA_SOLVER_PCG}.get(scene.solver, BA_SOLVER_AUTO)
    o.max_lm_iters = scene.lm_iters
    o.huber_delta = scene.huber_delta
    o.pcg_tol = scene.pcg_tol
    o.pcg_max_iters = scene.pcg_max_iters
    o.refine = 1 if scene.refine else 0
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def solve_scene(scene, precision: Optional[str] = None, use_torch: bool = False, **kw):
    """Load a scene, solve it, return (report dict, cam_qt, pts)."""
    with ba_create(options_for_scene(scene, precision, **kw), use_torch=use_torch) as h:
        ba_set_problem(h, scene.cam_qt, scene.pts, scene.obs_cam, scene.obs_pt, scene.obs_uv,
                       scene.intrinsics(), scene.cam_fixed)
        rep = ba_solve(h)
        q, p = ba_get_state(h, scene.n_cams, scene.n_pts)
    return rep, q, p
