"""Python binding of the GB300 Jacobi3D library (``include/jacobi.h``).

Argument marshalling only: every call goes through ctypes into
``_build/libjacobi_gb300.so``, whose CUDA kernels (sm_103a) do all the work.
There is no CPU fallback; loading fails loudly when the library is not built.

The module exposes the C functions under their C names (``jacobi_create``,
``jacobi_step``, ``channel_send``, ...), raising :class:`JacobiError` on a
non-zero status, plus a small convenience wrapper :class:`Jacobi3D`.
Device buffers are passed as integers (e.g. ``tensor.data_ptr()``); streams as
integers, ``torch.cuda.Stream`` objects or ``None`` (legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

c_int32, c_int64, c_uint32, c_uint64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
c_double, c_size_t, c_void_p = ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p

JACOBI_OK, JACOBI_EINVAL, JACOBI_ENOMEM, JACOBI_EBUSY, JACOBI_EAGAIN = 0, 1, 2, 3, 4
JACOBI_ETIMEDOUT, JACOBI_ECUDA, JACOBI_ESEQ = 5, 6, 7
JACOBI_F64, JACOBI_F32 = 0, 1
JACOBI_BC_LINEAR, JACOBI_BC_LINEAR_NOISE, JACOBI_BC_UNIFORM = 0, 1, 2
JACOBI_INTERIOR_ZERO, JACOBI_INTERIOR_UNIFORM, JACOBI_INTERIOR_BC = 0, 1, 2
JACOBI_SPLIT_COUNT, JACOBI_SPLIT_SHAPE = 0, 1
JACOBI_PATH_FUSED, JACOBI_PATH_EXPLICIT, JACOBI_PATH_PERSISTENT, JACOBI_PATH_GRAPH = 0, 1, 2, 3
JACOBI_PATH_CHANNEL, JACOBI_PATH_MESSAGING, JACOBI_PATH_HOST_STAGED = 4, 5, 6
JACOBI_SOLVE_CONVERGED, JACOBI_SOLVE_MAX_ITERS, JACOBI_SOLVE_STAGNATED = 0, 1, 2
JACOBI_LAYOUT_INTERIOR, JACOBI_LAYOUT_PADDED = 0, 1
JACOBI_MAX_BLOCK_EXTENT = 32764
FACES = ("xm", "xp", "ym", "yp", "zm", "zp")

PATHS = {"fused": JACOBI_PATH_FUSED, "explicit": JACOBI_PATH_EXPLICIT,
         "persistent": JACOBI_PATH_PERSISTENT, "graph": JACOBI_PATH_GRAPH,
         "channel": JACOBI_PATH_CHANNEL, "messaging": JACOBI_PATH_MESSAGING,
         "host_staged": JACOBI_PATH_HOST_STAGED}
PATH_NAMES = {v: k for k, v in PATHS.items()}
DTYPES = {"f64": JACOBI_F64, "f32": JACOBI_F32}
NP_DTYPES = {JACOBI_F64: np.float64, JACOBI_F32: np.float32}
BCS = {"linear": JACOBI_BC_LINEAR, "linear_noise": JACOBI_BC_LINEAR_NOISE, "uniform": JACOBI_BC_UNIFORM}
INTERIORS = {"zero": JACOBI_INTERIOR_ZERO, "uniform": JACOBI_INTERIOR_UNIFORM, "bc": JACOBI_INTERIOR_BC}


class jacobi_dim3(ctypes.Structure):
    _fields_ = [("nx", c_int64), ("ny", c_int64), ("nz", c_int64)]


class jacobi_split(ctypes.Structure):
    _fields_ = [("mode", c_int32), ("pad_", c_int32), ("x", c_int64), ("y", c_int64), ("z", c_int64)]


class jacobi_init(ctypes.Structure):
    _fields_ = [("bc", c_int32), ("interior", c_int32), ("bc_seed", c_uint64),
                ("interior_seed", c_uint64), ("noise_amp", c_double)]


class jacobi_block_info(ctypes.Structure):
    _fields_ = [("grid", c_int64), ("origin", c_int64 * 3), ("extent", c_int64 * 3),
                ("neighbour", c_int64 * 6)]


class jacobi_info_t(ctypes.Structure):
    _fields_ = [("n_grids", c_int64), ("n_blocks", c_int64), ("n_points", c_int64),
                ("iteration", c_int64), ("dtype", c_int32), ("path", c_int32),
                ("halo_bytes_per_iter", c_int64), ("workspace_bytes", c_size_t), ("stages", c_int32),
                ("item_kinds", c_int32), ("fp64_int_adds", c_int32), ("pad_", c_int32),
                ("kind_items", c_int32 * 8), ("zchunk", c_int64), ("cw_cap", c_int32), ("pad2_", c_int32)]


class jacobi_tune_result(ctypes.Structure):
    _fields_ = [("path", c_int32), ("stages", c_int32), ("ms_per_iter", c_double), ("n_tried", c_int32),
                ("from_cache", c_int32), ("zchunk", c_int64), ("cw_cap", c_int32), ("pad_", c_int32)]


class serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_uint64), ("max_slots", c_int32), ("dtype", c_int32),
                ("check_every", c_int32), ("round_checks", c_int32), ("stall_checks", c_int64)]


class serve_request(ctypes.Structure):
    _fields_ = [("grid", jacobi_dim3), ("split", jacobi_split), ("init", jacobi_init), ("tol", c_double),
                ("max_iters", c_int64), ("out", c_void_p)]


class serve_result(ctypes.Structure):
    _fields_ = [("status", c_int32), ("pad_", c_int32), ("iters", c_int64), ("rel", c_double),
                ("t_arrive_ns", c_int64), ("t_admit_ns", c_int64), ("t_done_ns", c_int64)]


class serve_stats_t(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("admitted", c_int64), ("completed", c_int64), ("queued", c_int64),
                ("running", c_int64), ("rounds", c_int64), ("iterations", c_int64), ("bytes_in_use", c_uint64),
                ("lups", c_int64)]


class JacobiError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func}: {msg} (code {code})")
        self.code = code


_lib = None
_lock = threading.Lock()

P = c_void_p
_SIGS = {
    "jacobi_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "jacobi_last_error": (ctypes.c_char_p, []),
    "jacobi_decompose": (ctypes.c_int, [jacobi_dim3, c_int64, ctypes.POINTER(jacobi_dim3)]),
    "jacobi_workspace_bytes": (ctypes.c_int, [jacobi_dim3, jacobi_split, ctypes.c_int, ctypes.POINTER(c_size_t)]),
    "jacobi_workspace_bytes_batch": (ctypes.c_int, [c_int64, P, P, ctypes.c_int, ctypes.POINTER(c_size_t)]),
    "jacobi_create": (ctypes.c_int, [jacobi_dim3, jacobi_split, ctypes.c_int, P, P, c_size_t, P, ctypes.POINTER(P)]),
    "jacobi_create_batch": (ctypes.c_int, [c_int64, P, P, ctypes.c_int, P, P, c_size_t, P, ctypes.POINTER(P)]),
    "jacobi_destroy": (ctypes.c_int, [P]),
    "jacobi_info": (ctypes.c_int, [P, ctypes.POINTER(jacobi_info_t)]),
    "jacobi_block": (ctypes.c_int, [P, c_int64, ctypes.POINTER(jacobi_block_info)]),
    "jacobi_set_path": (ctypes.c_int, [P, c_int32]),
    "jacobi_set_state": (ctypes.c_int, [P, c_int64, P, c_int32, P]),
    "jacobi_copy_out": (ctypes.c_int, [P, c_int64, P, c_int32, c_int32, P]),
    "jacobi_step": (ctypes.c_int, [P, c_int64, P]),
    "jacobi_residual": (ctypes.c_int, [P, P, P, P]),
    "jacobi_step_timed": (ctypes.c_int, [P, c_int64, P, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "jacobi_solve": (ctypes.c_int, [P, c_double, c_int64, c_int64, c_int64, P, P, P, P]),
    "jacobi_sync": (ctypes.c_int, [P, P]),
    "jacobi_autotune": (ctypes.c_int, [P, c_int64, P, ctypes.POINTER(jacobi_tune_result)]),
    "jacobi_autotune_path": (ctypes.c_int, [P, c_int32, c_int64, P, ctypes.POINTER(jacobi_tune_result)]),
    "jacobi_set_shape": (ctypes.c_int, [P, c_int64, c_int32, P]),
    "jacobi_read_face": (ctypes.c_int, [P, c_int64, c_int32, P, P]),
    "jacobi_debug_drop_block": (ctypes.c_int, [P, c_int64]),
    "jacobi_measure_local_halo": (ctypes.c_int, [P, c_int32]),
    "jacobi_selftest_dadd": (ctypes.c_int, [P, P, c_int64, P, P]),
    "jacobi_selftest_widen": (ctypes.c_int, [P, P]),
    "jacobi_selftest_div6": (ctypes.c_int, [P, P]),
    "jacobi_pipe_rates": (ctypes.c_int, [ctypes.POINTER(c_double), ctypes.POINTER(c_double), P]),
    "jacobi_residual_noalloc": (ctypes.c_int, [P, jacobi_dim3, ctypes.c_int, P, P]),
    "channel_open": (ctypes.c_int, [P, c_uint32, c_int64, c_int64, c_size_t, ctypes.POINTER(P)]),
    "channel_send": (ctypes.c_int, [P, c_int64, P, c_size_t, P]),
    "channel_recv": (ctypes.c_int, [P, c_int64, P, c_size_t, P]),
    "channel_slot": (ctypes.c_int, [P, c_int64, c_int32, ctypes.POINTER(P)]),
    "channel_release": (ctypes.c_int, [P, c_int64, P]),
    "channel_sync": (ctypes.c_int, [P, P]),
    "channel_pingpong": (ctypes.c_int, [P, c_size_t, c_int64, c_int32, P]),
    "channel_close": (ctypes.c_int, [P]),
    "channel_bandwidth": (ctypes.c_int, [P, c_size_t, c_int32, c_int64, c_int32, c_int32, P]),
    "channel_send_host": (ctypes.c_int, [P, c_int64, P, c_size_t, P]),
    "channel_recv_host": (ctypes.c_int, [P, c_int64, P, c_size_t, P]),
    "channel_send_msg": (ctypes.c_int, [P, c_int64, P, c_size_t, P]),
    "channel_recv_msg": (ctypes.c_int, [P, c_int64, P, c_size_t, P]),
    "serve_create": (ctypes.c_int, [ctypes.POINTER(serve_config), ctypes.POINTER(P)]),
    "serve_submit": (ctypes.c_int, [P, ctypes.POINTER(serve_request), ctypes.POINTER(c_uint64)]),
    "serve_poll": (ctypes.c_int, [P, c_uint64, ctypes.POINTER(serve_result)]),
    "serve_stats": (ctypes.c_int, [P, ctypes.POINTER(serve_stats_t)]),
    "serve_destroy": (ctypes.c_int, [P]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the compiled library (ctypes.CDLL).  Raises if it is not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                if not build_if_missing:
                    raise RuntimeError(
                        "the CUDA library is not built (run __graft_entry__.build() or "
                        "python -m paper_2102_12416_gb300._build); there is no CPU fallback")
                _build.build()
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _stream(s) -> int | None:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    return int(s)


def _check(rc: int, func: str):
    if rc != 0:
        msg = load().jacobi_last_error().decode(errors="replace")
        raise JacobiError(rc, func, msg or load().jacobi_strerror(rc).decode())


def _call(name, *args):
    rc = getattr(load(), name)(*args)
    _check(rc, name)


def _mk_split(split) -> jacobi_split:
    mode, (x, y, z) = split
    return jacobi_split(JACOBI_SPLIT_COUNT if mode == "count" else JACOBI_SPLIT_SHAPE, 0, x, y, z)


def _mk_init(init: dict | None) -> jacobi_init:
    init = dict(init or {})
    return jacobi_init(BCS[init.get("bc", "linear")], INTERIORS[init.get("interior", "zero")],
                       int(init.get("bc_seed", 0)) & 0xFFFFFFFFFFFFFFFF,
                       int(init.get("interior_seed", 0)) & 0xFFFFFFFFFFFFFFFF,
                       float(init.get("noise_amp", 0.0)))


# ---- the C functions under their own names -----------------------------------

def jacobi_strerror(code: int) -> str:
    return load().jacobi_strerror(code).decode()


def jacobi_last_error() -> str:
    return load().jacobi_last_error().decode(errors="replace")


def jacobi_decompose(grid, nblocks: int):
    out = jacobi_dim3()
    _call("jacobi_decompose", jacobi_dim3(*grid), nblocks, ctypes.byref(out))
    return (out.nx, out.ny, out.nz)


def jacobi_workspace_bytes(grid, split, dtype="f64") -> int:
    out = c_size_t()
    _call("jacobi_workspace_bytes", jacobi_dim3(*grid), _mk_split(split), DTYPES[dtype], ctypes.byref(out))
    return out.value


def jacobi_workspace_bytes_batch(grids, splits, dtype="f64") -> int:
    n = len(grids)
    g = (jacobi_dim3 * n)(*[jacobi_dim3(*x) for x in grids])
    s = (jacobi_split * n)(*[_mk_split(x) for x in splits])
    out = c_size_t()
    _call("jacobi_workspace_bytes_batch", n, ctypes.cast(g, P), ctypes.cast(s, P), DTYPES[dtype], ctypes.byref(out))
    return out.value


def jacobi_create_batch(grids, splits, dtype="f64", inits=None, workspace=None, ws_bytes=0, stream=None) -> int:
    n = len(grids)
    g = (jacobi_dim3 * n)(*[jacobi_dim3(*x) for x in grids])
    s = (jacobi_split * n)(*[_mk_split(x) for x in splits])
    ini = (jacobi_init * n)(*[_mk_init(inits[q] if inits else None) for q in range(n)])
    h = P()
    _call("jacobi_create_batch", n, ctypes.cast(g, P), ctypes.cast(s, P), DTYPES[dtype], ctypes.cast(ini, P),
          workspace, ws_bytes, _stream(stream), ctypes.byref(h))
    return h.value


def jacobi_create(grid, split, dtype="f64", init=None, workspace=None, ws_bytes=0, stream=None) -> int:
    return jacobi_create_batch([grid], [split], dtype, [init] if init else None, workspace, ws_bytes, stream)


def jacobi_destroy(h):
    _call("jacobi_destroy", h)


def jacobi_info(h) -> jacobi_info_t:
    out = jacobi_info_t()
    _call("jacobi_info", h, ctypes.byref(out))
    return out


def jacobi_block(h, b) -> jacobi_block_info:
    out = jacobi_block_info()
    _call("jacobi_block", h, b, ctypes.byref(out))
    return out


def jacobi_set_path(h, path):
    _call("jacobi_set_path", h, PATHS[path] if isinstance(path, str) else int(path))


def jacobi_set_state(h, grid, src, src_on_device=False, stream=None):
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src)
        _call("jacobi_set_state", h, grid, src.ctypes.data, 0, _stream(stream))
    else:
        _call("jacobi_set_state", h, grid, int(src), 1 if src_on_device else 0, _stream(stream))


def jacobi_copy_out(h, grid, dst, dst_on_device=False, layout=JACOBI_LAYOUT_INTERIOR, stream=None):
    if isinstance(dst, np.ndarray):
        assert dst.flags.c_contiguous
        _call("jacobi_copy_out", h, grid, dst.ctypes.data, 0, layout, _stream(stream))
    else:
        _call("jacobi_copy_out", h, grid, int(dst), 1 if dst_on_device else 0, layout, _stream(stream))


def jacobi_step(h, n_iters, stream=None):
    _call("jacobi_step", h, n_iters, _stream(stream))


def jacobi_step_timed(h, n_iters, stream=None):
    """(compute_ms, exchange_ms) summed over n_iters iterations (see include/jacobi.h)."""
    a, b = c_double(), c_double()
    _call("jacobi_step_timed", h, n_iters, _stream(stream), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def jacobi_residual(h, n_grids, stream=None):
    rel = (c_double * n_grids)()
    ab = (c_double * n_grids)()
    _call("jacobi_residual", h, ctypes.cast(rel, P), ctypes.cast(ab, P), _stream(stream))
    return list(rel), list(ab)


def jacobi_solve(h, n_grids, tol, max_iters, check_every, stall_checks=0, stream=None):
    it = (c_int64 * n_grids)()
    rel = (c_double * n_grids)()
    st = (c_int32 * n_grids)()
    _call("jacobi_solve", h, tol, max_iters, check_every, stall_checks, ctypes.cast(it, P), ctypes.cast(rel, P),
          ctypes.cast(st, P), _stream(stream))
    return list(it), list(rel), list(st)


def jacobi_autotune(h, iters_per_trial, stream=None) -> jacobi_tune_result:
    out = jacobi_tune_result()
    _call("jacobi_autotune", h, iters_per_trial, _stream(stream), ctypes.byref(out))
    return out


def jacobi_autotune_path(h, path, iters_per_trial, stream=None) -> jacobi_tune_result:
    """The autotuner's search restricted to one path ("fused", "graph" or
    "persistent" or its jacobi_path value)."""
    out = jacobi_tune_result()
    _call("jacobi_autotune_path", h, PATHS[path] if isinstance(path, str) else int(path), iters_per_trial,
          _stream(stream), ctypes.byref(out))
    return out


def jacobi_set_shape(h, zchunk=0, cw_cap=8, stream=None):
    _call("jacobi_set_shape", h, zchunk, cw_cap, _stream(stream))


def jacobi_sync(h, stream=None):
    _call("jacobi_sync", h, _stream(stream))


def jacobi_read_face(h, block, face, dst: np.ndarray, stream=None):
    _call("jacobi_read_face", h, block, face, dst.ctypes.data, _stream(stream))


def jacobi_selftest_dadd(a_dev, b_dev, n, out_dev, stream=None):
    _call("jacobi_selftest_dadd", int(a_dev), int(b_dev), n, int(out_dev), _stream(stream))


def jacobi_selftest_widen(stream=None):
    """Number of binary32 inputs whose integer-pipe widening differs from the
    conversion instruction (all 2^32 bit patterns, on the device)."""
    n = ctypes.c_uint64(0)
    _call("jacobi_selftest_widen", ctypes.addressof(n), _stream(stream))
    return n.value


def jacobi_selftest_div6(stream=None):
    """Number of binary32 inputs whose FP32-update division RN(s / 6) differs
    from the division instruction sequence (all 2^32 bit patterns, on the device)."""
    n = ctypes.c_uint64(0)
    _call("jacobi_selftest_div6", ctypes.addressof(n), _stream(stream))
    return n.value


def jacobi_pipe_rates(stream=None):
    """(FP64-pipe adds/s, integer-pipe FP64 adds/s) measured on the current GPU."""
    a, b = c_double(), c_double()
    _call("jacobi_pipe_rates", ctypes.byref(a), ctypes.byref(b), _stream(stream))
    return a.value, b.value


def jacobi_measure_local_halo(h, on):
    _call("jacobi_measure_local_halo", h, 1 if on else 0)


def jacobi_debug_drop_block(h, block):
    _call("jacobi_debug_drop_block", h, block)


JACOBI_NOALLOC_MAX_PLANES = 16384


def jacobi_residual_noalloc(u_padded_dev, grid, dtype, out_dev, stream=None):
    """Residual of a device padded array into a device buffer of 3 doubles
    (|r|, |b|, rel); allocates nothing (see include/jacobi.h)."""
    _call("jacobi_residual_noalloc", int(u_padded_dev), jacobi_dim3(*grid), DTYPES[dtype], int(out_dev),
          _stream(stream))


def channel_open(h, channel_id, block_a, block_b, max_bytes) -> int:
    ch = P()
    _call("channel_open", h, channel_id, block_a, block_b, max_bytes, ctypes.byref(ch))
    return ch.value


def channel_send(ch, from_block, src, nbytes, stream=None):
    _call("channel_send", ch, from_block, int(src), nbytes, _stream(stream))


def channel_recv(ch, at_block, dst, nbytes, stream=None):
    _call("channel_recv", ch, at_block, None if dst is None else int(dst), nbytes, _stream(stream))


def channel_release(ch, at_block, stream=None):
    _call("channel_release", ch, at_block, _stream(stream))


def channel_slot(ch, at_block, parity) -> int:
    out = P()
    _call("channel_slot", ch, at_block, parity, ctypes.byref(out))
    return out.value


def channel_sync(ch, stream=None):
    _call("channel_sync", ch, _stream(stream))


def channel_pingpong(ch, nbytes, round_trips, ctas_per_side=1, stream=None):
    _call("channel_pingpong", ch, nbytes, round_trips, ctas_per_side, _stream(stream))


def channel_bandwidth(ch, nbytes, window, iterations, ctas_per_side=1, bidirectional=False, stream=None):
    _call("channel_bandwidth", ch, nbytes, window, iterations, ctas_per_side, 1 if bidirectional else 0,
          _stream(stream))


def channel_send_host(ch, from_block, src, nbytes, stream=None):
    _call("channel_send_host", ch, from_block, int(src), nbytes, _stream(stream))


def channel_recv_host(ch, at_block, dst, nbytes, stream=None):
    _call("channel_recv_host", ch, at_block, int(dst), nbytes, _stream(stream))


def channel_send_msg(ch, from_block, src, nbytes, stream=None):
    _call("channel_send_msg", ch, from_block, int(src), nbytes, _stream(stream))


def channel_recv_msg(ch, at_block, dst, nbytes, stream=None):
    _call("channel_recv_msg", ch, at_block, int(dst), nbytes, _stream(stream))


def channel_close(ch):
    _call("channel_close", ch)


def serve_create(hbm_budget_bytes, max_slots, dtype="f32", check_every=100, round_checks=2, stall_checks=0) -> int:
    cfg = serve_config(int(hbm_budget_bytes), max_slots, DTYPES[dtype], check_every, round_checks, stall_checks)
    s = P()
    _call("serve_create", ctypes.byref(cfg), ctypes.byref(s))
    return s.value


def serve_submit(s, grid, split, init=None, tol=1e-6, max_iters=20000, out=None) -> int:
    """Queue one solve; `out` (optional) is a C-contiguous host array of the
    server's dtype and the grid's interior shape (nz, ny, nx) that receives the
    final iterate before the result is posted.  The caller keeps it alive."""
    req = serve_request(jacobi_dim3(*grid), _mk_split(split), _mk_init(init), float(tol), int(max_iters),
                        None if out is None else out.ctypes.data)
    t = c_uint64()
    _call("serve_submit", s, ctypes.byref(req), ctypes.byref(t))
    return t.value


def serve_poll(s, ticket):
    """The serve_result when done, or None while pending."""
    res = serve_result()
    rc = load().serve_poll(s, ticket, ctypes.byref(res))
    if rc == JACOBI_EAGAIN:
        return None
    _check(rc, "serve_poll")
    return res


def serve_stats(s) -> serve_stats_t:
    out = serve_stats_t()
    _call("serve_stats", s, ctypes.byref(out))
    return out


def serve_destroy(s):
    _call("serve_destroy", s)


# ---- convenience wrapper -----------------------------------------------------

class Jacobi3D:
    """One handle holding one or more grids (see jacobi_create_batch)."""

    def __init__(self, grids, splits, dtype="f64", inits=None, path="fused", stream=None, workspace=None,
                 ws_bytes=0):
        if isinstance(grids, tuple):
            grids, splits, inits = [grids], [splits], ([inits] if inits else None)
        self.grids = [tuple(int(v) for v in g) for g in grids]
        self.dtype = dtype
        self.np_dtype = NP_DTYPES[DTYPES[dtype]]
        self.stream = stream
        self.h = jacobi_create_batch(self.grids, splits, dtype, inits, workspace, ws_bytes, stream)
        self.set_path(path)

    def close(self):
        if self.h:
            jacobi_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self):
        return jacobi_info(self.h)

    def block(self, b):
        return jacobi_block(self.h, b)

    def set_path(self, path):
        jacobi_set_path(self.h, path)

    def step(self, n):
        jacobi_step(self.h, n, self.stream)

    def step_timed(self, n):
        """Advance n iterations; returns (compute_ms, exchange_ms) for the whole call."""
        return jacobi_step_timed(self.h, n, self.stream)

    def sync(self):
        jacobi_sync(self.h, self.stream)

    def autotune(self, iters_per_trial=50, path=None) -> dict:
        """Tune path, ring depth and work-item shape (path given: shape and
        ring depth for that path only) and apply the result."""
        r = (jacobi_autotune(self.h, iters_per_trial, self.stream) if path is None
             else jacobi_autotune_path(self.h, path, iters_per_trial, self.stream))
        return {"path": PATH_NAMES[r.path], "stages": r.stages, "ms_per_iter": r.ms_per_iter,
                "n_tried": r.n_tried, "from_cache": bool(r.from_cache), "zchunk": r.zchunk, "cw_cap": r.cw_cap}

    def set_shape(self, zchunk=0, cw_cap=8):
        jacobi_set_shape(self.h, zchunk, cw_cap, self.stream)

    def launch_kinds(self) -> int:
        return max(1, self.info.item_kinds)

    def kind_items(self) -> dict:
        """Work items per step kernel variant (non-empty ones only)."""
        names = ("tiles", "stream8", "stream4", "stream2", "stream8_ragged", "stream4_ragged", "stream2_ragged")
        ki = self.info.kind_items
        return {n: ki[k] for k, n in enumerate(names) if ki[k]}

    def residual(self):
        return jacobi_residual(self.h, len(self.grids), self.stream)

    def solve(self, tol, max_iters, check_every, stall_checks=0):
        return jacobi_solve(self.h, len(self.grids), tol, max_iters, check_every, stall_checks, self.stream)

    def set_state(self, padded: np.ndarray, grid=0):
        jacobi_set_state(self.h, grid, np.ascontiguousarray(padded, dtype=self.np_dtype), stream=self.stream)

    def copy_out(self, grid=0, padded=False) -> np.ndarray:
        nx, ny, nz = self.grids[grid]
        o = 2 if padded else 0
        out = np.empty((nz + o, ny + o, nx + o), dtype=self.np_dtype)
        jacobi_copy_out(self.h, grid, out, layout=JACOBI_LAYOUT_PADDED if padded else JACOBI_LAYOUT_INTERIOR,
                        stream=self.stream)
        return out

    def read_face(self, block, face) -> np.ndarray:
        bi = self.block(block)
        ex, ey, ez = bi.extent
        shape = {0: (ez, ey), 1: (ez, ey), 2: (ez, ex), 3: (ez, ex), 4: (ey, ex), 5: (ey, ex)}[face]
        out = np.empty(shape, dtype=self.np_dtype)
        jacobi_read_face(self.h, block, face, out, self.stream)
        return out
