"""CPU oracle for the 3D 7-point Jacobi hot path (paper Sec. 4.3).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
(``__graft_entry__.smoke``) and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with the CUDA library and never imports it;
the only module both sides use is ``jacobi_inputs`` (seeded input generators,
none of the method's arithmetic).

Contents
  * ``jacobi`` / ``residual`` / ``solve``: thin ctypes wrappers over
    ``oracle.c`` (monolithic padded-array Jacobi in FP64, or FP32 state with
    an FP64 residual), built by ``build()`` with gcc ``-O2 -ffp-contract=off``.
  * ``block_extents`` / ``decompose`` / ``faces``: the plain definitions of
    the block split (Sec. 4.3: equal-size cuboid blocks chosen to minimise
    surface area) and of a block's six halo faces (the data a block sends to
    its up-to-six neighbours each iteration, Sec. 4.3), written out with
    Python loops and numpy slicing.

Pins (tests/test_oracle_pins.py): linear fixed point, eigenmode decay in closed
form, brute-force dense iteration and direct solve on 4^3 / 4x3x5, the closed
form of the residual norm, mirror symmetry and thread-count invariance.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

CONVERGED, MAX_ITERS, STAGNATED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, p, d = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
            pd = ctypes.POINTER(ctypes.c_double)
            pi64 = ctypes.POINTER(ctypes.c_int64)
            pint = ctypes.POINTER(ctypes.c_int)
            for t in ("f64", "f32"):
                getattr(lib, f"oracle_jacobi_{t}").argtypes = [i64, i64, i64, p, i64]
                getattr(lib, f"oracle_residual_{t}").argtypes = [i64, i64, i64, p, pd, pd]
                getattr(lib, f"oracle_solve_{t}").argtypes = [
                    i64, i64, i64, p, d, i64, i64, i64, pi64, pd, pint]
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _suffix(u: np.ndarray) -> str:
    if u.dtype == np.float64:
        return "f64"
    if u.dtype == np.float32:
        return "f32"
    raise TypeError(f"oracle supports float64 / float32 states, got {u.dtype}")


def _check(u: np.ndarray):
    if u.ndim != 3 or min(u.shape) < 3 or not u.flags.c_contiguous:
        raise ValueError("expected a C-contiguous padded (nz+2, ny+2, nx+2) array")
    nz, ny, nx = (s - 2 for s in u.shape)
    return nx, ny, nz


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def threads() -> int:
    return int(_load().oracle_threads())


def jacobi(u: np.ndarray, n_iters: int) -> np.ndarray:
    """Return u after n_iters Jacobi sweeps (Sec. 4.3); u is not modified."""
    nx, ny, nz = _check(u)
    out = np.array(u, copy=True, order="C")
    rc = getattr(_load(), f"oracle_jacobi_{_suffix(u)}")(nx, ny, nz, out.ctypes.data, int(n_iters))
    if rc:
        raise MemoryError("oracle_jacobi: allocation failed")
    return out


def residual(u: np.ndarray):
    """Return (|b - A u|_2, |b|_2, relative residual) in FP64."""
    nx, ny, nz = _check(u)
    rn, bn = ctypes.c_double(), ctypes.c_double()
    rc = getattr(_load(), f"oracle_residual_{_suffix(u)}")(
        nx, ny, nz, u.ctypes.data, ctypes.byref(rn), ctypes.byref(bn))
    if rc:
        raise MemoryError("oracle_residual: allocation failed")
    rel = rn.value / bn.value if bn.value > 0 else rn.value
    return rn.value, bn.value, rel


def solve(u: np.ndarray, tol: float, max_iters: int, check_every: int, stall_checks: int = 0):
    """Jacobi until rel <= tol; returns (u_k, k, rel(u_k), status)."""
    nx, ny, nz = _check(u)
    out = np.array(u, copy=True, order="C")
    it, rel, st = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int()
    rc = getattr(_load(), f"oracle_solve_{_suffix(u)}")(
        nx, ny, nz, out.ctypes.data, float(tol), int(max_iters), int(check_every),
        int(stall_checks), ctypes.byref(it), ctypes.byref(rel), ctypes.byref(st))
    if rc:
        raise ValueError("oracle_solve failed (bad arguments or allocation)")
    return out, it.value, rel.value, st.value


# ---------------------------------------------------------------------------
# Block decomposition and halo faces: plain definitions (Sec. 4.3).
# ---------------------------------------------------------------------------

def block_extents(n: int, mode: str, param: int):
    """Per-axis (origin, extent) list.

    mode "shape": blocks of `param` points, the last one partial.
    mode "count": `param` blocks; the first n % param get one extra point.
    """
    if n < 1 or param < 1:
        raise ValueError("sizes must be positive")
    if mode == "shape":
        out, o = [], 0
        while o < n:
            out.append((o, min(param, n - o)))
            o += param
        return out
    if mode == "count":
        if param > n:
            raise ValueError("more blocks than points")
        q, r = divmod(n, param)
        out, o = [], 0
        for b in range(param):
            e = q + (1 if b < r else 0)
            out.append((o, e))
            o += e
        return out
    raise ValueError(mode)


def decompose(grid, nblocks: int):
    """Block counts (px, py, pz) with px*py*pz == nblocks and p <= n per axis
    that minimise the total block surface 2*sum_b(ab + bc + ca) of the
    split into near-equal cuboids; among equal surfaces the lexicographically
    smallest (px, py, pz) is taken.  Brute force over all factor triples."""
    nx, ny, nz = grid
    best = None
    for px in range(1, nblocks + 1):
        if nblocks % px:
            continue
        for py in range(1, nblocks // px + 1):
            if (nblocks // px) % py:
                continue
            pz = nblocks // (px * py)
            if px > nx or py > ny or pz > nz:
                continue
            area = 0
            for (_, ex), (_, ey), (_, ez) in itertools.product(
                    block_extents(nx, "count", px), block_extents(ny, "count", py),
                    block_extents(nz, "count", pz)):
                area += 2 * (ex * ey + ey * ez + ez * ex)
            key = (area, px, py, pz)
            if best is None or key < best:
                best = key
    if best is None:
        raise ValueError("no decomposition fits the grid")
    return best[1:]


FACE_NAMES = ("xm", "xp", "ym", "yp", "zm", "zp")


def faces(block: np.ndarray):
    """The six boundary planes of a block interior (nz, ny, nx), as sent to the
    neighbours: x-faces laid out (z, y), y-faces (z, x), z-faces (y, x)."""
    return {
        "xm": np.ascontiguousarray(block[:, :, 0]),
        "xp": np.ascontiguousarray(block[:, :, -1]),
        "ym": np.ascontiguousarray(block[:, 0, :]),
        "yp": np.ascontiguousarray(block[:, -1, :]),
        "zm": np.ascontiguousarray(block[0, :, :]),
        "zp": np.ascontiguousarray(block[-1, :, :]),
    }
