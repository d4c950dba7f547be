"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no Jacobi arithmetic: only the problem data (boundary values
and initial interior), the workload shapes (grid sizes, request arrivals) and
the counter-based random generator they are drawn from.  The CUDA library
implements the same generator and boundary formula again in its own init
kernel; tests check the two bit for bit.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator.  The n-th output (n = 0, 1, ...) of a stream seeded with `seed` is
``mix(seed + (n + 1) * GAMMA)`` modulo 2^64, with GAMMA = 0x9E3779B97F4A7C15
and ``mix`` the generator's output finaliser (two xor-shift-multiply rounds
and a final xor-shift).  A uniform double in [0, 1) is ``(x >> 11) * 2^-53``.

Grid values are keyed by the GLOBAL padded linear index
``(k * (ny + 2) + j) * (nx + 2) + i`` so that the data never depends on how the
grid is split into blocks.

Boundary functions (the paper gives none; these are the synthetic problems):
  * ``linear``:       g = (x + 2y) + 3z with x = i / (nx + 1) etc. (unit cube,
                      node-centred).  A linear function is harmonic for the
                      7-point Laplacian, so g is an exact discrete fixed point.
  * ``linear_noise``: g + noise_amp * U(bc_seed, idx).
  * ``uniform``:      U(bc_seed, idx).
Every product and sum above is rounded separately in FP64 (no fused
multiply-add); an FP32 state takes the FP64 value rounded to nearest.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = 2.0 ** -53

BC_LINEAR, BC_LINEAR_NOISE, BC_UNIFORM = 0, 1, 2
BC_NAMES = {"linear": BC_LINEAR, "linear_noise": BC_LINEAR_NOISE, "uniform": BC_UNIFORM}


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n) -> np.ndarray:
    """n-th output (0-based; array or scalar) of SplitMix64 seeded with `seed`."""
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (n + np.uint64(1)) * GAMMA
    return splitmix64_mix(state)


def u01(seed: int, n) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of the n-th output times 2^-53."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * _TWO_M53


def padded_index(nx: int, ny: int, nz: int) -> np.ndarray:
    """Global padded linear index of every point, shape (nz+2, ny+2, nx+2)."""
    return np.arange((nz + 2) * (ny + 2) * (nx + 2), dtype=np.uint64).reshape(nz + 2, ny + 2, nx + 2)


def coordinates(nx: int, ny: int, nz: int):
    """Node coordinates x_i = i / (nx + 1) (IEEE FP64 division), likewise y, z."""
    x = np.arange(nx + 2, dtype=np.float64) / np.float64(nx + 1)
    y = np.arange(ny + 2, dtype=np.float64) / np.float64(ny + 1)
    z = np.arange(nz + 2, dtype=np.float64) / np.float64(nz + 1)
    return x, y, z


def linear_function(nx: int, ny: int, nz: int) -> np.ndarray:
    """g = (x + 2y) + 3z on the padded node grid, each operation rounded."""
    x, y, z = coordinates(nx, ny, nz)
    two_y = 2.0 * y
    three_z = 3.0 * z
    xy = x[None, None, :] + two_y[None, :, None]
    return xy + three_z[:, None, None]


def boundary_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    m = np.zeros((nz + 2, ny + 2, nx + 2), dtype=bool)
    m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = (True,) * 6
    return m


def initial_grid(nx: int, ny: int, nz: int, bc: str = "linear", bc_seed: int = 0,
                 interior: str = "zero", interior_seed: int = 0, noise_amp: float = 1e-3,
                 dtype=np.float64) -> np.ndarray:
    """Padded initial grid (nz+2, ny+2, nx+2): Dirichlet boundary + interior."""
    idx = padded_index(nx, ny, nz)
    if bc == "linear":
        g = linear_function(nx, ny, nz)
    elif bc == "linear_noise":
        noise = np.float64(noise_amp) * u01(bc_seed, idx)
        g = linear_function(nx, ny, nz) + noise
    elif bc == "uniform":
        g = u01(bc_seed, idx)
    else:
        raise ValueError(bc)
    if interior == "zero":
        inner = np.zeros_like(g)
    elif interior == "uniform":
        inner = u01(interior_seed, idx)
    elif interior == "bc":
        inner = g.copy()
    else:
        raise ValueError(interior)
    out = np.where(boundary_mask(nx, ny, nz), g, inner)
    return np.ascontiguousarray(out.astype(dtype))


def interior_of(u: np.ndarray) -> np.ndarray:
    return u[1:-1, 1:-1, 1:-1]


# ---------------------------------------------------------------------------
# Workload shapes (sizes, seeds and arrival processes of the synthetic runs).
# ---------------------------------------------------------------------------

# 3D 7-point Jacobi workloads.  `split` is ("count", (px, py, pz)) or
# ("shape", (bx, by, bz)).
WORKLOADS = {
    "jacobi3d-fp64-64c-2x2x2": dict(grid=(64, 64, 64), split=("count", (2, 2, 2)), dtype="f64",
                                    bc="linear", bc_seed=0, interior="uniform", interior_seed=0,
                                    iters=100),
    "jacobi3d-fp64-512c-8x8x8": dict(grid=(512, 512, 512), split=("count", (8, 8, 8)), dtype="f64",
                                     bc="uniform", bc_seed=1, interior="zero", interior_seed=0,
                                     iters=1000),
    # One GPU's share of the paper's weak-scaling base problem (1536^3 doubles on
    # a node of six GPUs, Sec. 4.3), overdecomposed into 64^3 blocks.
    "jacobi3d-fp64-1536x768x512": dict(grid=(1536, 768, 512), split=("shape", (64, 64, 64)), dtype="f64",
                                       bc="uniform", bc_seed=1, interior="zero", interior_seed=0, iters=100),
    # 256^3 versions of the two above: small cases for profiler captures
    # (two 134 MB FP64 state copies, still larger than L2).
    "jacobi3d-fp64-256c-4x4x4": dict(grid=(256, 256, 256), split=("count", (4, 4, 4)), dtype="f64",
                                     bc="uniform", bc_seed=1, interior="zero", interior_seed=0,
                                     iters=20),
    "jacobi3d-fp32-256c-4x4x4": dict(grid=(256, 256, 256), split=("count", (4, 4, 4)), dtype="f32",
                                     bc="linear_noise", bc_seed=3, noise_amp=1e-3,
                                     interior="zero", interior_seed=0, iters=20),
    "jacobi3d-fp32-768c-12x12x12": dict(grid=(768, 768, 768), split=("count", (12, 12, 12)),
                                        dtype="f32", bc="linear_noise", bc_seed=3, noise_amp=1e-3,
                                        interior="zero", interior_seed=0, tol=1e-6, iters=200),
}


# Batched workloads: `n_grids` independent grids with sides drawn by
# batched_sides(), each split into blocks of `block` (partial edge blocks).
BATCHED = {
    "jacobi3d-batched256-fp32": dict(n_grids=256, sides_seed=2, block=(32, 32, 32), dtype="f32", bc="uniform",
                                     interior="zero", iters=500),
    "jacobi3d-batched256-fp64": dict(n_grids=256, sides_seed=2, block=(32, 32, 32), dtype="f64", bc="uniform",
                                     interior="zero", iters=500),
    # the first 32 grids of the batch: a small case for profiler captures
    "jacobi3d-batched32-fp32": dict(n_grids=32, sides_seed=2, block=(32, 32, 32), dtype="f32", bc="uniform",
                                    interior="zero", iters=20),
}


def workload_grids(name: str):
    """(grids, splits, inits, dtype, iters) of a named workload (single or batched)."""
    if name in WORKLOADS:
        w = WORKLOADS[name]
        init = dict(bc=w["bc"], bc_seed=w["bc_seed"], interior=w["interior"], interior_seed=w["interior_seed"])
        if "noise_amp" in w:
            init["noise_amp"] = w["noise_amp"]
        return [w["grid"]], [w["split"]], [init], w["dtype"], w["iters"]
    b = BATCHED[name]
    sides = batched_sides(b["n_grids"], b["sides_seed"])
    inits = [dict(bc=b["bc"], bc_seed=batched_seed(g, b["sides_seed"]), interior=b["interior"])
             for g in range(b["n_grids"])]
    return sides, [("shape", b["block"])] * b["n_grids"], inits, b["dtype"], b["iters"]


def batched_sides(n_grids: int = 256, seed: int = 2):
    """Per-grid (nx, ny, nz), each side uniform over {16, 32, ..., 192}."""
    u = u01(seed, np.arange(3 * n_grids, dtype=np.uint64)).reshape(n_grids, 3)
    sides = 16 * (1 + np.floor(u * 12.0).astype(np.int64))
    return [tuple(int(s) for s in row) for row in sides]


def batched_seed(grid_id: int, seed: int = 2) -> int:
    return (seed << 32) | grid_id


def serving_requests(n: int = 10000, arrival_seed: int = 5, size_seed: int = 6,
                     mean_interarrival_ms: float = 2.0, mu: float = math.log(64.0),
                     sigma: float = 0.5, lo: int = 32, hi: int = 256):
    """Poisson arrivals (exponential gaps) and lognormal sides clipped to [lo, hi].

    Returns a list of dicts: arrival time (s), grid (nx, ny, nz), seed.
    Normal deviates come from the Box-Muller transform of two uniforms.
    """
    ua = u01(arrival_seed, np.arange(n, dtype=np.uint64))
    gaps = -mean_interarrival_ms * 1e-3 * np.log1p(-ua)
    t = np.cumsum(gaps)
    us = u01(size_seed, np.arange(6 * n, dtype=np.uint64)).reshape(n, 3, 2)
    zn = np.sqrt(-2.0 * np.log1p(-us[..., 0])) * np.cos(2.0 * np.pi * us[..., 1])
    sides = np.clip(np.rint(np.exp(mu + sigma * zn)), lo, hi).astype(np.int64)
    return [dict(arrival_s=float(t[r]), grid=tuple(int(s) for s in sides[r]), seed=1000 + r)
            for r in range(n)]
