"""Pins for the CPU oracle against facts fixed by mathematics, not by the oracle.

Each test is chosen so that a plausible slip in the oracle (a dropped or
doubled neighbour, a wrong coefficient such as 1/7, a swapped axis, a wrong
sign in the residual, an off-by-one in the boundary or the iteration count)
makes at least one of them fail.

The Jacobi iteration is the one the paper's proxy application runs
(Sec. 4.3); the stencil and residual readings are stated in oracle/oracle.c.
"""
import math
import os

import numpy as np
import pytest

import jacobi_inputs as J


def _mode(nx, ny, nz, p, q, s):
    x, y, z = J.coordinates(nx, ny, nz)
    return (np.sin(s * np.pi * z)[:, None, None] * np.sin(q * np.pi * y)[None, :, None]
            * np.sin(p * np.pi * x)[None, None, :])


def _lam(nx, ny, nz, p, q, s):
    return (math.cos(p * math.pi / (nx + 1)) + math.cos(q * math.pi / (ny + 1))
            + math.cos(s * math.pi / (nz + 1))) / 3.0


def _dense_system(u):
    """Dense Jacobi matrix M, offset c and system (A, b) of the padded grid u.

    Built point by point from the definition of the 7-point neighbourhood, with
    no reference to the oracle's code."""
    nz, ny, nx = (d - 2 for d in u.shape)
    n = nx * ny * nz

    def lin(i, j, k):
        return ((k - 1) * ny + (j - 1)) * nx + (i - 1)

    N = np.zeros((n, n))
    bvec = np.zeros(n)
    for k in range(1, nz + 1):
        for j in range(1, ny + 1):
            for i in range(1, nx + 1):
                p = lin(i, j, k)
                for di, dj, dk in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
                    a, b_, c = i + di, j + dj, k + dk
                    if 1 <= a <= nx and 1 <= b_ <= ny and 1 <= c <= nz:
                        N[p, lin(a, b_, c)] += 1.0
                    else:
                        bvec[p] += u[c, b_, a]
    A = 6.0 * np.eye(n) - N
    return N / 6.0, bvec / 6.0, A, bvec


def _interior_vec(u):
    return J.interior_of(u).reshape(-1).copy()


# ---------------------------------------------------------------------------
# Stencil and boundary handling
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 9, 7), (5, 31, 3)])
def test_linear_fixed_point_f64(oracle_mod, shape):
    """x + 2y + 3z is harmonic for the 7-point Laplacian: a discrete fixed point."""
    nx, ny, nz = shape
    g = J.initial_grid(nx, ny, nz, "linear", interior="bc")
    u = oracle_mod.jacobi(g, 100)
    assert np.max(np.abs(u - g)) <= 1e-14
    rn, bn, rel = oracle_mod.residual(u)
    assert rel <= 1e-15 and bn > 1.0


def test_linear_fixed_point_f32(oracle_mod):
    """In FP32 the linear fixed point stays within one ulp of its largest
    values (2^-21 in [4, 8)) and shows no drift on average: each update rounds
    s/6 once, to nearest, so the rounding errors have no preferred sign.
    Multiplying by the float nearest 1/6 instead scales every update by
    1 + 2^-25 and lifts the whole interior (mean error +7.5e-7, 4.5 ulps at
    the top after 2000 iterations on this grid)."""
    g = J.initial_grid(20, 13, 9, "linear", interior="bc", dtype=np.float32)
    for k in (100, 2000):
        d = oracle_mod.jacobi(g, k).astype(np.float64) - g
        assert np.max(np.abs(d)) <= 2.0 ** -21
        assert abs(np.mean(J.interior_of(d))) <= 1e-8


def test_fp32_update_is_nearest_float_to_sum_over_6(oracle_mod):
    """One FP32 sweep rounds once after the float32 neighbour sum s (taken in
    the stated pair order): the new value is the float nearest s/6.  s/6 is
    never halfway between two floats (s = M 2^E with M < 2^24, so s/6 is either
    exact or has a non-terminating binary expansion), hence the nearest float
    is unique and rounding the FP64 quotient to float finds it."""
    u0 = J.initial_grid(9, 7, 6, "uniform", bc_seed=91, interior="uniform", interior_seed=92,
                        dtype=np.float32)
    u1 = oracle_mod.jacobi(u0, 1)
    c = u0
    s = ((c[1:-1, 1:-1, :-2] + c[1:-1, 1:-1, 2:]) + (c[1:-1, :-2, 1:-1] + c[1:-1, 2:, 1:-1])) \
        + (c[:-2, 1:-1, 1:-1] + c[2:, 1:-1, 1:-1])
    assert s.dtype == np.float32
    want = (s.astype(np.float64) / 6.0).astype(np.float32)
    assert np.array_equal(J.interior_of(u1), want)


@pytest.mark.parametrize("shape,mode,k", [((16, 16, 16), (1, 1, 1), 20),
                                           ((20, 12, 9), (2, 1, 3), 8),
                                           ((11, 17, 14), (3, 2, 1), 12)])
def test_eigenmode_decay_closed_form(oracle_mod, shape, mode, k):
    """u0 = g + A*sin(p pi x) sin(q pi y) sin(s pi z) decays as lambda^k exactly,
    lambda = (cos(p pi hx) + cos(q pi hy) + cos(s pi hz)) / 3."""
    nx, ny, nz = shape
    amp = 0.5
    g = J.initial_grid(nx, ny, nz, "linear", interior="bc")
    m = _mode(nx, ny, nz, *mode)
    u0 = g.copy()
    J.interior_of(u0)[...] += amp * J.interior_of(m)
    uk = oracle_mod.jacobi(u0, k)
    lam = _lam(nx, ny, nz, *mode)
    want = lam ** k * amp * J.interior_of(m)
    got = J.interior_of(uk) - J.interior_of(g)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)) + 1e-14


@pytest.mark.parametrize("shape", [(4, 4, 4), (4, 3, 5)])
def test_bruteforce_dense_iteration(oracle_mod, shape):
    """u_{k+1} = M u_k + c with M, c built densely from the neighbourhood."""
    nx, ny, nz = shape
    u0 = J.initial_grid(nx, ny, nz, "uniform", bc_seed=11, interior="uniform", interior_seed=12)
    M, c, _, _ = _dense_system(u0)
    v = _interior_vec(u0)
    for k in range(1, 31):
        v = M @ v + c
        if k in (1, 2, 7, 30):
            got = _interior_vec(oracle_mod.jacobi(u0, k))
            assert np.max(np.abs(got - v)) <= 1e-14


@pytest.mark.parametrize("shape", [(4, 4, 4), (4, 3, 5)])
def test_converged_matches_direct_solve(oracle_mod, shape):
    nx, ny, nz = shape
    u0 = J.initial_grid(nx, ny, nz, "uniform", bc_seed=21, interior="zero")
    _, _, A, b = _dense_system(u0)
    exact = np.linalg.solve(A, b)
    u, iters, rel, st = oracle_mod.solve(u0, 1e-13, 10000, 1)
    assert st == oracle_mod.CONVERGED and rel <= 1e-13 and iters > 10
    assert np.max(np.abs(_interior_vec(u) - exact)) <= 1e-12
    # |b| is the 2-norm of the boundary contribution vector of the dense system.
    _, bn, _ = oracle_mod.residual(u0)
    assert abs(bn - np.linalg.norm(b)) <= 1e-14 * np.linalg.norm(b)


# ---------------------------------------------------------------------------
# Residual
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_residual_eigenmode_closed_form(oracle_mod, dtype):
    """r = b - A u = -6 (1 - lambda) A_m * mode on the interior, so
    |r| = 6 (1 - lambda) |A_m| |mode|."""
    nx, ny, nz = 18, 14, 10
    amp = 0.25
    p, q, s = 2, 1, 1
    g = J.initial_grid(nx, ny, nz, "linear", interior="bc")
    m = _mode(nx, ny, nz, p, q, s)
    u = g.copy()
    J.interior_of(u)[...] += amp * J.interior_of(m)
    u = u.astype(dtype)
    want = 6.0 * (1.0 - _lam(nx, ny, nz, p, q, s)) * amp * np.linalg.norm(J.interior_of(m))
    rn, _, _ = oracle_mod.residual(u)
    tol = 1e-11 if dtype == np.float64 else 2e-5
    assert abs(rn - want) <= tol * want


def test_residual_dense(oracle_mod):
    """|b - A u| against the dense system at a random state."""
    u = J.initial_grid(4, 3, 5, "uniform", bc_seed=31, interior="uniform", interior_seed=32)
    _, _, A, b = _dense_system(u)
    r = b - A @ _interior_vec(u)
    rn, bn, rel = oracle_mod.residual(u)
    assert abs(rn - np.linalg.norm(r)) <= 1e-13 * np.linalg.norm(r)
    assert abs(rel - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-13


# ---------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry_bit_exact(oracle_mod, axis):
    """Mirroring the grid along an axis only swaps the two operands of one
    addition, so the result mirrors bit for bit."""
    u0 = J.initial_grid(13, 10, 7, "uniform", bc_seed=41, interior="uniform", interior_seed=42)
    a = oracle_mod.jacobi(u0, 9)
    b = oracle_mod.jacobi(np.ascontiguousarray(np.flip(u0, axis)), 9)
    assert np.array_equal(np.flip(a, axis), b)


def test_xy_transpose_bit_exact(oracle_mod):
    """Swapping x and y swaps the first two pair sums: bit-exact as well."""
    u0 = J.initial_grid(9, 9, 6, "uniform", bc_seed=43, interior="uniform", interior_seed=44)
    a = oracle_mod.jacobi(u0, 5)
    b = oracle_mod.jacobi(np.ascontiguousarray(np.swapaxes(u0, 1, 2)), 5)
    assert np.array_equal(np.swapaxes(a, 1, 2), b)


def test_thread_count_invariance(oracle_mod):
    u0 = J.initial_grid(40, 33, 29, "uniform", bc_seed=51, interior="uniform", interior_seed=52)
    n = oracle_mod.threads()
    try:
        oracle_mod.set_threads(1)
        a = oracle_mod.jacobi(u0, 7)
        ra = oracle_mod.residual(a)
        oracle_mod.set_threads(max(n, 3))
        b = oracle_mod.jacobi(u0, 7)
        rb = oracle_mod.residual(b)
    finally:
        oracle_mod.set_threads(n)
    assert np.array_equal(a, b) and ra == rb


def test_max_principle(oracle_mod):
    """Jacobi averages: values stay within the range of the initial data."""
    u0 = J.initial_grid(17, 11, 8, "uniform", bc_seed=61, interior="uniform", interior_seed=62)
    u = oracle_mod.jacobi(u0, 25)
    assert u.min() >= u0.min() and u.max() <= u0.max()
    assert np.array_equal(u[0], u0[0]) and np.array_equal(u[:, :, -1], u0[:, :, -1])


# ---------------------------------------------------------------------------
# Solve semantics
# ---------------------------------------------------------------------------

def test_solve_counts_match_closed_form(oracle_mod):
    """With u0 = g + A*mode the relative residual after k steps is
    lambda^k * |r0| / |b|; the first multiple of check_every below tol is known."""
    nx, ny, nz = 12, 12, 12
    g = J.initial_grid(nx, ny, nz, "linear", interior="bc")
    m = _mode(nx, ny, nz, 1, 1, 1)
    u0 = g.copy()
    J.interior_of(u0)[...] += J.interior_of(m)
    r0, bn, rel0 = oracle_mod.residual(u0)
    lam = _lam(nx, ny, nz, 1, 1, 1)
    tol = 1e-7
    check = 5
    kmin = math.ceil(math.log(tol / rel0) / math.log(lam))
    want = check * math.ceil(kmin / check)
    u, iters, rel, st = oracle_mod.solve(u0, tol, 10 ** 6, check)
    assert st == oracle_mod.CONVERGED and iters == want and rel <= tol


def test_solve_cap_and_start_converged(oracle_mod):
    g = J.initial_grid(8, 8, 8, "linear", interior="bc")
    _, iters, rel, st = oracle_mod.solve(g, 1e-12, 100, 10)
    assert (iters, st) == (0, oracle_mod.CONVERGED)
    u0 = J.initial_grid(8, 8, 8, "uniform", bc_seed=1, interior="zero")
    u, iters, rel, st = oracle_mod.solve(u0, 1e-30, 7, 5)
    assert (iters, st) == (7, oracle_mod.MAX_ITERS)
    assert np.array_equal(u, oracle_mod.jacobi(u0, 7))
    assert rel == oracle_mod.residual(u)[2]


def test_solve_fp32_stagnates(oracle_mod):
    """An FP32 state cannot reach a tolerance below its rounding floor."""
    u0 = J.initial_grid(10, 10, 10, "linear_noise", bc_seed=3, interior="zero", dtype=np.float32)
    _, iters, rel, st = oracle_mod.solve(u0, 1e-12, 100000, 10, stall_checks=5)
    assert st == oracle_mod.STAGNATED and rel > 1e-12 and iters < 100000


# ---------------------------------------------------------------------------
# Block split and faces
# ---------------------------------------------------------------------------

def test_decompose_known_answers(oracle_mod):
    assert oracle_mod.decompose((64, 64, 64), 8) == (2, 2, 2)
    assert oracle_mod.decompose((512, 512, 512), 512) == (8, 8, 8)
    assert oracle_mod.decompose((96, 96, 96), 6) == (1, 2, 3)  # minimise px + py + pz
    # Long x axis: cut x first (surface 2*(ny*nz*px + ...)).
    assert oracle_mod.decompose((1024, 64, 64), 8) == (8, 1, 1)
    assert oracle_mod.decompose((1536, 768, 512), 6) == (3, 2, 1)
    with pytest.raises(ValueError):
        oracle_mod.decompose((2, 2, 2), 27)


def test_block_extents(oracle_mod):
    assert oracle_mod.block_extents(100, "shape", 32) == [(0, 32), (32, 32), (64, 32), (96, 4)]
    assert oracle_mod.block_extents(10, "count", 4) == [(0, 3), (3, 3), (6, 2), (8, 2)]
    for n in (1, 7, 64, 97):
        for p in (1, 2, 5):
            if p <= n:
                e = oracle_mod.block_extents(n, "count", p)
                assert sum(x for _, x in e) == n and max(x for _, x in e) - min(x for _, x in e) <= 1


def test_faces_coordinates(oracle_mod):
    nx, ny, nz = 5, 4, 3
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    blk = (i + 10 * j + 100 * k).astype(np.float64)
    f = oracle_mod.faces(blk)
    assert f["xm"].shape == (nz, ny) and np.all(f["xm"] % 10 == 0)
    assert np.all(f["xp"] % 10 == nx - 1)
    assert f["ym"].shape == (nz, nx) and np.all((f["yp"] // 10) % 10 == ny - 1)
    assert f["zm"].shape == (ny, nx) and np.all(f["zp"] // 100 == nz - 1)


# ---------------------------------------------------------------------------
# Shared input generator
# ---------------------------------------------------------------------------

def _golden(name):
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)


def test_splitmix64_published_vector():
    """First outputs of SplitMix64 seeded with 1234567 (published vector, cited
    in the fixture)."""
    want = [int(l) for l in open(_golden("splitmix64_seed1234567.txt")) if l.strip() and not l.startswith("#")]
    got = [int(x) for x in J.splitmix64(1234567, np.arange(len(want)))]
    assert len(want) == 5 and got == want


def test_oracle_regression_fixtures(oracle_mod):
    """The oracle reproduces its committed fixtures bit for bit (they were
    written by tests/golden/make_golden.py, which calls only the oracle; a
    change to the oracle's arithmetic has to rewrite them)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", _golden("make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    for stem, grid, dtype, inputs, iters in mg.CASES:
        assert mg.render(grid, dtype, inputs, iters) == open(_golden(stem + ".txt")).read(), stem


def test_inputs_basic():
    u = J.initial_grid(6, 5, 4, "linear", interior="zero")
    assert u[-1, -1, -1] == 6.0 and u[0, 0, 0] == 0.0
    assert np.all(J.interior_of(u) == 0)
    v = J.initial_grid(6, 5, 4, "uniform", bc_seed=7, interior="uniform", interior_seed=8)
    assert v.min() >= 0.0 and v.max() < 1.0
    w = J.initial_grid(6, 5, 4, "uniform", bc_seed=7, interior="uniform", interior_seed=8,
                       dtype=np.float32)
    assert np.array_equal(w, v.astype(np.float32))
    sides = J.batched_sides()
    assert len(sides) == 256 and all(s % 16 == 0 and 16 <= s <= 192 for t in sides for s in t)
    reqs = J.serving_requests(200)
    assert all(32 <= s <= 256 for r in reqs for s in r["grid"])
    assert all(b["arrival_s"] > a["arrival_s"] for a, b in zip(reqs, reqs[1:]))
