"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Bars:
  * init, pack/unpack, decomposition and the FP64 stencil: bit-exact (every
    FP64 operation is rounded exactly as the oracle rounds it, and the
    integer-pipe adder is exact);
  * FP32 stencil: bit-exact against the FP32 oracle (same operation order),
    and within 1e-5 relative (inf-norm) of the FP64 oracle after the stated
    iterations;
  * residual norms: within 1e-12 relative (the per-point residuals are
    bit-identical; only the summation order differs);
  * solve iteration counts: equal.
"""
import math

import numpy as np
import pytest

import jacobi_inputs as J
import paper_2102_12416_gb300 as jg

pytestmark = pytest.mark.gpu

RES_TOL = 1e-12
FP32_VS_FP64 = 1e-5  # relative inf-norm distance of an FP32 run from the FP64 oracle


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2102_12416_gb300 import _build
    _build.build()
    jg.load()


def _mask_edges(p):
    """Padded copy_out writes edges and corners as 0 (the stencil never reads them)."""
    q = p.copy()
    nz, ny, nx = q.shape
    for a in (0, -1):
        for b in (0, -1):
            q[a, b, :] = 0
            q[a, :, b] = 0
            q[:, a, b] = 0
    return q


def _solver(grid, split, dtype="f64", init=None, path="fused"):
    return jg.Jacobi3D(grid, split, dtype, init, path=path)


INIT_CASES = [
    ((64, 64, 64), ("count", (2, 2, 2)), "f64", dict(bc="linear", interior="uniform", interior_seed=0)),
    ((45, 37, 29), ("count", (3, 5, 7)), "f64", dict(bc="uniform", bc_seed=1, interior="zero")),
    ((50, 20, 33), ("shape", (16, 16, 16)), "f32", dict(bc="linear_noise", bc_seed=3, noise_amp=1e-3)),
    ((33, 47, 18), ("shape", (32, 32, 32)), "f32", dict(bc="uniform", bc_seed=9, interior="uniform",
                                                        interior_seed=10)),
]


@pytest.mark.parametrize("grid,split,dtype,init", INIT_CASES)
def test_init_matches_shared_generator(grid, split, dtype, init):
    with _solver(grid, split, dtype, init) as s:
        got = s.copy_out(padded=True)
    want = J.initial_grid(*grid, dtype=np.float64 if dtype == "f64" else np.float32, **init)
    assert np.array_equal(got, _mask_edges(want))


def test_set_state_roundtrip():
    grid = (40, 31, 22)
    u = J.initial_grid(*grid, "uniform", bc_seed=5, interior="uniform", interior_seed=6)
    with _solver(grid, ("shape", (16, 8, 8))) as s:
        s.set_state(u)
        assert np.array_equal(s.copy_out(padded=True), _mask_edges(u))
        assert np.array_equal(s.copy_out(), J.interior_of(u))


ALL_PATHS = ["fused", "explicit", "persistent", "graph", "channel", "messaging", "host_staged"]


@pytest.mark.parametrize("path", ALL_PATHS)
def test_config1_bit_exact(oracle_mod, path):
    """64^3 FP64, 2x2x2 blocks of 32^3, linear boundary, U[0,1) interior, 100 iterations."""
    w = J.WORKLOADS["jacobi3d-fp64-64c-2x2x2"]
    init = dict(bc=w["bc"], bc_seed=w["bc_seed"], interior=w["interior"], interior_seed=w["interior_seed"])
    u0 = J.initial_grid(*w["grid"], **init)
    want = oracle_mod.jacobi(u0, w["iters"])
    with _solver(w["grid"], w["split"], "f64", init, path) as s:
        s.step(w["iters"])
        s.sync()
        got = s.copy_out(padded=True)
    assert np.array_equal(got, _mask_edges(want))


SPLITS = [("count", (1, 1, 1)), ("count", (2, 2, 2)), ("count", (3, 5, 7)), ("shape", (16, 16, 16)),
          ("shape", (7, 9, 5)), ("shape", (45, 8, 29))]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("path", ["fused", "persistent"])
def test_decomposition_invariance(oracle_mod, dtype, path):
    grid = (45, 37, 29)
    init = dict(bc="uniform", bc_seed=21, interior="uniform", interior_seed=22)
    npdt = np.float64 if dtype == "f64" else np.float32
    u0 = J.initial_grid(*grid, dtype=npdt, **init)
    want = oracle_mod.jacobi(u0, 13)
    for split in SPLITS:
        with _solver(grid, split, dtype, init, path) as s:
            s.step(13)
            got = s.copy_out()
        assert np.array_equal(got, J.interior_of(want)), (split, path)


def test_fp32_error_vs_fp64_oracle(oracle_mod):
    grid = (64, 64, 64)
    init = dict(bc="linear_noise", bc_seed=3, noise_amp=1e-3, interior="zero")
    ref = oracle_mod.jacobi(J.initial_grid(*grid, **init), 200)
    with _solver(grid, ("count", (2, 2, 2)), "f32", init) as s:
        s.step(200)
        got = s.copy_out().astype(np.float64)
    err = np.max(np.abs(got - J.interior_of(ref))) / np.max(np.abs(J.interior_of(ref)))
    assert err <= FP32_VS_FP64


@pytest.mark.parametrize("grid,shape,dtype", [((40, 24, 19), (16, 8, 8), "f64"),
                                               ((43, 27, 19), (13, 7, 8), "f32"),
                                               ((23, 10, 9), (5, 3, 4), "f64")])
def test_packed_faces_equal_neighbour_planes(grid, shape, dtype):
    """After k steps every receive slot holds the neighbour's boundary plane of
    u_k (pack + channel transfer: fused, explicit, or through the host-driven
    channel, messaging and host-staging forms) or the Dirichlet values.
    Ragged block extents exercise the padded rows and slots."""
    init = dict(bc="uniform", bc_seed=31, interior="uniform", interior_seed=32)
    for path in ("fused", "explicit", "channel", "messaging", "host_staged"):
        with _solver(grid, ("shape", shape), dtype, init, path) as s:
            s.step(3)
            full = s.copy_out(padded=True)
            full_ref = J.initial_grid(*grid, dtype=np.float64 if dtype == "f64" else np.float32, **init)
            for b in range(s.info.n_blocks):
                bi = s.block(b)
                (ox, oy, oz), (ex, ey, ez) = tuple(bi.origin), tuple(bi.extent)
                # ghost planes around the block, from the gathered padded grid
                # (boundary values come from the generator: padded copy_out of a
                # Dirichlet face is itself the slot, so use the generator there)
                src = full.copy()
                src[0], src[-1] = full_ref[0], full_ref[-1]
                src[:, 0], src[:, -1] = full_ref[:, 0], full_ref[:, -1]
                src[:, :, 0], src[:, :, -1] = full_ref[:, :, 0], full_ref[:, :, -1]
                zs, ys, xs = slice(oz + 1, oz + 1 + ez), slice(oy + 1, oy + 1 + ey), slice(ox + 1, ox + 1 + ex)
                want = {
                    0: src[zs, ys, ox], 1: src[zs, ys, ox + ex + 1],
                    2: src[zs, oy, xs], 3: src[zs, oy + ey + 1, xs],
                    4: src[oz, ys, xs], 5: src[oz + ez + 1, ys, xs],
                }
                for f in range(6):
                    assert np.array_equal(s.read_face(b, f), want[f]), (path, b, f)


RAGGED_SHAPES = [(1, 1), (2, 3), (3, 5), (5, 2), (6, 7), (7, 1), (9, 6), (11, 13)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("path", ["graph", "persistent"])
def test_ragged_block_shapes(oracle_mod, dtype, path):
    """Blocks whose rows are not a whole number of 16-byte vectors, or whose
    planes are not a whole number of 4-row groups, stream through padded rows:
    iterates stay bit-exact and the residual matches the oracle."""
    grid = (23, 21, 9)
    init = dict(bc="uniform", bc_seed=41, interior="uniform", interior_seed=42)
    npdt = np.float64 if dtype == "f64" else np.float32
    u0 = J.initial_grid(*grid, dtype=npdt, **init)
    want = oracle_mod.jacobi(u0, 7)
    rn, _, rel = oracle_mod.residual(want)
    for sx, sy in RAGGED_SHAPES:
        with _solver(grid, ("shape", (sx, sy, 4)), dtype, init, path) as s:
            s.step(7)
            got = s.copy_out()
            grel, gabs = s.residual()
        assert np.array_equal(got, J.interior_of(want)), (sx, sy)
        assert abs(gabs[0] - rn) <= RES_TOL * rn and abs(grel[0] - rel) <= RES_TOL * rel, (sx, sy)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_persistent_replays_continue(oracle_mod, dtype):
    """The persistent path captures its cooperative launch once per launch
    shape and replays it, reading the start iteration from device memory:
    calls of the same and of different lengths continue where the last one
    stopped, bit-exact with the oracle."""
    grid, split = (45, 37, 29), ("count", (3, 5, 7))
    init = dict(bc="uniform", bc_seed=23, interior="uniform", interior_seed=24)
    npdt = np.float64 if dtype == "f64" else np.float32
    u0 = J.initial_grid(*grid, dtype=npdt, **init)
    with _solver(grid, split, dtype, init, "persistent") as s:
        for n in (7, 7, 7, 5, 7):
            s.step(n)
        s.sync()
        got = s.copy_out()
    assert np.array_equal(got, J.interior_of(oracle_mod.jacobi(u0, 33)))


@pytest.mark.parametrize("ws", ["1", "0"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_persistent_kernels_vs_oracle(oracle_mod, monkeypatch, dtype, ws):
    """Both persistent kernels (warp-specialised, JACOBI_PERSIST_WS=1, and
    barrier-driven, 0) on uneven grids with ragged and 64-wide blocks, at
    several work-item shapes: iterates bit-exact with the oracle, a fused
    residual within 1e-12, and a solve that stops at the oracle's check."""
    monkeypatch.setenv("JACOBI_PERSIST_WS", ws)
    grids = [(70, 64, 37), (45, 37, 29), (33, 18, 50)]
    splits = [("shape", (64, 64, 64)), ("count", (3, 5, 2)), ("shape", (11, 9, 16))]
    inits = [dict(bc="uniform", bc_seed=61 + g, interior="uniform", interior_seed=71 + g) for g in range(3)]
    npdt = np.float64 if dtype == "f64" else np.float32
    u0 = [J.initial_grid(*grids[g], dtype=npdt, **inits[g]) for g in range(3)]
    want = [oracle_mod.jacobi(u0[g], 9) for g in range(3)]
    for zc, cw in ((0, 8), (1, 8), (2, 2)):
        with jg.Jacobi3D(grids, splits, dtype, inits, path="persistent") as s:
            if zc:
                s.set_shape(zc, cw)
            s.step(4)
            s.step(5)
            s.sync()
            rel, ab = s.residual()
            for g in range(3):
                assert np.array_equal(s.copy_out(g), J.interior_of(want[g])), (zc, cw, g)
                rn, _, orel = oracle_mod.residual(want[g])
                assert abs(ab[g] - rn) <= RES_TOL * rn and abs(rel[g] - orel) <= RES_TOL * orel
    zi = [dict(bc="uniform", bc_seed=61 + g, interior="zero") for g in range(3)]
    with jg.Jacobi3D(grids, splits, dtype, zi, path="persistent") as s:
        its, rels, sts = s.solve(1e-5, 5000, 10)
        got = [s.copy_out(g) for g in range(3)]
    for g in range(3):
        ou, k, orel, ost = oracle_mod.solve(J.initial_grid(*grids[g], dtype=npdt, **zi[g]), 1e-5, 5000, 10)
        assert (its[g], sts[g]) == (k, ost), g
        assert np.array_equal(got[g], J.interior_of(ou)), g


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_residual_parity(oracle_mod, dtype):
    grid = (37, 29, 41)
    init = dict(bc="linear_noise", bc_seed=7, noise_amp=1e-3, interior="uniform", interior_seed=8)
    npdt = np.float64 if dtype == "f64" else np.float32
    u0 = J.initial_grid(*grid, dtype=npdt, **init)
    for k in (0, 9):
        uk = oracle_mod.jacobi(u0, k)
        rn, bn, rel = oracle_mod.residual(uk)
        with _solver(grid, ("shape", (16, 16, 16)), dtype, init) as s:
            s.step(k)
            grel, gabs = s.residual()
        assert abs(gabs[0] - rn) <= RES_TOL * rn
        assert abs(grel[0] - rel) <= RES_TOL * rel


def test_residual_closed_form_linear(oracle_mod):
    """At the linear fixed point r = 0 in exact arithmetic; in FP64 each r_i is
    rounding noise of at most ~6 ulps of |s| <= 36, so rel stays below 1e-14.
    Per-point values are bit-identical with the oracle's, so the two sums of
    squares agree to the summation-order tolerance."""
    grid = (48, 40, 36)
    with _solver(grid, ("count", (2, 2, 2)), "f64", dict(bc="linear", interior="bc")) as s:
        rel, ab = s.residual()
    rn, _, orel = oracle_mod.residual(J.initial_grid(*grid, "linear", interior="bc"))
    assert rel[0] <= 1e-14
    assert abs(ab[0] - rn) <= RES_TOL * rn


@pytest.mark.parametrize("path", ["fused", "persistent"])
def test_solve_matches_oracle(oracle_mod, path):
    grid = (20, 16, 12)
    init = dict(bc="uniform", bc_seed=41, interior="zero")
    u0 = J.initial_grid(*grid, **init)
    tol, cap, check = 1e-8, 5000, 7
    want, k, rel, st = oracle_mod.solve(u0, tol, cap, check)
    with _solver(grid, ("shape", (8, 8, 8)), "f64", init, path) as s:
        it, grel, gst = s.solve(tol, cap, check)
        got = s.copy_out(padded=True)
    assert (it[0], gst[0]) == (k, st)
    assert abs(grel[0] - rel) <= RES_TOL * rel
    assert np.array_equal(got, _mask_edges(want))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_tile_only_persistent_solve_matches_oracle(oracle_mod, dtype):
    """Persistent launches whose items are all tiles (the barrier-driven
    kernel, the first iteration of a check launch fusing the residual):
    iteration count, status and frozen state equal the oracle's solve, the
    residual within the residual bar."""
    grid = (37, 30, 26)
    init = dict(bc="uniform", bc_seed=43, interior="zero")
    npdt = np.float64 if dtype == "f64" else np.float32
    u0 = J.initial_grid(*grid, dtype=npdt, **init)
    tol, cap, check = 1e-6, 3000, 9
    want, k, rel, st = oracle_mod.solve(u0, tol, cap, check)
    with _solver(grid, ("shape", (16, 16, 16)), dtype, init, "persistent") as s:
        s.set_shape(0, 0)  # every block as tiles
        assert set(s.kind_items()) == {"tiles"}
        it, grel, gst = s.solve(tol, cap, check)
        got = s.copy_out(padded=True)
    assert (it[0], gst[0]) == (k, st)
    assert abs(grel[0] - rel) <= RES_TOL * rel
    assert np.array_equal(got, _mask_edges(want))


def test_solve_cap_and_stagnation(oracle_mod):
    grid = (16, 16, 16)
    init = dict(bc="linear_noise", bc_seed=3, noise_amp=1e-3, interior="zero")
    with _solver(grid, ("count", (2, 2, 2)), "f32", init) as s:
        it, rel, st = s.solve(1e-14, 100000, 10, stall_checks=5)
    u0 = J.initial_grid(*grid, dtype=np.float32, **init)
    _, k, orel, ost = oracle_mod.solve(u0, 1e-14, 100000, 10, stall_checks=5)
    assert st[0] == jg.JACOBI_SOLVE_STAGNATED == ost and it[0] == k
    with _solver(grid, ("count", (2, 2, 2)), "f64", init) as s:
        it, rel, st = s.solve(1e-30, 23, 10)
    assert (it[0], st[0]) == (23, jg.JACOBI_SOLVE_MAX_ITERS)


def test_batched_solve_alone_equals_mix(oracle_mod):
    """Each grid's state in a batch is bit-identical to solving it alone, with
    the same iteration count; the residual may differ in its last bits because
    a handle splits blocks into work items according to its total size."""
    grids = [(24, 16, 40), (16, 16, 16), (48, 32, 16)]
    inits = [dict(bc="uniform", bc_seed=(2 << 32) | g, interior="zero") for g in range(3)]
    splits = [("shape", (16, 16, 16))] * 3
    with jg.Jacobi3D(grids, splits, "f64", inits) as s:
        its, rels, sts = s.solve(1e-7, 20000, 10)
        mix = [s.copy_out(g) for g in range(3)]
    for g in range(3):
        with jg.Jacobi3D([grids[g]], [splits[g]], "f64", [inits[g]]) as s1:
            it1, rel1, st1 = s1.solve(1e-7, 20000, 10)
            alone = s1.copy_out()
        assert (it1[0], st1[0]) == (its[g], sts[g])
        assert abs(rel1[0] - rels[g]) <= RES_TOL * rels[g]
        assert np.array_equal(alone, mix[g])
        _, k, _, _ = oracle_mod.solve(J.initial_grid(*grids[g], **inits[g]), 1e-7, 20000, 10)
        assert k == its[g]


@pytest.mark.parametrize("path", ["explicit", "channel", "messaging", "host_staged"])
def test_exchange_forms_timed_and_batched(oracle_mod, path):
    """The unfused exchange forms on a batch of grids with ragged blocks, split
    across jacobi_step_timed and jacobi_step calls: every grid bit-exact with
    the oracle, the phase times positive.  A batched solve then freezes grids
    at different checks; each grid's result equals its solve alone (the
    exchanges of the grids still running never touch a frozen grid)."""
    grids = [(24, 16, 40), (19, 23, 11), (48, 32, 16)]
    inits = [dict(bc="uniform", bc_seed=(2 << 32) | g, interior="uniform", interior_seed=70 + g) for g in range(3)]
    splits = [("shape", (16, 16, 16)), ("shape", (7, 9, 5)), ("count", (3, 2, 1))]
    with jg.Jacobi3D(grids, splits, "f64", inits, path=path) as s:
        comp, exch = s.step_timed(5)
        s.step(4)
        assert comp > 0 and exch > 0
        outs = [s.copy_out(g) for g in range(3)]
    for g in range(3):
        want = oracle_mod.jacobi(J.initial_grid(*grids[g], **inits[g]), 9)
        assert np.array_equal(outs[g], J.interior_of(want)), g
    zinits = [dict(bc="uniform", bc_seed=(2 << 32) | g, interior="zero") for g in range(3)]
    with jg.Jacobi3D(grids, splits, "f64", zinits, path=path) as s:
        its, rels, sts = s.solve(1e-7, 20000, 10)
        mix = [s.copy_out(g) for g in range(3)]
    assert len(set(its)) > 1
    for g in range(3):
        with jg.Jacobi3D([grids[g]], [splits[g]], "f64", [zinits[g]], path=path) as s1:
            it1, _, st1 = s1.solve(1e-7, 20000, 10)
            assert (it1[0], st1[0]) == (its[g], sts[g])
            assert np.array_equal(s1.copy_out(), mix[g]), g


def test_local_halo_measurement_switch(oracle_mod):
    """With the halo-share switch on, every block stores its new boundary
    planes into its own receive slots (same kernels and bytes, faces kept
    local); switched off and the state reset, the exchange is back and the
    iterates are the oracle's again."""
    grid, split = (40, 24, 19), ("shape", (16, 8, 8))
    init = dict(bc="uniform", bc_seed=33, interior="uniform", interior_seed=34)
    u0 = J.initial_grid(*grid, **init)
    with _solver(grid, split, "f64", init, "graph") as s:
        jg.jacobi_measure_local_halo(s.h, 1)
        s.step(3)
        full = s.copy_out(padded=True)
        for b in range(s.info.n_blocks):
            bi = s.block(b)
            (ox, oy, oz), (ex, ey, ez) = tuple(bi.origin), tuple(bi.extent)
            blk = full[oz + 1:oz + 1 + ez, oy + 1:oy + 1 + ey, ox + 1:ox + 1 + ex]
            own = {0: blk[:, :, 0], 1: blk[:, :, -1], 2: blk[:, 0, :], 3: blk[:, -1, :], 4: blk[0], 5: blk[-1]}
            for f in range(6):
                if bi.neighbour[f] >= 0:
                    assert np.array_equal(s.read_face(b, f), own[f]), (b, f)
        jg.jacobi_measure_local_halo(s.h, 0)
        s.set_state(u0)
        s.step(33)
        got = s.copy_out()
    assert np.array_equal(got, J.interior_of(oracle_mod.jacobi(u0, 33)))


# ---- the 512^3 FP64 workload (8x8x8 blocks of 64^3) -------------------------------

def _cfg2():
    w = J.WORKLOADS["jacobi3d-fp64-512c-8x8x8"]
    init = dict(bc=w["bc"], bc_seed=w["bc_seed"], interior=w["interior"], interior_seed=w["interior_seed"])
    return w, init


def test_config2_full_size_vs_oracle(oracle_mod):
    """Full 512^3 grid, the benchmark's launch configuration, 260 iterations (the
    front from the boundary has reached every point), compared bit for bit;
    the residual norms (|b - Au|, |b| and rel, over blocks whose planes are
    split into two row windows) within 1e-12 of the oracle's."""
    w, init = _cfg2()
    u0 = J.initial_grid(*w["grid"], **init)
    want = oracle_mod.jacobi(u0, 260)
    with _solver(w["grid"], w["split"], "f64", init, "graph") as s:
        s.step(260)
        got = s.copy_out()
        rel, ab = s.residual()
    assert np.array_equal(got, J.interior_of(want))
    rn, bn, orel = oracle_mod.residual(want)
    assert abs(ab[0] - rn) <= RES_TOL * rn and abs(rel[0] - orel) <= RES_TOL * orel


def test_weak_scaling_slab_full_size_vs_oracle(oracle_mod):
    """One GPU's share of the paper's weak-scaling base problem (1536^3 points
    per node of six GPUs, Sec. 4.3): 1536 x 768 x 512 FP64 in 64^3 blocks,
    the benchmark's launch configuration, 24 iterations bit-exact with the
    oracle (the front from the boundary reaches 24 points in)."""
    w = J.WORKLOADS["jacobi3d-fp64-1536x768x512"]
    init = dict(bc=w["bc"], bc_seed=w["bc_seed"], interior=w["interior"], interior_seed=w["interior_seed"])
    u0 = J.initial_grid(*w["grid"], **init)
    with _solver(w["grid"], w["split"], "f64", init, "graph") as s:
        assert set(s.kind_items()) == {"stream8"}
        s.step(24)
        got = s.copy_out()
    want = oracle_mod.jacobi(u0, 24)
    del u0
    assert np.array_equal(got, J.interior_of(want))


def test_config2_invariance_1000_iters():
    """1000 iterations: 8x8x8 blocks equal 2x2x2 blocks bit for bit."""
    w, init = _cfg2()
    outs = []
    for split in (w["split"], ("count", (2, 2, 2))):
        with _solver(w["grid"], split, "f64", init, "graph") as s:
            s.step(w["iters"])
            outs.append(s.copy_out())
    assert np.array_equal(outs[0], outs[1])


def test_config2_eigenmode_closed_form():
    """Eigenmode decay after 1000 iterations at full size: lambda^1000 exactly."""
    w, _ = _cfg2()
    nx, ny, nz = w["grid"]
    g = J.initial_grid(nx, ny, nz, "linear", interior="bc")
    x, y, z = J.coordinates(nx, ny, nz)
    mode = np.sin(np.pi * z)[:, None, None] * np.sin(np.pi * y)[None, :, None] * np.sin(2 * np.pi * x)[None, None, :]
    u0 = g.copy()
    J.interior_of(u0)[...] += 0.5 * J.interior_of(mode)
    lam = (math.cos(2 * math.pi / (nx + 1)) + math.cos(math.pi / (ny + 1)) + math.cos(math.pi / (nz + 1))) / 3
    with _solver(w["grid"], w["split"], "f64", dict(bc="linear", interior="bc"), "graph") as s:
        s.set_state(u0)
        s.step(w["iters"])
        got = s.copy_out() - J.interior_of(g)
    want = lam ** w["iters"] * 0.5 * J.interior_of(mode)
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))


def test_fp32_solve_to_tolerance_vs_fp64_oracle(oracle_mod):
    """FP32 state, FP64 residual: a 48^3 proxy of the 768^3 FP32 workload
    (same boundary family, 12^3 blocks) solved to 1e-6 stops at the same check
    as the FP32 oracle with a bit-identical solution.  Its drift from the FP64
    iteration after the same number of steps (FP32 rounding accumulated over
    ~5200 iterations, each update rounding s/6 once; measured 1.3e-6) is
    within the 1e-5 relative (inf-norm) bar."""
    w = J.WORKLOADS["jacobi3d-fp32-768c-12x12x12"]
    init = dict(bc=w["bc"], bc_seed=w["bc_seed"], noise_amp=w["noise_amp"], interior=w["interior"])
    grid = (48, 48, 48)
    with _solver(grid, ("count", (12, 12, 12)), "f32", init) as s:
        it, rel, st = s.solve(1e-6, 100000, 100, stall_checks=50)
        got = s.copy_out()
    u32, k32, rel32, st32 = oracle_mod.solve(J.initial_grid(*grid, dtype=np.float32, **init), 1e-6, 100000, 100, 50)
    assert (it[0], st[0]) == (k32, st32) and st[0] == jg.JACOBI_SOLVE_CONVERGED
    assert np.array_equal(got, J.interior_of(u32))
    ref = J.interior_of(oracle_mod.jacobi(J.initial_grid(*grid, **init), k32))
    assert np.max(np.abs(got.astype(np.float64) - ref)) / np.max(np.abs(ref)) <= FP32_VS_FP64


# ---- FP32 in 64^3 blocks: the 8-consumer-warp streaming kernel of the 768^3 workload

def _w768():
    w = J.WORKLOADS["jacobi3d-fp32-768c-12x12x12"]
    init = dict(bc=w["bc"], bc_seed=w["bc_seed"], noise_amp=w["noise_amp"], interior=w["interior"])
    return w, init


@pytest.mark.parametrize("path", ["graph", "persistent", "explicit"])
def test_fp32_64c_blocks_bit_exact(oracle_mod, path):
    """128^3 FP32 in 2x2x2 blocks of 64^3: whole 64x64 planes streamed by CTAs
    of 8 consumer warps (the kernel the 768^3 workload runs), bit-exact with
    the FP32 oracle after 30 iterations, residual within 1e-12."""
    _, init = _w768()
    grid = (128, 128, 128)
    u0 = J.initial_grid(*grid, dtype=np.float32, **init)
    want = oracle_mod.jacobi(u0, 30)
    rn, _, rel = oracle_mod.residual(want)
    with _solver(grid, ("count", (2, 2, 2)), "f32", init, path) as s:
        if path != "persistent":
            assert s.kind_items() == {"stream8": s.info.kind_items[1]}
        s.step(30)
        s.sync()
        got = s.copy_out()
        grel, gabs = s.residual()
    assert np.array_equal(got, J.interior_of(want))
    assert abs(gabs[0] - rn) <= RES_TOL * rn and abs(grel[0] - rel) <= RES_TOL * rel


@pytest.mark.parametrize("path", ["graph", "persistent"])
def test_fp32_ragged_61x62x64_blocks(oracle_mod, path):
    """Blocks of 61 x 62 x 64 FP32 points: rows padded to 64 and planes to 64
    rows, so the 8-warp kernel runs its ragged variant (padding lanes and rows
    take the ghost values); bit-exact with the FP32 oracle, faces included."""
    _, init = _w768()
    grid = (122, 124, 64)
    u0 = J.initial_grid(*grid, dtype=np.float32, **init)
    want = oracle_mod.jacobi(u0, 25)
    with _solver(grid, ("shape", (61, 62, 64)), "f32", init, path) as s:
        if path == "graph":
            assert s.kind_items() == {"stream8_ragged": s.info.kind_items[4]}
        s.step(25)
        s.sync()
        got = s.copy_out()
    assert np.array_equal(got, J.interior_of(want))


def test_fp32_768c_workload_vs_oracle(oracle_mod):
    """The 768^3 FP32 workload itself (12^3 blocks of 64^3) in the benchmark's
    launch configuration: after 20 iterations bit-exact with the FP32 oracle;
    after the workload's 200 iterations within 1e-5 relative of the FP64
    oracle (FP32 rounding alone: each update rounds s/6 once)."""
    w, init = _w768()
    u0 = J.initial_grid(*w["grid"], **init)
    u0f = u0.astype(np.float32)
    want20 = J.interior_of(oracle_mod.jacobi(u0f, 20))
    with _solver(w["grid"], w["split"], "f32", init, "graph") as s:
        assert set(s.kind_items()) == {"stream8"}
        s.step(20)
        got = s.copy_out()
        assert np.array_equal(got, want20)
        del got, want20
        s.step(w["iters"] - 20)
        got = s.copy_out()
    ref = J.interior_of(oracle_mod.jacobi(u0, w["iters"]))
    err = np.max(np.abs(got.astype(np.float64) - ref)) / np.max(np.abs(ref))
    assert err <= FP32_VS_FP64


# ---- the batched workload: 256 grids, sides in {16..192}, 32^3 blocks -----------

def _batched(name):
    return J.workload_grids(name)


@pytest.mark.parametrize("name", ["jacobi3d-batched256-fp32", "jacobi3d-batched256-fp64"])
def test_batched_full_size(oracle_mod, name):
    """All 256 grids stepped together for the workload's 500 iterations: the
    graph and persistent paths agree bit for bit on every grid, and the three
    smallest grids (which the oracle finishes in seconds) match the oracle."""
    grids, splits, inits, dtype, iters = _batched(name)
    npdt = np.float64 if dtype == "f64" else np.float32
    small = sorted(range(len(grids)), key=lambda g: grids[g][0] * grids[g][1] * grids[g][2])[:3]
    outs = {}
    for path in ("graph", "persistent"):
        with jg.Jacobi3D(grids, splits, dtype, inits, path=path) as s:
            s.step(iters)
            s.sync()
            outs[path] = [s.copy_out(g) for g in range(len(grids))]
    for g in range(len(grids)):
        assert np.array_equal(outs["graph"][g], outs["persistent"][g]), g
    for g in small:
        want = oracle_mod.jacobi(J.initial_grid(*grids[g], dtype=npdt, **inits[g]), iters)
        assert np.array_equal(outs["graph"][g], J.interior_of(want)), g


def test_autotune_keeps_results(tmp_path, monkeypatch, oracle_mod):
    """The autotuner times shapes x paths (and ring depths) on a scratch handle,
    applies the winner and caches it; the tuned handle's iterates equal the
    oracle's."""
    monkeypatch.setenv("JACOBI_TUNE_CACHE", str(tmp_path / "tune.txt"))
    grids, splits, inits, dtype, _ = _batched("jacobi3d-batched256-fp32")
    grids, splits, inits = grids[:12], splits[:12], inits[:12]
    with jg.Jacobi3D(grids, splits, dtype, inits) as s:
        r = s.autotune(8)
        assert r["n_tried"] >= 6 and not r["from_cache"] and r["ms_per_iter"] > 0
        info = s.info
        assert jg.PATH_NAMES[info.path] == r["path"] and info.stages == r["stages"]
        assert (info.zchunk, info.cw_cap) == (r["zchunk"], r["cw_cap"])
        s.step(17)
        s.sync()
        tuned = [s.copy_out(g) for g in range(len(grids))]
    with jg.Jacobi3D(grids, splits, dtype, inits) as s:
        r2 = s.autotune(8)
        assert r2["from_cache"]
        assert (r2["path"], r2["stages"], r2["zchunk"], r2["cw_cap"]) == (r["path"], r["stages"], r["zchunk"],
                                                                        r["cw_cap"])
    for g in (0, 5, 11):
        want = oracle_mod.jacobi(J.initial_grid(*grids[g], dtype=np.float32, **inits[g]), 17)
        assert np.array_equal(tuned[g], J.interior_of(want))


def test_autotune_path_keeps_path_and_results(tmp_path, monkeypatch, oracle_mod):
    """The search restricted to the persistent path applies that path with its
    best shape and ring depth, is cached apart from the full search, and the
    tuned handle's iterates equal the oracle's; another path is refused."""
    monkeypatch.setenv("JACOBI_TUNE_CACHE", str(tmp_path / "tune.txt"))
    grids, splits, inits, dtype, _ = _batched("jacobi3d-batched256-fp32")
    grids, splits, inits = grids[:8], splits[:8], inits[:8]
    with jg.Jacobi3D(grids, splits, dtype, inits) as s:
        r = s.autotune(8, path="persistent")
        assert r["path"] == "persistent" and r["n_tried"] >= 2 and not r["from_cache"]
        info = s.info
        assert jg.PATH_NAMES[info.path] == "persistent" and info.stages == r["stages"]
        assert (info.zchunk, info.cw_cap) == (r["zchunk"], r["cw_cap"])
        s.step(13)
        s.sync()
        tuned = [s.copy_out(g) for g in range(len(grids))]
        with pytest.raises(jg.JacobiError):
            jg.jacobi_autotune_path(s.h, "explicit", 8, s.stream)
    with jg.Jacobi3D(grids, splits, dtype, inits) as s:
        assert s.autotune(8, path="persistent")["from_cache"]
        assert not s.autotune(8)["from_cache"]  # the full search has its own cache entry
    for g in (0, 3, 7):
        want = oracle_mod.jacobi(J.initial_grid(*grids[g], dtype=np.float32, **inits[g]), 13)
        assert np.array_equal(tuned[g], J.interior_of(want))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_shapes_give_identical_iterates(oracle_mod, dtype):
    """Every work-item shape (z-chunk depth, consumer-warp cap) on the graph
    and persistent paths gives the oracle's iterates on uneven grids with
    ragged blocks and 64-wide planes; a shape finer than the tables hold is
    refused."""
    grids = [(70, 64, 37), (45, 37, 29), (33, 18, 50)]
    splits = [("shape", (64, 64, 64)), ("count", (3, 5, 2)), ("shape", (11, 9, 16))]
    inits = [dict(bc="uniform", bc_seed=81 + g, interior="uniform", interior_seed=91 + g) for g in range(3)]
    npdt = np.float64 if dtype == "f64" else np.float32
    want = [J.interior_of(oracle_mod.jacobi(J.initial_grid(*grids[g], dtype=npdt, **inits[g]), 11))
            for g in range(3)]
    with jg.Jacobi3D(grids, splits, dtype, inits) as s0:
        zc0 = s0.info.zchunk
    for path in ("graph", "persistent"):
        for zc, cw in ((zc0, 8), (zc0, 2), (max(1, zc0 // 2), 4), (max(1, zc0 // 4), 2), (2 * zc0, 8),
                       (zc0, 0), (max(1, zc0 // 4), 0)):
            with jg.Jacobi3D(grids, splits, dtype, inits, path=path) as s:
                s.set_shape(zc, cw)
                assert (s.info.zchunk, s.info.cw_cap) == (min(zc, 37), cw)  # 37: the tallest block
                s.step(5)
                s.step(6)
                s.sync()
                for g in range(3):
                    assert np.array_equal(s.copy_out(g), want[g]), (path, zc, cw, g)
    with jg.Jacobi3D(grids, splits, dtype, inits) as s:
        if zc0 >= 8:
            with pytest.raises(jg.JacobiError) as e:
                s.set_shape(1, 2)
            assert e.value.code == jg.JACOBI_EINVAL


# ---- failure detection: bounded waits, no hang ----------------------------------

def test_persistent_wait_times_out(monkeypatch):
    monkeypatch.setenv("JACOBI_WAIT_MS", "200")
    with _solver((32, 32, 32), ("count", (2, 2, 2)), "f64", None, "persistent") as s:
        jg.jacobi_debug_drop_block(s.h, 3)
        s.step(5)
        with pytest.raises(jg.JacobiError) as e:
            s.sync()
        assert e.value.code == jg.JACOBI_ETIMEDOUT
        jg.jacobi_debug_drop_block(s.h, -1)
    # the context is still usable
    with _solver((32, 32, 32), ("count", (2, 2, 2)), "f64", None, "persistent") as s:
        s.step(3)
        s.sync()


@pytest.mark.parametrize("dtype,nx", [("f32", 1030), ("f64", 515)])
@pytest.mark.parametrize("path", ALL_PATHS)
def test_wide_rows_take_the_tile_kernel(oracle_mod, dtype, nx, path):
    """Rows wider than one CTA can stream (more than 256 16-byte vectors) go
    to the tile kernel, alone and next to streamed blocks; iterates stay
    bit-exact, faces are packed and the residual matches."""
    grid = (nx + 40, 11, 9)
    init = dict(bc="uniform", bc_seed=51, interior="uniform", interior_seed=52)
    npdt = np.float64 if dtype == "f64" else np.float32
    u0 = J.initial_grid(*grid, dtype=npdt, **init)
    want = oracle_mod.jacobi(u0, 6)
    rn, _, rel = oracle_mod.residual(want)
    # one wide block (tiles) beside a 40-wide one (streamed), split in z too
    with _solver(grid, ("shape", (nx, 11, 5)), dtype, init, path) as s:
        assert s.launch_kinds() >= 2
        s.step(6)
        got = s.copy_out()
        grel, gabs = s.residual()
    assert np.array_equal(got, J.interior_of(want))
    assert abs(gabs[0] - rn) <= RES_TOL * rn and abs(grel[0] - rel) <= RES_TOL * rel
