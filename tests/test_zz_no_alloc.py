"""The allocation-free residual entry point, checked against the oracle and
against jacobi_residual.

jacobi_residual_noalloc is for callers that may not allocate device memory
when they need a residual: services that reserve all device memory at
start-up and forbid later allocations, and loops that cannot afford the
device-wide synchronisation a cudaMalloc or cudaFree may bring.  It keeps its
reduction scratch in a fixed array inside the library, so two calls in a row
must each see only their own data.  The test compares two consecutive calls
on different states with the CPU oracle's residual of the same state and with
the handle-based jacobi_residual (the tolerance of the other residual parity
tests), and checks that a grid larger than the fixed scratch is refused.
"""
import pytest

import paper_2102_12416_gb300 as jg

pytestmark = pytest.mark.gpu

RES_TOL = 1e-12

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2102_12416_gb300 import _build
    _build.build()
    jg.load()


def _reference(grid, dtype, init, iters):
    """rel and |r| from the existing entry point, and the state it saw."""
    with jg.Jacobi3D(grid, ("shape", (16, 16, 16)), dtype, init) as s:
        s.step(iters)
        rel, ab = s.residual()
        state = s.copy_out(padded=True)
    # padded copy-out zeroes the edges and corners, which the stencil never reads
    return rel[0], ab[0], state


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_oracle_and_jacobi_residual_twice(oracle_mod, dtype):
    cases = [((40, 33, 27), dict(bc="uniform", bc_seed=71, interior="uniform", interior_seed=72), 5),
             ((24, 48, 35), dict(bc="linear_noise", bc_seed=73, noise_amp=1e-3, interior="zero"), 11)]
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for grid, init, iters in cases:  # two calls in a row on different states
        rel, ab, state = _reference(grid, dtype, init, iters)
        u = torch.from_numpy(state).cuda()
        jg.jacobi_residual_noalloc(u.data_ptr(), grid, dtype, out.data_ptr())
        torch.cuda.synchronize()
        got_r, got_b, got_rel = (float(v) for v in out.cpu())
        orn, obn, orel = oracle_mod.residual(state)
        assert abs(got_r - orn) <= RES_TOL * orn and abs(got_b - obn) <= RES_TOL * obn
        assert abs(got_rel - orel) <= RES_TOL * orel
        assert abs(got_r - ab) <= RES_TOL * ab
        assert abs(got_rel - rel) <= RES_TOL * rel
        assert abs(got_r / got_b - got_rel) <= 1e-15 * got_rel


def test_noalloc_rejects_grid_beyond_scratch():
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(jg.JacobiError) as e:
        jg.jacobi_residual_noalloc(dummy.data_ptr(), (4, 4, jg.JACOBI_NOALLOC_MAX_PLANES + 1), "f64",
                                   out.data_ptr())
    assert e.value.code == jg.JACOBI_EINVAL
