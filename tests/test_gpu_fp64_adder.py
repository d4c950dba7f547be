"""The FP64 stencil's integer-pipe adder (dadd_nn) must equal IEEE-754
round-to-nearest-even addition bit for bit on its domain (non-negative,
exponent field < 2040); numpy's float64 addition is the reference.  And the
step kernels give identical iterates whether the pair sums run on the integer
pipe or on the FP64 pipe (JACOBI_FP64_EMU=0), and the FP32 residual-only
launches (pair sums of widened values on the integer pipe inside the domain)
give identical norms either way.  The FP32 residual's
integer-pipe widening (binary32 -> binary64) equals the conversion
instruction on all 2^32 inputs, and so does the FP32 update's two-operation
division by 6 against the division instruction sequence."""
import numpy as np
import pytest

import jacobi_inputs as J
import paper_2102_12416_gb300 as jg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2102_12416_gb300 import _build
    _build.build()
    jg.load()


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    kind = rng.integers(0, 6, size=n)
    exp = np.where(kind == 0, 1023 - rng.integers(0, 40, size=n),          # [2^-39, 2)
          np.where(kind == 1, 1 + rng.integers(0, 2039, size=n),            # any normal < 2040
          np.where(kind == 2, 0,                                            # subnormal
                   1023 - rng.integers(0, 3, size=n)))).astype(np.uint64)   # near 1
    short = kind >= 4                                                       # few mantissa bits
    cut = rng.integers(0, 53, size=n).astype(np.uint64)
    mant = np.where(short, mant & ~((np.uint64(1) << cut) - np.uint64(1)), mant)
    a_bits = (exp << np.uint64(52)) | mant
    gap = rng.integers(0, 71, size=n).astype(np.int64)
    eb = np.maximum(exp.astype(np.int64) - gap, 0).astype(np.uint64)
    mb = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    cutb = rng.integers(0, 53, size=n).astype(np.uint64)
    mb = np.where(rng.random(n) < 0.3, mb & ~((np.uint64(1) << cutb) - np.uint64(1)), mb)
    b_bits = (eb << np.uint64(52)) | mb
    a, b = a_bits.view(np.float64).copy(), b_bits.view(np.float64).copy()
    b[::11] = 0.0
    b[::13] = a[::13]
    # exact-tie patterns: b is half an ulp of a (times an odd factor of 2^k)
    t = np.arange(0, n, 17)
    b[t] = np.ldexp(np.ones(len(t)), np.frexp(a[t])[1] - 54) * (1 + 2 * (t % 3))
    swap = rng.random(n) < 0.5
    return np.where(swap, b, a), np.where(swap, a, b)


def test_integer_pipe_adder_is_ieee_rne():
    for seed in (1, 2, 3):
        a, b = _pairs(1 << 22, seed)
        assert (a >= 0).all() and (b >= 0).all()
        want = (a + b).view(np.uint64)
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        out = torch.empty_like(da)
        jg.jacobi_selftest_dadd(da.data_ptr(), db.data_ptr(), len(a), out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, [(a[i].hex(), b[i].hex()) for i in bad[:4]]


def test_stencil_same_with_and_without_integer_adds(monkeypatch):
    grid, split = (96, 80, 72), ("shape", (32, 16, 24))
    init = dict(bc="uniform", bc_seed=5, interior="uniform", interior_seed=6)
    outs = []
    for emu in ("1", "0"):
        monkeypatch.setenv("JACOBI_FP64_EMU", emu)
        with jg.Jacobi3D(grid, split, "f64", init, path="graph") as s:
            s.step(150)
            rel, _ = s.residual()
            outs.append((s.copy_out(), rel[0]))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_negative_values_keep_the_fp64_pipe(oracle_mod):
    """A boundary with negative values is outside the adder's domain: the grid
    runs on the FP64 pipe and still matches the oracle."""
    nx, ny, nz = 40, 36, 32
    u = J.initial_grid(nx, ny, nz, "uniform", bc_seed=9, interior="uniform", interior_seed=10) - 0.5
    with jg.Jacobi3D((nx, ny, nz), ("shape", (16, 16, 16)), "f64") as s:
        s.set_state(u)
        s.step(40)
        got = s.copy_out()
    assert np.array_equal(got, J.interior_of(oracle_mod.jacobi(u, 40)))


def test_fp32_residual_same_with_and_without_integer_adds(monkeypatch, oracle_mod):
    """An FP32 state inside the adder's domain (non-negative, finite): the
    residual-only launch's integer-pipe pair sums give the same |r|, |b| and
    rel, bit for bit, as the FP64-pipe sums, and both match the oracle's FP64
    residual of the FP32 state within the residual bar."""
    grid, split = (45, 37, 29), ("shape", (16, 16, 16))
    init = dict(bc="linear_noise", bc_seed=21, noise_amp=1e-3, interior="uniform", interior_seed=22)
    u = J.initial_grid(*grid, dtype=np.float32, **init)
    uk = oracle_mod.jacobi(u, 17)
    rn, bn, rel = oracle_mod.residual(uk)
    outs = []
    for emu in ("1", "0"):
        monkeypatch.setenv("JACOBI_FP64_EMU", emu)
        with jg.Jacobi3D(grid, split, "f32", init, path="graph") as s:
            s.step(17)
            grel, gabs = s.residual()
            outs.append((grel[0], gabs[0]))
    assert outs[0] == outs[1]
    assert abs(outs[0][1] - rn) <= 1e-12 * rn and abs(outs[0][0] - rel) <= 1e-12 * rel


def test_fp32_negative_state_residual_keeps_the_fp64_pipe(oracle_mod):
    """An FP32 state with negative values is outside the adder's domain: its
    residual runs on the FP64 pipe and matches the oracle."""
    nx, ny, nz = 33, 30, 28
    u = J.initial_grid(nx, ny, nz, "uniform", bc_seed=23, interior="uniform", interior_seed=24,
                       dtype=np.float32) - np.float32(0.5)
    uk = oracle_mod.jacobi(u, 5)
    rn, bn, rel = oracle_mod.residual(uk)
    with jg.Jacobi3D((nx, ny, nz), ("shape", (16, 16, 16)), "f32") as s:
        s.set_state(u)
        s.step(5)
        grel, gabs = s.residual()
    assert abs(gabs[0] - rn) <= 1e-12 * rn and abs(grel[0] - rel) <= 1e-12 * rel


def test_widen_f32_exhaustive():
    # every binary32 bit pattern, on the device, bit for bit (NaN stays NaN)
    assert jg.jacobi_selftest_widen() == 0


def test_div6_f32_exhaustive():
    """The FP32 update's RN(s / 6) (one multiply and one fused multiply-add,
    with the division itself outside that form's proven domain) equals the
    division instruction sequence on all 2^32 binary32 inputs, bit for bit."""
    assert jg.jacobi_selftest_div6() == 0


def test_fp32_tiny_and_signed_values_divide_exactly(oracle_mod):
    """FP32 states whose neighbour sums fall outside the two-operation
    division's domain (|s| < 2^-121, negative zeros) take the exact fallback:
    iterates still equal the FP32 oracle's RN(s / 6) bit for bit, sign of zero
    included."""
    nx, ny, nz = 21, 13, 9
    u = J.initial_grid(nx, ny, nz, "uniform", bc_seed=13, interior="uniform", interior_seed=14,
                       dtype=np.float32)
    u = (u - np.float32(0.5)) * np.float32(2.0 ** -118)  # sums straddle 2^-121 and change sign
    u[:, :, : nx // 2] = np.float32(-0.0)
    with jg.Jacobi3D((nx, ny, nz), ("shape", (8, 8, 8)), "f32") as s:
        s.set_state(u)
        s.step(3)
        got = s.copy_out()
    want = J.interior_of(oracle_mod.jacobi(u, 3))
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
