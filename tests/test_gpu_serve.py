"""Serving (continuous batching) on the GPU.

* every served result equals a standalone jacobi_solve of the same grid and
  the oracle's solve: same iteration count and status, bit-identical final
  iterate (FP64 and FP32 states are both computed in the oracle's order);
* a request's result is bit-identical alone and in a mix of others;
* admission by HBM budget: with room for one grid at a time everything still
  completes, one by one, with the same results;
* malformed requests are rejected at submission.
"""
import time

import numpy as np
import pytest

import jacobi_inputs as J
import paper_2102_12416_gb300 as jg

pytestmark = pytest.mark.gpu

RES_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2102_12416_gb300 import _build
    _build.build()
    jg.load()


def _wait(s, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = jg.serve_poll(s, t)
                if r is not None:
                    out[t] = r
        if time.time() - t0 > timeout:
            raise TimeoutError(f"{len(tickets) - len(out)} requests still pending")
        time.sleep(0.002)
    return [out[t] for t in tickets]


REQS = [((24, 16, 40), ("shape", (16, 16, 16)), dict(bc="uniform", bc_seed=(2 << 32) | 1, interior="zero")),
        ((32, 32, 32), ("count", (2, 2, 2)), dict(bc="linear_noise", bc_seed=1001, noise_amp=1e-3, interior="zero")),
        ((20, 28, 12), ("shape", (8, 8, 8)), dict(bc="uniform", bc_seed=77, interior="uniform", interior_seed=78)),
        ((37, 21, 30), ("shape", (32, 32, 32)), dict(bc="linear_noise", bc_seed=1003, noise_amp=1e-3,
                                                     interior="zero"))]


def _serve(reqs, dtype, tol, cap, check, budget=8 << 30, slots=16):
    npdt = np.float64 if dtype == "f64" else np.float32
    s = jg.serve_create(budget, slots, dtype, check_every=check, round_checks=2)
    try:
        outs = [np.zeros(g[::-1], dtype=npdt) for g, _, _ in reqs]
        tickets = [jg.serve_submit(s, g, sp, ini, tol, cap, out=o) for (g, sp, ini), o in zip(reqs, outs)]
        res = _wait(s, tickets)
        stats = jg.serve_stats(s)
    finally:
        jg.serve_destroy(s)
    return res, outs, stats


def test_served_equals_standalone_and_oracle_f64(oracle_mod):
    tol, cap, check = 1e-8, 5000, 50
    res, outs, stats = _serve(REQS, "f64", tol, cap, check)
    assert stats.completed == len(REQS)
    for (g, sp, ini), r, o in zip(REQS, res, outs):
        with jg.Jacobi3D(g, sp, "f64", ini) as h:
            it, rel, st = h.solve(tol, cap, check)
            alone = h.copy_out()
        # a handle splits its blocks into more work items than the server does,
        # so only the residual's summation order differs
        assert (r.iters, r.status) == (it[0], st[0])
        assert abs(r.rel - rel[0]) <= RES_TOL * rel[0]
        assert np.array_equal(o, alone)
        want, k, orel, ost = oracle_mod.solve(J.initial_grid(*g, **ini), tol, cap, check)
        assert (r.iters, r.status) == (k, ost)
        assert abs(r.rel - orel) <= RES_TOL * orel
        assert np.array_equal(o, J.interior_of(want))


def test_alone_equals_mix_f32(oracle_mod):
    tol, cap, check = 1e-6, 20000, 100
    mix, mix_out, _ = _serve(REQS, "f32", tol, cap, check)
    for q in range(len(REQS)):
        alone, alone_out, _ = _serve([REQS[q]], "f32", tol, cap, check)
        a, m = alone[0], mix[q]
        assert (a.iters, a.status, a.rel) == (m.iters, m.status, m.rel)
        assert np.array_equal(alone_out[0], mix_out[q])
    # FP32 state arithmetic follows the FP32 oracle's order exactly
    g, sp, ini = REQS[1]
    want, k, orel, ost = oracle_mod.solve(J.initial_grid(*g, dtype=np.float32, **ini), tol, cap, check)
    assert (mix[1].iters, mix[1].status) == (k, ost)
    assert np.array_equal(mix_out[1], J.interior_of(want))


def test_budget_serialises_admission():
    tol, cap, check = 1e-6, 20000, 100
    free, free_out, _ = _serve(REQS, "f32", tol, cap, check)
    biggest = max(jg.jacobi_workspace_bytes(g, sp, "f32") for g, sp, _ in REQS)
    one, one_out, stats = _serve(REQS, "f32", tol, cap, check, budget=biggest + 1024)
    assert stats.completed == len(REQS)
    for a, b, x, y in zip(free, one, free_out, one_out):
        assert (a.iters, a.status, a.rel) == (b.iters, b.status, b.rel)
        assert np.array_equal(x, y)
    # serialised: each request was admitted only after the previous one finished
    for prev, nxt in zip(one, one[1:]):
        assert nxt.t_admit_ns >= prev.t_done_ns - 1


def test_rejects_bad_requests():
    s = jg.serve_create(1 << 30, 4, "f32", check_every=100)
    try:
        with pytest.raises(jg.JacobiError):
            jg.serve_submit(s, (16, 16, 16), ("count", (1, 1, 1)), None, 1e-6, 150)  # cap not a multiple
        with pytest.raises(jg.JacobiError):
            jg.serve_submit(s, (2048, 2048, 2048), ("shape", (64, 64, 64)), None, 1e-6, 1000)  # over budget
        with pytest.raises(jg.JacobiError):
            jg.serve_poll(s, 12345)
    finally:
        jg.serve_destroy(s)


def _bench_stream(indices, n=400):
    """Requests of the serving benchmark's own stream (FP32 state, 32^3
    blocks, noisy linear boundary), by index."""
    import bench
    c = bench.SERVE_CFG
    reqs = J.serving_requests(n)
    return [(reqs[i]["grid"], ("shape", c["block"]),
             dict(bc="linear_noise", bc_seed=reqs[i]["seed"], noise_amp=c["noise_amp"], interior="zero"))
            for i in indices], c


def test_bench_stream_small_requests_vs_oracle(oracle_mod):
    """The benchmark stream's requests with every side <= 56, served together
    with bench settings, equal the FP32 oracle's solve: same iterations and
    status, bit-identical final iterate, residual within 1e-12."""
    reqs = J.serving_requests(400)
    idx = [i for i, r in enumerate(reqs) if max(r["grid"]) <= 56][:8]
    sample, c = _bench_stream(idx)
    res, outs, _ = _serve(sample, "f32", c["tol"], c["cap"], c["check_every"], slots=32)
    for (g, sp, ini), r, o in zip(sample, res, outs):
        want, k, orel, ost = oracle_mod.solve(J.initial_grid(*g, dtype=np.float32, **ini), c["tol"], c["cap"],
                                              c["check_every"])
        assert (r.iters, r.status) == (k, ost), g
        assert abs(r.rel - orel) <= RES_TOL * orel, g
        assert np.array_equal(o, J.interior_of(want)), g


def test_bench_stream_large_requests_vs_standalone():
    """The stream's larger requests (every side >= 80), served together, equal
    standalone solves of the same grids on a handle (whose iterates the
    parity tests pin to the oracle): same iterations and status, bit-identical
    final iterate, residual within 1e-12."""
    reqs = J.serving_requests(200)
    idx = [i for i, r in enumerate(reqs) if min(r["grid"]) >= 80][:5]
    sample, c = _bench_stream(idx, 200)
    res, outs, _ = _serve(sample, "f32", c["tol"], c["cap"], c["check_every"], slots=32)
    for (g, sp, ini), r, o in zip(sample, res, outs):
        with jg.Jacobi3D(g, sp, "f32", ini) as h:
            it, rel, st = h.solve(c["tol"], c["cap"], c["check_every"])
            alone = h.copy_out()
        assert (r.iters, r.status) == (it[0], st[0]), g
        assert abs(r.rel - rel[0]) <= RES_TOL * rel[0], g
        assert np.array_equal(o, alone), g
