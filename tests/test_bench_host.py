"""Host-side pieces of bench.py (no GPU): the rule that ties committed ncu
counters to the kernel sources they were taken from, the CPU baseline's
sample, the reference arm's JSON line at one rank, the per-configuration
paths and tuner calls, and the full-size solve's flag."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_ncu_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    import bench
    (tmp_path / "profiles").mkdir()
    rec = {"workload": "w", "dram_bytes_per_launch": 123.0, "source_sha": "abc"}
    (tmp_path / "profiles" / "ncu_step_w.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "abc")
    assert bench.ncu_traffic("w")[0] == 123.0
    # counters taken from other kernel sources are not reported
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "def")
    assert bench.ncu_traffic("w")[0] is None
    assert bench.ncu_traffic("missing") == (None, None)


def test_kernel_source_hash_covers_the_step_kernel_sources(tmp_path, monkeypatch):
    import shutil
    import bench
    csrc = tmp_path / "paper_2102_12416_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2102_12416_gb300", "csrc"), csrc)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.kernel_source_sha()
    assert base == bench.kernel_source_sha()
    for name in ("step.cu", "common.cuh", "kernels.cuh"):
        p = csrc / name
        text = p.read_text()
        p.write_text(text + "\n")
        assert bench.kernel_source_sha() != base, name
        p.write_text(text)
    assert bench.kernel_source_sha() == base
    # host-only sources do not move it
    (csrc / "api.cu").write_text((csrc / "api.cu").read_text() + "\n")
    assert bench.kernel_source_sha() == base


def test_cpu_baseline_sample():
    import bench
    cb = bench.cpu_baseline("jacobi3d-fp64-64c-2x2x2", 2, single_thread=True)
    assert cb["kind"] == "oracle" and cb["unit"] == "GLUP/s" and cb["value"] > 0
    assert cb["cores"] >= 1 and cb["lups"] == 2 * 64 ** 3
    assert "2 of 100 iterations" in cb["sample"]
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0


def test_reference_arm_line_single_rank():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "jacobi3d-fp64-64c-2x2x2", "--steps", "2", "--warmup", "1", "--cpu-iters", "2"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["higher_is_better"] is True and line["unit"] == "GLUP/s" and line["dtype"] == "f64"
    assert line["config"]["workload"] == "jacobi3d-fp64-64c-2x2x2"
    assert line["e2e"] == {"value": line["value"], "unit": "GLUP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"


def test_instruction_roof_from_counters():
    """Per-pipe ceilings: executed warp instructions per launch over the pipe's
    peak issue rate x SMs x clock; the tightest pipe bounds the kernel."""
    import bench
    rec = {"inst_per_launch": {"alu": 4.0e8, "fp64": 1.5e7, "issue": 6.4e8},
           "peak_inst_per_sm_cycle": {"alu": 2.0, "fp64": 0.0625, "issue": 4.0}}
    roof = bench.instruction_roof(rec, 1 << 27, 2000.0, 100)
    t_alu = 4.0e8 / (2.0 * 100 * 2000e6)
    assert abs(roof["alu"]["bound_GLUPs"] - (1 << 27) / t_alu / 1e9) < 1e-9
    assert abs(roof["alu"]["thread_inst_per_lup"] - 32 * 4.0e8 / (1 << 27)) < 1e-9
    assert min(roof, key=lambda k: roof[k]["bound_GLUPs"]) == "fp64"
    assert bench.instruction_roof(None, 1, 2000.0, 100) is None
    assert bench.instruction_roof(rec, 1, None, 100) is None


def test_config_bench_paths_and_tuning(monkeypatch):
    """config_bench maps its path names onto handles and tuner calls: "auto"
    tunes everything from a graph-path handle, "persistent_tuned" tunes the
    shape for a persistent-path handle; every step is timed by events on the
    given stream (a fake library and fake events stand in for the GPU)."""
    import types
    import bench
    import jacobi_inputs as J
    made, tuned = [], []

    class FakeHandle:
        def __init__(self, grids, splits, dtype, inits, path="fused", stream=None):
            made.append(path)
            self.info = types.SimpleNamespace(zchunk=4, cw_cap=8, halo_bytes_per_iter=0)

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            return False

        def autotune(self, iters, path=None):
            tuned.append((iters, path))
            return {"path": path or "graph", "stages": 4}

        def step(self, n):
            pass

        def kind_items(self):
            return {"k": 1}

    class FakeEvent:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return 2.0  # ms

    jg = types.SimpleNamespace(Jacobi3D=FakeHandle)
    torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Event=FakeEvent))
    out = bench.config_bench(jg, J, torch, "jacobi3d-fp64-64c-2x2x2", None, 3, iters=10,
                             paths=("graph", "persistent_tuned", "auto"))
    assert made == ["graph", "persistent", "graph"]
    assert tuned == [(10, "persistent"), (10, None)]
    assert "autotune" not in out["graph"] and out["persistent_tuned"]["autotune"]["path"] == "persistent"
    # 64^3 points x 10 iterations per step, 2 ms per step
    assert abs(out["graph"]["GLUPs"] - 64 ** 3 * 10 / 2e-3 / 1e9) < 1e-9
    assert out["graph"]["us_per_iter"] == 2e3 / 10


def test_solve_full_flag_is_parsed(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--solve-full"])
    assert bench.parse_args().solve_full
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert not bench.parse_args().solve_full
