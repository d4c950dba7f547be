"""Multi-GPU runs are independent per-GPU replicas (the grids are partitioned
by request, no halo crosses a GPU): the host logic that turns per-rank timings
into whole-job figures, and the reference arm's rank handling, run here as two
gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
# rank r took (r + 1) * 10 ms for (r + 1) * 1000 updates
ms, units = bench.replica_totals(dist, "cpu", (rank + 1) * 10.0, (rank + 1) * 1000)
print(json.dumps({"rank": rank, "world": world, "ms": ms, "units": units}), flush=True)
dist.barrier()
dist.destroy_process_group()
'''


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code_args, world=2, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(r), **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable, *code_args], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_replica_totals_two_gloo_ranks():
    pytest.importorskip("torch")
    import json
    outs = _launch(["-c", WORKER, ROOT])
    rows = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for row in rows:
        assert row["world"] == 2
        assert row["ms"] == 20.0          # the slowest rank's time
        assert row["units"] == 3000.0     # every rank's work


def test_replica_totals_single_process():
    import bench
    assert bench.replica_totals(None, "cpu", 12.5, 7) == (12.5, 7.0)


def test_reference_arm_only_rank0_reports(tmp_path):
    """Under two ranks the reference arm (the CPU oracle) runs on rank 0
    alone; the other rank exits 0 at once without output."""
    pytest.importorskip("torch")
    outs = _launch(["bench.py", "--impl", "reference", "--workload", "jacobi3d-fp64-64c-2x2x2",
                    "--steps", "1", "--warmup", "0", "--cpu-iters", "2"])
    import json
    line = json.loads([l for l in outs[0].splitlines() if l.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert outs[1].strip() == ""
