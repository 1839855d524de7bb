"""The benchmark's N>1 path on CPU: two gloo ranks (replicas of the workload, weak scaling).
Whole-job steps are summed over ranks and the time is the max over ranks; the reference
arm runs on rank 0 only and the other ranks exit without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank = dist.get_rank()
steps, secs = bench.aggregate(100.0 * (rank + 1), 1.0 + rank, dist)
print(json.dumps({{"rank": rank, "steps": steps, "secs": secs}}))
dist.destroy_process_group()
"""


def _launch(code, world=2):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    return procs, outs


def test_aggregate_sums_steps_and_takes_max_time():
    import json
    procs, outs = _launch(WORKER.format(root=ROOT))
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for r in res:
        assert r["steps"] == 300.0 and r["secs"] == 2.0


def test_reference_arm_runs_on_rank_zero_only():
    import json
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            "sys.exit(bench.main(['--impl', 'reference', '--workload', 'small', '--steps', '1', "
            "'--warmup', '0', '--gpus', '2']))")
    procs, outs = _launch(code)
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    lines = [[l for l in o.splitlines() if l.startswith("{")] for o, _ in outs]
    assert len(lines[0]) == 1 and lines[1] == []
    d = json.loads(lines[0][0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.parametrize("argv,workload,driver,cap", [
    ([], "jittered", "persistent", 22),
    (["--config", "1"], "small", "persistent", 16),
    (["--config", "3"], "mixed", "hybrid", 24),
    (["--config", "4"], "uneven", "hybrid", 26),
    (["--config", "4", "--driver", "graph", "--capacity-log2", "25"], "uneven", "graph", 25),
])
def test_bench_workload_defaults(argv, workload, driver, cap):
    """Configuration numbers pick the workload; the driver and capacity default per
    workload (the fastest measured driver) unless given."""
    sys.path.insert(0, ROOT)
    import bench
    a = bench.parse_args(argv)
    assert (a.workload, a.driver, a.capacity_log2) == (workload, driver, cap)
