"""The benchmark's N>1 path on CPU: two gloo ranks (replicas of the workload, weak scaling).
Whole-job steps are summed over ranks and the time is the max over ranks; the reference
arm runs on rank 0 only and the other ranks exit without work."""
import os
import socket
import subprocess
import sys

import numpy as np
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
    ([], "uneven", None, 26),
    (["--config", "2"], "jittered", "persistent", 22),
    (["--config", "1"], "small", "persistent", 16),
    (["--config", "3"], "mixed", "hybrid", 24),
    (["--config", "4"], "uneven", None, 26),
    (["--config", "4", "--driver", "graph", "--capacity-log2", "25"], "uneven", "graph", 25),
])
def test_bench_workload_defaults(argv, workload, driver, cap):
    """Configuration numbers pick the workload (the batched events by default); layout,
    block size and driver default to the autotuner's pick for the workload where it has
    one (None above), else to the fastest measured driver; capacity per workload."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2302_08252_gb300 import tuned
    a = bench.parse_args(argv)
    t = tuned.config(workload)
    if driver is None:
        driver = t["driver"]
        assert (a.layout, a.block_size, a.form) == (t["layout"], t["block_size"], t["form"])
    assert (a.workload, a.driver, a.capacity_log2) == (workload, driver, cap)


def test_oracle_samples_are_bounded():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2302_08252_gb300 import workloads as W
    p = W.uneven_events(256, 1000)
    s, what = bench.oracle_sample("uneven", p, 256, reference=True)
    assert len(s) == (len(p) + 31) // 32 and "one primary in 32" in what
    assert np.array_equal(s["id"], p["id"][::32]) and np.array_equal(s["event"], p["event"][::32])
    s, _ = bench.oracle_sample("uneven", p, 256, reference=False)
    assert len(s) == (len(p) + 3) // 4
    q = W.jittered_electrons()
    s, what = bench.oracle_sample("jittered", q, 1000, reference=True)
    assert len(s) == 100 and what == "first 100 events"
    assert len(bench.oracle_sample("jittered", q, 1000, reference=False)[0]) == 1000
