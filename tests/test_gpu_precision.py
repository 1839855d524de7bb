"""Precision comparison on the mixed-primary workload (10,000 primaries: 50% e-, 25% e+,
25% photons, log-uniform 100 MeV - 100 GeV, 1 cm^2 spot; one event each), GPU needed.

Runs the same primaries through
  fp32     the tuned path: FP32 state and stepping (strict mode), FP64 deposits and ledger
  fp64     the all-FP64 GPU build
  oracle64 the FP64 reference oracle (CPU, all cores)
  oracle32 the strict FP32 oracle (CPU, all cores; the bit-exact target of fp32)
and computes, per layer (absorber + gap summed), the mean deposit per primary and its
standard error, each result's error against oracle64, and the run times.  As a test it
asserts the precision claims on the whole workload: fp32 bit-exact with oracle32 (steps
and per-iteration counts; deposits to 1e-6), fp64 on oracle64's histories (steps and
iterations), and fp32's and fp64's per-layer means within 3 standard errors and 1 % of
oracle64's on the layers holding at least 1 % of the deposit.  Run as a script it prints
the report as one JSON object:

    python tests/test_gpu_precision.py [--n 10000] [--out FILE]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)


import pytest


def precision_report(n=10000, capacity_log2=24):
    import torch

    import oracle
    from paper_2302_08252_gb300 import et
    from paper_2302_08252_gb300 import workloads as W
    from parity import run_gpu

    geom = W.calorimeter()
    p = W.mixed_primaries(n)
    e_in = p["ekin"].astype(np.float64)
    res = {"workload": f"{n} mixed primaries (50% e-, 25% e+, 25% gamma), 0.1-100 GeV "
                       "log-uniform, 1 cm^2 spot, one event each", "runs": {}}

    t = time.perf_counter()
    g = run_gpu(geom, p, n, form="dense", layout="aosoa32", driver="persistent", mode=0,
                id_log=False, capacity_log2=capacity_log2)
    torch.cuda.synchronize()
    res["runs"]["fp32"] = {"seconds": time.perf_counter() - t, "steps": int(sum(g["counters"]["steps"]))}
    t = time.perf_counter()
    s64, l64, steps64, it64 = et.et_run_fp64(geom, et.et_build_toy_tables_fp64(), p, 1, n,
                                             capacity_log2)
    res["runs"]["fp64"] = {"seconds": time.perf_counter() - t, "steps": int(steps64)}
    nth = os.cpu_count() or 1
    t = time.perf_counter()
    o64 = oracle.run(geom, p, n_events=n, seed=1, mode=oracle.REF_FP64, nthreads=nth)
    res["runs"]["oracle64"] = {"seconds": time.perf_counter() - t,
                               "steps": int(o64["steps"].sum()), "threads": nth}
    t = time.perf_counter()
    o32 = oracle.run(geom, p, n_events=n, seed=1, mode=oracle.STRICT_FP32, nthreads=nth)
    res["runs"]["oracle32"] = {"seconds": time.perf_counter() - t,
                               "steps": int(o32["steps"].sum()), "threads": nth}

    def layers(score):
        return score.reshape(n, -1, 2).sum(2)  # [event][layer]

    ref = layers(o64["score"])
    ref_mean = ref.mean(0)
    big = ref_mean >= 0.01 * ref_mean.sum()
    res["layer_mean_mev_oracle64"] = [float(x) for x in ref_mean]
    res["layer_se_mev_oracle64"] = [float(x) for x in ref.std(0, ddof=1) / np.sqrt(n)]
    for name, score in (("fp32", g["score"]), ("fp64", s64), ("oracle32", o32["score"])):
        lg = layers(score)
        diff = lg.mean(0) - ref_mean
        se = np.sqrt(ref.var(0, ddof=1) / n + lg.var(0, ddof=1) / n)
        ev = np.abs(score - o64["score"]) / e_in[:, None]
        res[name] = {
            "layer_rel_err_max_big_layers": float(np.max(np.abs(diff[big]) / ref_mean[big])),
            "layer_err_in_se_max": float(np.max(np.abs(diff) / np.maximum(se, 1e-300))),
            "total_deposit_rel_err": float(diff.sum() / ref_mean.sum()),
            "per_event_slab_abs_err_over_e_max": float(ev.max()),
            "steps_rel_diff": float(res["runs"][name]["steps"] / res["runs"]["oracle64"]["steps"] - 1.0),
        }
    # the bit-exact pair
    res["fp32_vs_oracle32"] = {
        "steps_equal": bool(g["counters"]["steps"] == [int(x) for x in o32["steps"]]),
        "counts_equal": bool(np.array_equal(g["counts"].astype(np.int64),
                                            o32["counts"].astype(np.int64))),
        "deposit_rel_err_max": float(np.max(np.abs(g["score"] - o32["score"]) /
                                            np.maximum(np.abs(o32["score"]), 1e-300))),
    }
    res["fp64_vs_oracle64"] = {"steps_equal": int(steps64) == int(o64["steps"].sum()),
                               "iterations": [int(it64), int(o64["n_iters"])]}
    return res


@pytest.mark.gpu
def test_precision_mixed_primaries():
    r = precision_report()
    assert r["fp32_vs_oracle32"]["steps_equal"] and r["fp32_vs_oracle32"]["counts_equal"]
    assert r["fp32_vs_oracle32"]["deposit_rel_err_max"] <= 1e-6
    assert r["fp64_vs_oracle64"]["steps_equal"]
    it = r["fp64_vs_oracle64"]["iterations"]
    assert it[0] == it[1]
    for name in ("fp32", "fp64", "oracle32"):
        assert r[name]["layer_err_in_se_max"] <= 3.0, name
        assert r[name]["layer_rel_err_max_big_layers"] <= 0.01, name
    assert r["fp64"]["per_event_slab_abs_err_over_e_max"] <= 1e-9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=10000)
    ap.add_argument("--out", default=None)
    ap.add_argument("--capacity-log2", type=int, default=24)
    a = ap.parse_args()
    line = json.dumps(precision_report(a.n, a.capacity_log2))
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
