"""Layout and driver study (the comparison of the paper's Sec. 4 figure): runtime of one
complete transport of a workload for every track-buffer form, layout and driver.

    python -m paper_2302_08252_gb300.study [--workload jittered|mixed|uneven|uneven32|small]
        [--forms dense sparse] [--layouts aos soa aosoa32 aosoa64]
        [--drivers hostloop persistent graph hybrid] [--hybrid-tracks-log2 17 21]
        [--split 0 1] [--reps 3] [--out FILE]

Prints one JSON object per candidate (track-steps/s, best-of-reps seconds) and writes
the list to --out.  The hybrid driver is timed once per threshold 2^k of
`--hybrid-tracks-log2` (default 2^21).  `--split 1` times the split step kernels (transport pass, then
per-process interaction passes) of the host-loop, graph and hybrid drivers.  Every
candidate computes the same histories in strict mode, so only the time differs.  GPU
required.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import autotune
from . import workloads as W


def workload(name: str):
    if name == "jittered":
        return W.jittered_electrons(), 1000
    if name == "small":
        return W.small_electrons(), 16
    if name == "mixed":
        return W.mixed_primaries(10000), 10000
    if name == "uneven":
        p = W.uneven_events(256, 1000)
        return p, 256
    if name == "uneven32":  # the first 32 of those events: a case small enough to profile
        p = W.uneven_events(256, 1000)
        return W.select_events(p, list(range(32))), 256
    raise ValueError(name)


def steps_of(geom, primaries, n_events, form, layout, driver, capacity_log2, **ctx_kw):
    """Track-steps of one complete run: the total and the per-type counts (e-, e+, gamma)."""
    from . import et
    ctx = et.make_context(geom, max_events=n_events, capacity_log2=capacity_log2,
                          form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                          layout=layout, driver=driver, **ctx_kw)
    et.et_inject(ctx, primaries)
    total = int(et.et_run_until_empty(ctx)["steps"])
    return total, [int(x) for x in et.et_read_counters(ctx)["steps"]]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="jittered",
                    choices=["jittered", "small", "mixed", "uneven", "uneven32"])
    ap.add_argument("--forms", nargs="+", default=["dense", "sparse"])
    ap.add_argument("--layouts", nargs="+", default=list(autotune.LAYOUTS))
    ap.add_argument("--drivers", nargs="+", default=["hostloop", "persistent"])
    ap.add_argument("--split", nargs="+", type=int, default=[0], choices=[0, 1])
    ap.add_argument("--hybrid-tracks-log2", nargs="+", type=int, default=[21])
    ap.add_argument("--block-size", type=int, default=256)
    ap.add_argument("--dense-capacity-log2", type=int, default=22)
    ap.add_argument("--sparse-capacity-log2", type=int, default=24)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    geom = W.calorimeter()
    prim, n_events = workload(a.workload)
    rows = []
    steps = by_type = None
    for form in a.forms:
        cap = a.dense_capacity_log2 if form == "dense" else a.sparse_capacity_log2
        for layout in a.layouts:
            for driver in a.drivers:
                for split, tk in [(sp, k) for sp in a.split
                                  for k in (a.hybrid_tracks_log2 if driver == "hybrid" else [0])]:
                    if split and driver == "persistent":
                        continue  # no split form of the persistent kernel
                    kw = {"split": True} if split else {}
                    if driver == "hybrid":
                        kw["hybrid_tracks"] = 1 << tk
                    if steps is None:
                        steps, by_type = steps_of(geom, prim, n_events, form, layout, driver, cap,
                                                  **kw)
                    t = autotune.time_config(geom, prim, n_events, form, layout, a.block_size,
                                             driver, reps=a.reps, capacity_log2=cap, **kw)
                    r = {"workload": a.workload, "form": form, "layout": layout,
                         "driver": driver, "split": bool(split), "block_size": a.block_size,
                         "hybrid_tracks": kw.get("hybrid_tracks", 0),
                         "seconds": t, "steps": steps, "steps_by_type": by_type,
                         "track_steps_per_s": steps / t}
                    rows.append(r)
                    print(json.dumps(r), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
