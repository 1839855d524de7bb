"""Autotuner for the batched transport: picks the track layout, the block size and the
per-type launch split for a workload by timing the candidates on a sample of it.

Launch splits:
  persistent   one cooperative kernel runs all particle types and all iterations
  hybrid       the persistent kernel for iterations below 2^21 active tracks, the graph
               (below) for the larger ones
  graph        one step kernel per particle type per iteration, captured once in a CUDA
               graph whose WHILE condition is set from the device
  hostloop     one step kernel per particle type per iteration, launched from the host
               after reading the counts back (the plain form)
Block sizes are 64-256: the step kernels use up to ~120 registers per thread, so larger
blocks would not fit a 64 K-register SM.

Every candidate computes the same histories (strict mode is bit-exact across layouts,
block sizes and drivers), so the choice affects speed only.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

LAYOUTS = ("aos", "soa", "aosoa8", "aosoa16", "aosoa32", "aosoa64", "aosoa128", "hotcold")
BLOCKS = (64, 128, 256)
DRIVERS = ("persistent", "graph", "hostloop", "hybrid")


def sample_events(primaries: np.ndarray, n_events: int, seed: int = 7) -> np.ndarray:
    """A random subset of events (numbers kept: the random streams are keyed by event)."""
    from . import workloads as W
    ev = np.unique(primaries["event"])
    rng = np.random.Generator(np.random.Philox(key=seed))
    pick = np.sort(rng.choice(ev, size=min(n_events, len(ev)), replace=False))
    return W.select_events(primaries, pick)


def time_config(geom, primaries, n_events, form, layout, block, driver, reps=3,
                capacity_log2=22, **ctx_kw) -> float:
    """Best-of-reps seconds for one complete run (GPU); ctx_kw: further context options."""
    import torch

    from . import et
    ctx = et.make_context(geom, max_events=n_events, capacity_log2=capacity_log2,
                          form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                          layout=layout, driver=driver, block_size=block, **ctx_kw)
    d = torch.from_numpy(primaries.view(np.uint8).copy()).cuda()
    best = float("inf")
    for r in range(reps + 1):
        et.et_reset(ctx)
        et.et_inject_device(ctx, d, len(primaries))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        et.et_run_until_empty(ctx)
        torch.cuda.synchronize()
        if r:  # the first run warms up
            best = min(best, time.perf_counter() - t0)
    return best


def autotune(geom, primaries, n_events, form="dense", layouts=LAYOUTS, blocks=BLOCKS,
             drivers=DRIVERS, sample=None, timer=None, reps=3, capacity_log2=22) -> dict:
    """Time every candidate and return {"best": {...}, "table": [...]}.  `sample`: tune on
    that many events of the workload.  `timer(layout, block, driver) -> seconds` replaces
    the GPU timing (tests)."""
    prim = primaries if sample is None else sample_events(primaries, sample)
    table = []
    for layout, block, driver in itertools.product(layouts, blocks, drivers):
        if timer is not None:
            t = timer(layout, block, driver)
        else:
            t = time_config(geom, prim, n_events, form, layout, block, driver, reps,
                            capacity_log2)
        table.append({"layout": layout, "block_size": block, "driver": driver, "seconds": t})
    best = min(table, key=lambda r: r["seconds"])
    return {"best": dict(best, form=form), "table": table, "tuned_on_events": int(
        len(np.unique(prim["event"])))}


def cached(path: str, key: str, compute):
    """Per-key result cache in a JSON file (e.g. key = GPU name + workload)."""
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    if key not in data:
        data[key] = compute()
        with open(path, "w") as f:
            json.dump(data, f, indent=1)
    return data[key]


def main(argv=None):
    """Tune on a sample of a workload's events, then time the chosen configuration and each
    driver at the default layout on the whole workload (GPU).

        python -m paper_2302_08252_gb300.autotune [--workload uneven] [--sample 32]
            [--capacity-log2 26] [--out FILE] [--write-tuned]
    """
    import argparse

    from . import study
    from . import workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="uneven", choices=["jittered", "small", "mixed", "uneven"])
    ap.add_argument("--sample", type=int, default=32)
    ap.add_argument("--capacity-log2", type=int, default=26)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=None)
    ap.add_argument("--write-tuned", action="store_true",
                    help="record the pick in tuned.json (the bench's default for the workload)")
    a = ap.parse_args(argv)
    geom = W.calorimeter()
    prim, n_events = study.workload(a.workload)
    tuned = autotune(geom, prim, n_events, sample=a.sample, reps=a.reps,
                     capacity_log2=min(a.capacity_log2, 24))  # a sample needs fewer slots
    b = tuned["best"]
    steps, _ = study.steps_of(geom, prim, n_events, "dense", b["layout"], b["driver"],
                              a.capacity_log2)
    full = []
    for layout, block, driver in [(b["layout"], b["block_size"], b["driver"]),
                                  ("aosoa32", 256, "persistent"), ("aosoa32", 256, "graph"),
                                  ("aosoa32", 256, "hostloop")]:
        t = time_config(geom, prim, n_events, "dense", layout, block, driver, a.reps,
                        a.capacity_log2)
        full.append({"layout": layout, "block_size": block, "driver": driver, "seconds": t,
                     "track_steps_per_s": steps / t})
        print(json.dumps(full[-1]), flush=True)
    res = {"workload": a.workload, "events": n_events, "primaries": int(len(prim)),
           "steps": steps, "tuned_on_events": tuned["tuned_on_events"], "best": b,
           "table": tuned["table"], "full": full}
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
    if a.write_tuned:
        from . import tuned as T
        n_cand = len(tuned["table"])
        T.write(a.workload, b, f"{tuned['tuned_on_events']}-event sample of the {a.workload}"
                f" workload, all {n_cand} candidates, best of {a.reps}",
                f"python -m paper_2302_08252_gb300.autotune --workload {a.workload}"
                f" --sample {a.sample} --write-tuned")
    return res


if __name__ == "__main__":
    main()
