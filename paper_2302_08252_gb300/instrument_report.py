"""Instrumented runs of the memory-access study (paper Sec. 5): per-field read/write
counts of every track buffer and per-byte heatmaps, for the sparse single buffer in AoS
and SoA layout and the dense double buffer in AoS layout.

Workload as in the paper's heatmap run: 25 electrons of 10 GeV in 5 events (the paper
injects `-particles 25 -batch 5`), small buffers.  Writes into --out:
  heatmap_<form>_<layout>_<type>[_<half>].png   per-byte counts, one row per track (64 B)
  slots_<form>_<type>.png                         per-track-slot counts (slot utilisation)
  trace_<form>_<layout>.txt                       reads and writes per field and type
  summary.json                                    slots used, max counts per type, ...
With --full-trace, also the field trace of the whole 1,000 x 10 GeV jittered workload
(persistent driver; dense AoSoA-32 and sparse AoS):
  trace_full_<form>_<layout>.txt

Usage: python -m paper_2302_08252_gb300.instrument_report --out DIR [--full-trace]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

from . import et, heatmap
from . import workloads as W

TYPES = ("electrons", "positrons", "photons")


def heatmap_workload(n: int = 25, events: int = 5, ekin_mev: float = 10000.0) -> np.ndarray:
    p = W.gun(n, ekin_mev)
    p["event"] = (np.arange(n) // (n // events)).astype(np.uint32)
    return W.assign_ids(p)


def run(form: str, layout: str, capacity_log2: int, out: str, prim: np.ndarray) -> dict:
    """The events run one after another (the paper's batches): inject, run until empty."""
    geom = W.calorimeter()
    n_events = int(prim["event"].max()) + 1
    cap = 1 << capacity_log2
    ctx = et.make_context(geom, max_events=n_events, capacity_log2=capacity_log2,
                          form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                          layout=layout, driver="hostloop", instrument=True)
    tot = {"steps": 0, "iterations": 0}
    for e in range(n_events):
        et.et_inject(ctx, prim[prim["event"] == e])
        r = et.et_run_until_empty(ctx)
        tot["steps"] += r["steps"]
        tot["iterations"] += r["iterations"]
    tr = et.et_read_field_trace(ctx)
    with open(os.path.join(out, f"trace_{form}_{layout}.txt"), "w") as f:
        f.write(heatmap.trace_table(tr) + "\n")
    cnt = et.et_read_counters(ctx)
    res = {"steps": tot["steps"], "iterations": tot["iterations"],
           "slots_high_water": cnt["slot_high_water"], "trace": tr.astype(int).tolist(),
           "max_word_count": [], "front_fraction": []}
    halves = (0, 1) if form == "dense" else (0,)
    for t in range(3):
        words = sum(et.et_read_heatmap(ctx, t, h, cap).astype(np.uint64) for h in halves)
        per_slot = None
        if layout == "aos":
            per_slot = words.reshape(cap, 16).sum(1)
            used = int(np.count_nonzero(per_slot))
            n_rows = max(1, int(np.flatnonzero(per_slot).max()) + 1) if used else 1
            shown = min(((n_rows + 63) // 64) * 64, 64 * 4096)
            heatmap.write_png(os.path.join(out, f"slots_{form}_{t}.png"),
                              per_slot[:shown].reshape(-1, 64), scale=2)
            res.setdefault("slots_touched", []).append(used)
            # share of all accesses that fall in the first 10% of the used slot range
            cut = max(1, n_rows // 10)
            res["front_fraction"].append(float(per_slot[:cut].sum() / max(1, per_slot.sum())))
        extent = heatmap.used_extent(words)
        rows = heatmap.heatmap_rows(words, 64, n_bytes=max(64, ((extent + 63) // 64) * 64))
        heatmap.write_png(os.path.join(out, f"heatmap_{form}_{layout}_{t}.png"),
                          rows[: min(len(rows), 4096)], scale=2)
        res["max_word_count"].append(int(words.max()))
    return res


def full_trace(form: str, layout: str, capacity_log2: int, out: str) -> dict:
    """Per-field reads and writes over the whole jittered workload (one run)."""
    geom = W.calorimeter()
    prim = W.jittered_electrons()
    ctx = et.make_context(geom, max_events=len(prim), capacity_log2=capacity_log2,
                          form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                          layout=layout, driver="persistent", instrument=True)
    et.et_inject(ctx, prim)
    r = et.et_run_until_empty(ctx)
    tr = et.et_read_field_trace(ctx)
    with open(os.path.join(out, f"trace_full_{form}_{layout}.txt"), "w") as f:
        f.write(heatmap.trace_table(tr) + "\n")
    return {"steps": int(r["steps"]), "iterations": int(r["iterations"]),
            "trace": tr.astype(int).tolist()}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--sparse-capacity-log2", type=int, default=23)
    ap.add_argument("--dense-capacity-log2", type=int, default=17)
    ap.add_argument("--full-trace", action="store_true",
                    help="also trace the whole 1,000 x 10 GeV jittered workload")
    args = ap.parse_args(argv)
    os.makedirs(args.out, exist_ok=True)
    prim = heatmap_workload()
    summary = {}
    for form, layout in (("sparse", "aos"), ("sparse", "soa"), ("dense", "aos")):
        cl2 = args.dense_capacity_log2 if form == "dense" else args.sparse_capacity_log2
        summary[f"{form}_{layout}"] = run(form, layout, cl2, args.out, prim)
    for form in ("sparse", "dense"):
        heatmap.layout_svg(os.path.join(args.out, f"layout_{form}_aos.svg"), "aos")
    heatmap.layout_svg(os.path.join(args.out, "layout_soa.svg"), "soa", cap=4)
    heatmap.layout_svg(os.path.join(args.out, "layout_aosoa32.svg"), "aosoa32", n_tracks=2)
    if args.full_trace:
        summary["full_dense_aosoa32"] = full_trace("dense", "aosoa32", 21, args.out)
        summary["full_sparse_aos"] = full_trace("sparse", "aos", 24, args.out)
    with open(os.path.join(args.out, "summary.json"), "w") as f:
        json.dump(summary, f, indent=1)
    for k, v in summary.items():
        if k.startswith("full_"):
            print(k, "steps", v["steps"], "iterations", v["iterations"])
            continue
        print(k, "steps", v["steps"], "slots", v["slots_high_water"], "max", v["max_word_count"],
              "front", [round(x, 3) for x in v["front_fraction"]])


if __name__ == "__main__":
    main()
