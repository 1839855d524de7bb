#!/usr/bin/env python3
"""Benchmark of the EM shower transport hot path (one JSON line on rank 0).

A step is one complete transport run of the workload (reset, inject, iterate until no
track is left).  The default workload is the batched one: 256 events of uneven size
(1-1,000 primaries each, log-uniform; mixed e-/e+/gamma of 0.1-100 GeV; 41,001 primaries,
5.36 G track-steps) into the 50-layer Pb/lAr calorimeter, in the tuned form (dense double
buffer, strict FP32 with FP64 scoring) with the layout, block size and driver the
autotuner picked for it (tuned.json in the package).  --config 1/2/3 select the small
gun, the 1,000 x 10 GeV electron shower and the 10,000 mixed primaries.  Reported:

  value         track-steps/s, primaries resident in device memory, L2 flushed between steps
  e2e           the same through the C ABI with host buffers (H2D of the primaries and D2H
                of the scores inside each timed step)
  roofline      the transport kernels against the HBM roofline: algorithmic bytes per run
                (64 B read per step + 64 B per survivor + 64 B per secondary = 64 (2 S - P))
                over their CUDA-event duration, against the measured copy bandwidth
  plain         the plain form (sparse single buffer, AoS, host loop) on the same workload
  cpu_baseline  the CPU oracle on the host cores

--impl reference times the CPU oracle (the reference arm of this build).  Under torchrun
each rank runs its own replica of the workload (independent events: weak scaling); the
time is the max over ranks and the value the steps of all ranks over that time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "track-steps/s and HBM GB/s (frac of peak), tuned vs plain; p99 event latency"
UNIT = "track-steps/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uneven", choices=["jittered", "small", "mixed", "uneven"])
    ap.add_argument("--config", type=int, default=None, choices=[1, 2, 3, 4],
                    help="the workload by number: 1 small, 2 jittered, 3 mixed, 4 uneven (default)")
    ap.add_argument("--form", default=None, choices=["dense", "sparse"])
    ap.add_argument("--layout", default=None, choices=["aos", "soa", "aosoa8", "aosoa16", "aosoa32",
                                                       "aosoa64", "aosoa128", "hotcold"],
                    help="default: the autotuner's pick for the workload, else aosoa32")
    ap.add_argument("--driver", default=None, choices=["hostloop", "graph", "persistent", "hybrid"],
                    help="default: the autotuner's pick for the workload, else persistent for"
                         " the single showers and hybrid for the mixed primaries")
    ap.add_argument("--mode", default="strict", choices=["strict", "fast"])
    ap.add_argument("--msc", action="store_true",
                    help="the toy model v2: multiple scattering of e+- (default: v1)")
    ap.add_argument("--block-size", type=int, default=None)
    ap.add_argument("--capacity-log2", type=int, default=None,
                    help="track slots per type: 2^N (default per workload: 16, 22, 24, 26)")
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--serving-events", type=int, default=1000)
    a = ap.parse_args(argv)
    if a.config is not None:
        a.workload = {1: "small", 2: "jittered", 3: "mixed", 4: "uneven"}[a.config]
    from paper_2302_08252_gb300 import tuned
    t = tuned.config(a.workload) or {}
    a.tuned = bool(t)
    if a.form is None:
        a.form = t.get("form", "dense")
    if a.layout is None:
        a.layout = t.get("layout", "aosoa32")
    if a.block_size is None:
        a.block_size = t.get("block_size", 256)
    if a.driver is None:
        a.driver = t.get("driver") or {"small": "persistent", "jittered": "persistent",
                                       "mixed": "hybrid", "uneven": "hybrid"}[a.workload]
    if a.capacity_log2 is None:
        a.capacity_log2 = {"small": 16, "jittered": 22, "mixed": 24, "uneven": 26}[a.workload]
    return a


# ------------------------------------------------------------------ distributed plumbing

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    group = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        group = dist
    return rank, world, local, group


def barrier(group):
    if group is not None:
        group.barrier()


def aggregate(local_steps: float, local_seconds: float, group):
    """Whole-job steps (sum over ranks) and time (max over ranks)."""
    if group is None:
        return local_steps, local_seconds
    import torch
    dev = "cuda" if torch.cuda.is_available() and group.get_backend() == "nccl" else "cpu"
    s = torch.tensor([local_steps], dtype=torch.float64, device=dev)
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    group.all_reduce(s, op=group.ReduceOp.SUM)
    group.all_reduce(t, op=group.ReduceOp.MAX)
    return float(s.item()), float(t.item())


# ------------------------------------------------------------------ inputs

def make_workload(name: str, rank: int, msc: bool = False):
    from paper_2302_08252_gb300 import workloads as W
    if name == "jittered":
        p = W.jittered_electrons(seed=W.PRIMARY_SEED + rank)
        desc = "1000 e- 10 GeV, 1 mrad jitter, 50x(2.3 mm Pb + 5.7 mm lAr)"
    elif name == "small":
        p = W.small_electrons()
        desc = "16 e- 1 GeV on +z, 50x(2.3 mm Pb + 5.7 mm lAr)"
    elif name == "mixed":
        p = W.mixed_primaries(10000, seed=W.PRIMARY_SEED + rank)
        desc = "10000 mixed e-/e+/gamma 0.1-100 GeV, 1 cm2 spot, 50x(2.3 mm Pb + 5.7 mm lAr)"
    else:
        p = W.uneven_events(256, 1000, seed=W.PRIMARY_SEED + rank)
        desc = ("256 events of 1-1000 mixed e-/e+/gamma primaries (0.1-100 GeV), "
                "50x(2.3 mm Pb + 5.7 mm lAr)")
    n_events = int(p["event"].max()) + 1
    if msc:
        desc += "; toy model v2 (multiple scattering of e+-)"
    return W.calorimeter(), p, n_events, desc


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples during the run (timestamps kept to select the timed window)."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if device_id:
            cmd += ["-i", device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return []
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                    rows.append({"t": ts + frac, "sm": float(parts[1]), "sm_max": float(parts[2]),
                                 "power": parts[3], "active": parts[4], "hw": parts[5],
                                 "hw_thermal": parts[6], "sw_thermal": parts[7],
                                 "sw_power": parts[8]})
                except (ValueError, IndexError):
                    continue
        os.unlink(self.out.name)
        return rows


def summarize_clocks(rows, t0, t1):
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
    inside = [r for r in rows if t0 - 0.05 <= r["t"] <= t1 + 0.05] or rows
    reasons = set()
    for r in inside:
        for key, name in (("hw", "hw_slowdown"), ("hw_thermal", "hw_thermal_slowdown"),
                          ("sw_thermal", "sw_thermal_slowdown"), ("sw_power", "sw_power_cap")):
            if r[key].lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(r["sm"] for r in inside),
            "sm_max_mhz": max(r["sm_max"] for r in inside), "reasons": sorted(reasons),
            "samples": len(inside)}


# ------------------------------------------------------------------ helpers

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes(steps: int, primaries: int) -> int:
    """64 B read per step, 64 B per survivor (steps - deaths), 64 B per secondary; every
    track dies once, so deaths = primaries + secondaries and the sum is 64 (2 S - P)."""
    return 64 * (2 * steps - primaries)


def committed_traffic(kernel_key: str):
    """DRAM bytes per track-step of the transport kernel from the committed ncu summary,
    only while the library sources are the ones it was measured on."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        from paper_2302_08252_gb300 import build
        if d.get("kernel_fingerprint") != build.kernel_fingerprint():
            return None
        return d.get("kernels", {}).get(kernel_key)
    except (OSError, ValueError):
        return None


def run_config(et, geom, prim, n_events, args, form, layout, driver, steps, warmup, flush,
               timing=True, reuse_slots=False):
    import torch
    # the sparse form without slot reuse needs room for every track of the run
    cap = args.capacity_log2 if form == "dense" else max(args.capacity_log2, 24)
    ctx = et.make_context(geom, max_events=n_events, capacity_log2=cap,
                          form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                          layout=layout, driver=driver,
                          mode=et.MODE_STRICT if args.mode == "strict" else et.MODE_FAST,
                          block_size=args.block_size, seed=1, reuse_slots=reuse_slots,
                          msc=args.msc)
    d_prim = torch.from_numpy(prim.view(np.uint8).copy()).cuda()
    n = len(prim)
    stream = torch.cuda.current_stream()

    def one():
        et.et_reset(ctx)
        et.et_inject_device(ctx, d_prim, n)
        return et.et_run_until_empty(ctx)

    for _ in range(warmup):
        one()
    et.et_set_timing(ctx, timing)
    et.et_read_timing(ctx)
    ms_steps, tot_steps, launches, iters = [], 0, 0, 0
    for _ in range(steps):
        flush.add_(1)  # write > L2 between timed steps
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tot = one()
        b.record(stream)
        b.synchronize()
        ms_steps.append(a.elapsed_time(b))
        tot_steps += tot["steps"]
        iters += tot["iterations"]
        launches += et.et_read_counters(ctx)["kernel_launches"]
    kms, klaunch = et.et_read_timing(ctx)
    return {"ctx": ctx, "ms": ms_steps, "steps": tot_steps, "launches": launches,
            "kernel_ms": kms, "kernel_launches": klaunch, "iterations": iters, "n_prim": n}


def e2e_measure(et, ctx, prim, n_events, n_slabs, steps):
    """Through the C ABI from host memory: each step resets the context, injects the
    primaries from a host array (the library stages them in pinned memory and copies them
    to the device), runs to completion and reads every event's deposits and ledger back
    into pinned host buffers."""
    import torch
    score = torch.empty((n_events, n_slabs), dtype=torch.float64, pin_memory=True).numpy()
    ledger = np.zeros((n_events, 6), dtype=np.float64)
    torch.cuda.synchronize()
    secs, tot = 0.0, 0
    h2d = prim.nbytes
    d2h = n_events * n_slabs * 8 + n_events * 5 * 8
    for k in range(steps + 1):  # the first pass warms up (pinned staging is allocated)
        t0 = time.perf_counter()
        et.et_reset(ctx)
        et.et_inject(ctx, prim)
        r = et.et_run_until_empty(ctx)
        et.et_read_scoring_all(ctx, n_events, n_slabs, out=(score, ledger))
        if k:
            secs += time.perf_counter() - t0
            tot += r["steps"]
    return tot, secs, h2d, d2h


def serving_measure(geom, args):
    """Continuous batching under a Poisson stream of uneven events (1-1000 primaries of
    mixed types, 0.1-100 GeV each) through the library's native serving loop: p50/p99
    arrival-to-result latency over the events after the first 10 % (warm-up) and
    sustained track-steps/s, tuned form (persistent driver, whatever --driver says: a
    round runs a few iterations, where one launch per round pays most) and the plain
    sparse single buffer on the same stream."""
    from paper_2302_08252_gb300 import serving
    reqs = serving.poisson_requests(args.serving_rate, args.serving_events)
    out = {"rate_per_s": args.serving_rate, "events": args.serving_events,
           "event_sizes": "primaries per event log-uniform 1-1000, 0.1-100 GeV each"}
    for name, form, layout, driver, cap in (("tuned", args.form, args.layout, "persistent", 22),
                                            ("plain", "sparse", "aos", "hostloop", 24)):
        srv = serving.Server(geom, form=form, layout=layout, driver=driver, capacity_log2=cap,
                             max_events=max(1024, args.serving_events), iters_per_round=16)
        st = srv.serve(reqs)
        q = st.latency_quantiles()
        out[name] = {"form": form, "layout": layout, "driver": driver,
                     "p50_ms": 1e3 * q["p50"], "p99_ms": 1e3 * q["p99"],
                     "steps_per_s": st.steps / st.wall, "steady_steps_per_s": st.steady_rate(),
                     "wall_s": st.wall,
                     "max_inflight": st.max_inflight, "rounds": st.rounds,
                     "latency_events": len(st.results) - int(0.1 * len(st.results))}
        del srv
    return out


def oracle_sample(workload: str, prim, n_events: int, reference: bool):
    """A bounded sample of the workload for the oracle (the CPU baseline, about 10-30 s on
    the host cores; the reference arm, about a second per step).  The batched events are
    sampled by primaries (every k-th, event numbers kept), so that the sample has the
    workload's per-primary mix and its events spread over all cores."""
    from paper_2302_08252_gb300 import workloads as W
    if workload == "uneven":
        k = 32 if reference else 4
        return prim[::k].copy(), f"one primary in {k} of the {len(prim)} (event numbers kept)"
    if reference and workload in ("jittered", "mixed"):
        m = 100 if workload == "jittered" else 1000
        return W.select_events(prim, list(range(min(m, n_events)))), f"first {m} events"
    return prim, "whole workload"


def cpu_baseline(geom, prim, n_events, workload, one_thread_primaries=50, msc=False):
    """The oracle on the host cores (a bounded sample of the workload on every core), and
    under "one_thread" its first one_thread_primaries primaries on one thread."""
    import oracle
    sample, what = oracle_sample(workload, prim, n_events, reference=False)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.run(geom, sample, n_events=n_events, seed=1, nthreads=cores, msc=msc)
    dt = time.perf_counter() - t0
    steps = int(r["steps"].sum())
    sample1 = sample[:one_thread_primaries].copy()
    t1 = time.perf_counter()
    r1 = oracle.run(geom, sample1, n_events=n_events, seed=1, nthreads=1, msc=msc)
    dt1 = time.perf_counter() - t1
    steps1 = int(r1["steps"].sum())
    return {"value": steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} ({len(sample)} primaries, {steps} steps) on {cores} threads,"
                      f" {dt:.2f} s wall",
            "one_thread": {"value": steps1 / dt1, "unit": UNIT, "cores": 1,
                           "sample": f"first {len(sample1)} primaries of that sample ({steps1}"
                                     f" steps) on 1 thread, {dt1:.2f} s"}}


# ------------------------------------------------------------------ arms

def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    geom, prim, n_events, desc = make_workload(args.workload, 0, args.msc)
    # a bounded sample: about a second of host-core work per step
    sample, what = oracle_sample(args.workload, prim, n_events, reference=True)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.run(geom, sample, n_events=n_events, seed=1, nthreads=cores, msc=args.msc)
    secs, steps = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.run(geom, sample, n_events=n_events, seed=1, nthreads=cores, msc=args.msc)
        secs += time.perf_counter() - t0
        steps += int(r["steps"].sum())
    value = steps / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": desc, "sample": what, "sample_primaries": int(len(sample)),
                   "mode": "strict",
                   "implementation": "CPU oracle (plain C, depth-first per event)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{what} per step ({len(sample)} primaries,"
                                   f" {steps // max(1, args.steps)} steps) on {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ours_arm(args, rank, world, group):
    import torch

    from paper_2302_08252_gb300 import et
    dev = torch.cuda.current_device()
    geom, prim, n_events, desc = make_workload(args.workload, rank, args.msc)
    n_slabs = len(geom["thickness"])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = None if args.no_clocks else ClockSampler(uuid)

    barrier(group)
    torch.cuda.synchronize()
    t_wall0 = time.time()
    tuned = run_config(et, geom, prim, n_events, args, args.form, args.layout, args.driver,
                       args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier(group)
    clock_rows = sampler.stop() if sampler else []

    secs = sum(tuned["ms"]) / 1e3
    all_steps, max_secs = aggregate(float(tuned["steps"]), secs, group)
    value = all_steps / max_secs
    steps_per_run = tuned["steps"] // args.steps

    peak, peak_kind = measured_hbm_peak()
    alg_per_launch = None
    achieved = None
    if tuned["kernel_launches"]:
        per_launch_ms = tuned["kernel_ms"] / tuned["kernel_launches"]
        # with the persistent driver one launch is one run; otherwise bytes are split evenly
        runs_per_launch = args.steps / tuned["kernel_launches"]
        alg_per_launch = algorithmic_bytes(steps_per_run, tuned["n_prim"]) * runs_per_launch
        achieved = alg_per_launch / (per_launch_ms / 1e3) / 1e9
    key = (f"{args.workload}/{args.mode}/{args.form}/{args.layout}/{args.driver}" +
           ("/msc" if args.msc else ""))
    tr = committed_traffic(key)
    traffic = tr * steps_per_run * (args.steps / max(1, tuned["kernel_launches"])) if tr else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_secs * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": desc, "form": args.form, "layout": args.layout,
                   "driver": args.driver, "mode": args.mode, "block_size": args.block_size,
                   "physics": "toy model v2 (multiple scattering)" if args.msc else "toy model v1",
                   "steps_per_run": steps_per_run,
                   "iterations_per_run": tuned["iterations"] // args.steps,
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "hbm_gbs_alg_whole_step": algorithmic_bytes(steps_per_run, tuned["n_prim"]) /
        (secs / args.steps) / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": f"transport kernel ({key})",
                     "alg_bytes_per_launch": alg_per_launch},
        "gpu_launches": tuned["launches"],
    }

    barrier(group)
    if args.e2e_steps > 0:
        e2e_steps, e2e_secs, h2d, d2h = e2e_measure(et, tuned["ctx"], prim, n_events, n_slabs,
                                                    args.e2e_steps)
        e2e_all, e2e_max = aggregate(float(e2e_steps), e2e_secs, group)
        line["e2e"] = {"value": e2e_all / e2e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h}
    if rank == 0 and world == 1:
        if not args.no_plain:
            # the large workloads create more tracks than a sparse buffer without reuse
            # can hold: there the plain form reuses the slots of dead tracks
            reuse = args.workload in ("mixed", "uneven")
            plain = run_config(et, geom, prim, n_events, args, "sparse", "aos", "hostloop",
                               args.plain_steps, 1, flush, timing=False, reuse_slots=reuse)
            pv = plain["steps"] / (sum(plain["ms"]) / 1e3)
            line["plain"] = {"value": pv, "unit": UNIT, "form": "sparse", "layout": "aos",
                             "driver": "hostloop", "steps": args.plain_steps,
                             "reuse_slots": reuse}
            line["tuned_vs_plain"] = value / pv
        if not args.no_serving and not args.msc:
            line["serving"] = serving_measure(geom, args)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(geom, prim, n_events, args.workload, msc=args.msc)
    line["clocks"] = summarize_clocks(clock_rows, t_wall0, t_wall1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    rank, world, local, group = dist_setup(args)
    try:
        if args.impl == "reference":
            return reference_arm(args, rank, world)
        return ours_arm(args, rank, world, group)
    finally:
        if group is not None:
            group.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
