"""Serving sweep (the serving configuration): p50/p99 arrival-to-result latency and
sustained track-steps/s against the Poisson arrival rate, for the tuned form and the plain
sparse single buffer under the same streams.  GPU required.

    python -m paper_2302_08252_gb300.serving_report [--rates 50 200 500 1000 2000]
        [--events 1000] [--warmup-frac 0.1] [--max-primaries 1000] [--out FILE]

Events follow the uneven-size distribution (1-1,000 primaries per event, log-uniform;
each primary 50/25/25 % e-/e+/gamma, 0.1-100 GeV).  `--max-primaries 1` gives the other
reading of the serving workload, one primary per event.  The first `warmup-frac` of the
events (by arrival) are left out of the quantiles.  Capacity: 2^24 track slots per type.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import serving
from . import workloads as W

FORMS = {"tuned": ("dense", "aosoa32", "persistent"), "plain": ("sparse", "aos", "hostloop")}


def run(rate: float, n_events: int, max_primaries: int, warmup_frac: float, form_key: str,
        capacity_log2: int = 24, tuned_driver: str = "persistent", iters_per_round: int = 16) -> dict:
    form, layout, driver = FORMS[form_key]
    if form_key == "tuned":
        driver = tuned_driver
    geom = W.calorimeter()
    reqs = serving.poisson_requests(rate, n_events, max_primaries=max_primaries)
    srv = serving.Server(geom, form=form, layout=layout, driver=driver,
                         capacity_log2=capacity_log2, max_events=max(1024, n_events),
                         iters_per_round=iters_per_round)
    st = srv.serve(reqs)
    skip = int(warmup_frac * n_events)
    kept = sorted(st.results, key=lambda r: r.arrival)[skip:]
    lat = np.array([r.latency for r in kept])
    gev = sum(float(r.primaries["ekin"].astype(np.float64).sum()) for r in reqs) / 1e3
    return {"rate_per_s": rate, "events": n_events, "max_primaries": max_primaries,
            "form": form, "layout": layout, "driver": driver,
            "offered_gev_per_s": gev / max(1e-9, reqs[-1].arrival),
            "p50_ms": 1e3 * float(np.quantile(lat, 0.5)),
            "p99_ms": 1e3 * float(np.quantile(lat, 0.99)),
            "steps_per_s": st.steps / st.wall, "steady_steps_per_s": st.steady_rate(),
            "wall_s": st.wall,
            "max_inflight": st.max_inflight, "rounds": st.rounds,
            "latency_events": int(len(lat))}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", type=float, nargs="+", default=[50, 200, 500, 1000, 2000])
    ap.add_argument("--events", type=int, default=1000)
    ap.add_argument("--max-primaries", type=int, default=1000)
    ap.add_argument("--warmup-frac", type=float, default=0.1)
    ap.add_argument("--forms", nargs="+", default=["tuned", "plain"])
    ap.add_argument("--tuned-driver", default="persistent",
                    choices=["persistent", "graph", "hostloop", "hybrid"])
    ap.add_argument("--iters-per-round", type=int, default=16)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    rows = []
    for rate in a.rates:
        for fk in a.forms:
            r = run(rate, a.events, a.max_primaries, a.warmup_frac, fk,
                    tuned_driver=a.tuned_driver, iters_per_round=a.iters_per_round)
            r["which"] = fk
            rows.append(r)
            print(json.dumps(r), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
