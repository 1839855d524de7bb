"""Continuous batching of shower events over the C ABI (the serving pattern).

Events arrive as a Geant4 offload hook would hand them over (each a set of primaries,
at an arrival time).  The server keeps one transport context on the GPU and drives the
library's native serving loop (et_serve_submit / et_serve_round, include/et.h):

  1. every arrived event is submitted with its reserve (estimated peak track slots per
     type); the library admits queued events in order while their reserves fit the free
     track-buffer capacity (admission by memory) and injects them;
  2. each round runs a few transport iterations with every shower in flight (new ones
     start while the others go on: their work overlaps on the device); after the round
     a scan of the active tracks marks the events that still have one, and a device
     kernel collects the events that have none left -- their per-layer deposits and
     ledgers -- into one buffer copied to pinned memory;
  3. a round returns the completions of the round before it: the GPU is already running
     the next round while the host admits and reads back.

Latency is arrival -> results on the host.  Every random draw is keyed by the event
number and the track's own step count, so an event's history does not depend on when it
was admitted or what else was in flight.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import et
from . import workloads as W

# Peak active tracks per GeV of event energy and per type (e-, e+, gamma), measured on
# the 1,000 x 10 GeV workload (295k, 84k, 787k at 10 TeV), times a safety factor.
PEAK_PER_GEV = np.array([29.5, 8.4, 78.7]) * 2.0


@dataclass
class Request:
    event: int                # event number (also the random-stream key): < max_events
    arrival: float            # seconds from the start of the stream
    primaries: np.ndarray     # PRIMARY_DTYPE records with .event == event


@dataclass
class Result:
    event: int
    arrival: float
    admitted: float
    done: float
    score: np.ndarray
    ledger: dict

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    steps: int = 0
    wall: float = 0.0
    max_inflight: int = 0
    rounds: int = 0
    timeline: list = field(default_factory=list)  # (time, steps so far, completions so far)

    def steady_rate(self, lo: float = 0.1, hi: float = 0.9) -> float:
        """Track-steps per second between the rounds that returned the lo and hi fractions
        of the completions: the sustained rate without the start-up and the final drain."""
        n = len(self.results)
        if n < 10 or len(self.timeline) < 3:
            return self.steps / max(self.wall, 1e-9)
        t = [x for x in self.timeline if x[2] >= lo * n]
        u = [x for x in self.timeline if x[2] >= hi * n]
        if not t or not u or u[0][0] <= t[0][0]:
            return self.steps / max(self.wall, 1e-9)
        return (u[0][1] - t[0][1]) / (u[0][0] - t[0][0])

    def latency_quantiles(self, qs=(0.5, 0.99), skip_frac: float = 0.1):
        """Latency quantiles over the events after the first skip_frac of the stream (by
        arrival): the warm-up, while the device fills, is left out."""
        res = sorted(self.results, key=lambda r: r.arrival)
        res = res[int(len(res) * skip_frac):] or res
        lat = np.array([r.latency for r in res])
        return {f"p{int(q * 100)}": float(np.quantile(lat, q)) for q in qs}


def reserve(primaries: np.ndarray) -> np.ndarray:
    """Estimated peak active tracks per type of one event."""
    gev = float(primaries["ekin"].astype(np.float64).sum()) / 1000.0
    return np.ceil(PEAK_PER_GEV * gev + 16.0)


class Server:
    def __init__(self, geom: dict, form: str = "dense", layout: str = "aos",
                 driver: str = "persistent", capacity_log2: int = 22, max_events: int = 1 << 14,
                 iters_per_round: int = 16, seed: int = 1, tables: dict | None = None,
                 **ctx_kw):
        self.geom = geom
        self.n_slabs = len(geom["thickness"])
        self.capacity = 1 << capacity_log2
        self.iters = iters_per_round
        self.ctx = et.make_context(geom, max_events=max_events, tables=tables,
                                   capacity_log2=capacity_log2,
                                   form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                                   layout=layout, driver=driver, seed=seed, serving=True,
                                   reuse_slots=(form == "sparse"), **ctx_kw)
        self.buf = et.ServeBuffers(self.ctx, self.n_slabs)

    def _collect(self, out, stats, submitted, t_done):
        events, rows, steps, inflight = out
        stats.steps += steps
        ns = self.n_slabs
        for e, row in zip(events, rows):
            r, t_sub = submitted.pop(int(e))
            score = row[:ns].copy()
            lg = row[ns:]
            ledger = {"injected": float(lg[0]), "below_cut": float(lg[1]),
                      "escaped": float(lg[2]), "mass_created": float(lg[3]),
                      "mass_consumed": float(lg[4]),
                      "deposited_cont": float(score.sum() - lg[1])}
            stats.results.append(Result(int(e), r.arrival, t_sub, t_done, score, ledger))
        stats.max_inflight = max(stats.max_inflight, inflight)

    def serve(self, requests: list[Request], realtime: bool = True) -> ServeStats:
        """Serve the requests (sorted by arrival).  realtime: arrivals follow the wall
        clock; otherwise every request is available at once (throughput mode)."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        submitted: dict[int, tuple[Request, float]] = {}
        stats = ServeStats()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while pending or submitted:
            t = now()
            while pending and (not realtime or pending[0].arrival <= t):
                r = pending.popleft()
                if r.event in submitted:  # its number is still in use: wait for it
                    pending.appendleft(r)
                    break
                et.et_serve_submit(self.ctx, r.primaries, r.event,
                                   reserve(r.primaries).astype(np.uint32))
                submitted[r.event] = (r, t)
            if not submitted:
                if pending:  # idle until the next arrival
                    time.sleep(max(0.0, pending[0].arrival - now()))
                continue
            out = et.et_serve_round(self.ctx, self.buf, self.iters)
            stats.rounds += 1
            t_done = now()
            self._collect(out, stats, submitted, t_done)
            stats.timeline.append((t_done, stats.steps, len(stats.results)))
        stats.wall = now()
        return stats


def poisson_requests(rate: float, n_events: int, max_primaries: int = 1000,
                     seed_arrivals: int = W.ARRIVAL_SEED, seed_events: int = W.PRIMARY_SEED,
                     first_event: int = 0) -> list[Request]:
    """Events of the uneven-size distribution (primaries per event log-uniform in
    [1, max_primaries], each primary 50/25/25 % e-/e+/gamma, 0.1-100 GeV log-uniform)
    arriving as a Poisson stream of the given rate."""
    arrivals = W.poisson_arrivals(rate, n_events, seed=seed_arrivals)
    p = W.uneven_events(n_events, max_primaries, seed=seed_events)
    p["event"] += np.uint32(first_event)
    p = W.assign_ids(p)
    return [Request(first_event + i, float(arrivals[i]), p[p["event"] == first_event + i])
            for i in range(n_events)]
