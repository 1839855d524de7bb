"""Continuous batching of shower events over the C ABI (the serving pattern).

Events arrive as a Geant4 offload hook would hand them over (each a set of primaries,
at an arrival time).  The server keeps a single transport context on the GPU and loops:

  1. admit waiting events whose arrival time has passed while their estimated track
     footprint fits the free track-buffer capacity (admission by memory), injecting all
     newly admitted events with one call;
  2. run a few transport iterations (the showers already in flight keep going, the new
     ones start: their work overlaps on the device);
  3. collect the events whose last track died (device-side live-track counters), read
     their per-layer deposits and ledgers, release their event numbers.

Latency is arrival -> results read on the host.  Every random draw is keyed by the
event number and the track's own step count, so an event's history does not depend on
when it was admitted or what else was in flight.
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

    def latency_quantiles(self, qs=(0.5, 0.99)):
        lat = np.array([r.latency for r in self.results])
        return {f"p{int(q * 100)}": float(np.quantile(lat, q)) for q in qs}


def reserve(primaries: np.ndarray) -> np.ndarray:
    """Estimated peak active tracks per type of one event."""
    gev = float(primaries["ekin"].astype(np.float64).sum()) / 1000.0
    return np.ceil(PEAK_PER_GEV * gev + 16.0)


class Server:
    def __init__(self, geom: dict, form: str = "dense", layout: str = "aos",
                 driver: str = "persistent", capacity_log2: int = 22, max_events: int = 1 << 14,
                 iters_per_round: int = 16, seed: int = 1, tables: dict | None = None):
        self.geom = geom
        self.n_slabs = len(geom["thickness"])
        self.capacity = 1 << capacity_log2
        self.iters = iters_per_round
        self.ctx = et.make_context(geom, max_events=max_events, tables=tables,
                                   capacity_log2=capacity_log2,
                                   form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                                   layout=layout, driver=driver, seed=seed, serving=True,
                                   reuse_slots=(form == "sparse"))

    def serve(self, requests: list[Request], realtime: bool = True) -> ServeStats:
        """Serve the requests (sorted by arrival).  realtime: arrivals follow the wall
        clock; otherwise every request is available at once (throughput mode)."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        inflight: dict[int, tuple[Request, float, np.ndarray]] = {}
        reserved = np.zeros(3)
        stats = ServeStats()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while pending or inflight:
            t = now()
            batch = []
            while pending and (not realtime or pending[0].arrival <= t):
                r = pending[0]
                need = reserve(r.primaries)
                if inflight and np.any(reserved + need > 0.9 * self.capacity):
                    break  # wait until memory frees up
                if r.event in inflight:
                    break
                pending.popleft()
                reserved += need
                inflight[r.event] = (r, t, need)
                batch.append(r.primaries)
            if batch:
                et.et_inject(self.ctx, np.concatenate(batch))
            stats.max_inflight = max(stats.max_inflight, len(inflight))
            if not inflight:
                if pending:  # idle until the next arrival
                    time.sleep(max(0.0, pending[0].arrival - now()))
                continue
            tot = et.et_run_until_empty(self.ctx, self.iters)
            stats.steps += tot["steps"]
            stats.rounds += 1
            for e in et.et_poll_completed(self.ctx):
                e = int(e)
                r, t_adm, need = inflight.pop(e)
                score, ledger = et.et_read_scoring(self.ctx, e, self.n_slabs)
                stats.results.append(Result(e, r.arrival, t_adm, now(), score, ledger))
                et.et_release_event(self.ctx, e)
                reserved -= need
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
