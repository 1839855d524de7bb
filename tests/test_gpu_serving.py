"""Serving with continuous batching through the library's native loop (et_serve_*):
events that arrive while others are on the GPU are admitted as memory frees up, their
work overlaps, and each event's result is the same as when it runs alone -- strict mode,
the same per-step deposits summed in another order, so within the parity tolerance --
for the dense form and for the sparse form with slot reuse.  Events are of realistic
size (100-160 mixed primaries each).  The serving run's total step count equals the sum
of the events' step counts alone (bit-exact), admission never overflows the buffers
(the status word stays clear), and a few events also match the oracle."""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import DEPOSIT_RTOL, oracle_run, run_gpu

pytestmark = pytest.mark.gpu


def _requests(n_events, rate, seed=5):
    """n_events events of 100-160 mixed primaries (energies capped at 2 GeV), Poisson
    arrivals at `rate` per second."""
    from paper_2302_08252_gb300 import serving
    sizes = 100 + (np.arange(n_events) * 37) % 61
    p = W.mixed_primaries(int(sizes.sum()), seed=seed)
    p["ekin"] = np.minimum(p["ekin"], np.float32(2000.0))
    p["event"] = np.repeat(np.arange(n_events, dtype=np.uint32), sizes)
    p = W.assign_ids(p)
    t = W.poisson_arrivals(rate, n_events, seed=W.ARRIVAL_SEED)
    return [serving.Request(i, float(t[i]), p[p["event"] == i]) for i in range(n_events)]


def _close(a, b):
    return np.all(np.abs(a - b) <= DEPOSIT_RTOL * np.abs(b) + 1e-9)


@pytest.mark.parametrize("form,driver", [("dense", "persistent"), ("sparse", "persistent"),
                                         ("dense", "hybrid")])
def test_each_event_same_alone_and_in_the_mix(geom, form, driver):
    # the hybrid driver with a low switch-over population runs the large rounds in the
    # graph of per-type step kernels
    from paper_2302_08252_gb300 import et, serving
    n_ev = 40
    reqs = _requests(n_ev, rate=2000.0)
    kw = {"hybrid_tracks": 1 << 12} if driver == "hybrid" else {}
    srv = serving.Server(geom, form=form, layout="aosoa32" if form == "dense" else "aos",
                         driver=driver, capacity_log2=20, max_events=64, iters_per_round=8, **kw)
    st = srv.serve(reqs, realtime=True)
    assert len(st.results) == n_ev and sorted(r.event for r in st.results) == list(range(n_ev))
    assert st.max_inflight > 1          # requests overlapped on the device
    assert et.et_read_counters(srv.ctx)["status"] == 0   # no buffer ever overflowed
    by_event = {r.event: r for r in st.results}
    steps_alone = 0
    for req in reqs:
        alone = run_gpu(geom, req.primaries, 64, form="dense", layout="aos", driver="hostloop",
                        id_log=False, capacity_log2=19)
        steps_alone += sum(alone["counters"]["steps"])
        got = by_event[req.event]
        assert _close(got.score, alone["score"][req.event]), req.event
        a = alone["ledger"][req.event]
        assert got.ledger["injected"] == a[0]
        for k, name in ((2, "below_cut"), (3, "escaped"), (4, "mass_created"),
                        (5, "mass_consumed")):
            assert got.ledger[name] == pytest.approx(a[k], rel=1e-9, abs=1e-9), (req.event, name)
    assert st.steps == steps_alone      # the same histories, step for step
    # and against the oracle for a few
    for req in reqs[:4]:
        o = oracle_run(geom, req.primaries, 64, idlog=False, nthreads=16)
        assert _close(by_event[req.event].score, o["score"][req.event])


def test_serving_admission_waits_for_memory(geom):
    """A capacity that holds only a few events' reserves: admission waits for completions,
    every event is served, and nothing overflows."""
    from paper_2302_08252_gb300 import et, serving
    reqs = _requests(24, rate=1e6, seed=6)           # all arrive at once
    srv = serving.Server(geom, form="dense", layout="aosoa32", driver="persistent",
                         capacity_log2=16, max_events=32, iters_per_round=8)
    need = [int(serving.reserve(r.primaries).max()) for r in reqs]
    assert max(need) < 0.9 * (1 << 16) < sum(need)  # they cannot all be in flight at once
    st = srv.serve(reqs, realtime=False)
    assert sorted(r.event for r in st.results) == list(range(24))
    assert et.et_read_counters(srv.ctx)["status"] == 0
    assert st.max_inflight >= 2


def test_sparse_slot_reuse_keeps_slots_bounded(geom):
    """Without reuse the sparse buffer needs a slot for every track ever created; with
    reuse, slots of dead tracks are handed out again, so the high-water mark stays far
    below the number of tracks."""
    from paper_2302_08252_gb300 import et
    p = W.small_electrons(16, 1000.0)
    o = oracle_run(geom, p, 16, idlog=False)
    ctx = et.make_context(geom, max_events=16, capacity_log2=18, form=et.FORM_SPARSE,
                          layout="aos", driver="persistent", reuse_slots=True)
    et.et_inject(ctx, p)
    et.et_run_until_empty(ctx)
    c = et.et_read_counters(ctx)
    assert c["steps"] == [int(x) for x in o["steps"]]
    score, _ = et.et_read_scoring_all(ctx, 16, len(geom["thickness"]))
    assert np.all(np.abs(score - o["score"]) <= DEPOSIT_RTOL * np.abs(o["score"]) + 1e-9)
    tracks = int(o["tracks"].sum())
    assert sum(c["slot_high_water"]) < tracks / 4


@pytest.mark.parametrize("driver", ["persistent", "hostloop"])
def test_serving_count_log_wraps(geom, driver):
    """A serving context runs for as long as requests keep coming: its iteration count log
    wraps instead of filling up (here 16 entries for a run of ~130 iterations)."""
    from paper_2302_08252_gb300 import et
    p = W.small_electrons(4, 1000.0)
    ctx = et.make_context(geom, max_events=4, capacity_log2=16, form=et.FORM_DENSE,
                          layout="aos", driver=driver, serving=True, max_iters=16)
    et.et_inject(ctx, p)
    tot = et.et_run_until_empty(ctx)
    assert tot["iterations"] > 16
    o = oracle_run(geom, p, 4, idlog=False)
    assert et.et_read_counters(ctx)["steps"] == [int(x) for x in o["steps"]]
    assert sorted(int(e) for e in et.et_poll_completed(ctx)) == [0, 1, 2, 3]
