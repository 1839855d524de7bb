"""Serving with continuous batching: events that arrive while others are on the GPU are
admitted as memory frees up, their work overlaps, and each event's result is the same
as when it runs alone (strict mode: the same per-step deposits, summed in another order,
so within the parity tolerance), for the dense form and for the sparse form with slot
reuse."""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import DEPOSIT_RTOL, oracle_run, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["dense", "sparse"])
def test_each_event_same_alone_and_in_the_mix(geom, form):
    from paper_2302_08252_gb300 import serving
    reqs = serving.poisson_requests(rate=3000.0, n_events=48, max_primaries=4)
    srv = serving.Server(geom, form=form, layout="aos", driver="persistent", capacity_log2=20,
                         max_events=64, iters_per_round=4)
    st = srv.serve(reqs, realtime=True)
    assert len(st.results) == len(reqs)
    assert st.max_inflight > 1          # requests overlapped on the device
    by_event = {r.event: r for r in st.results}
    for req in reqs[:12]:
        alone = run_gpu(geom, req.primaries, 64, form="dense", layout="aos", driver="hostloop",
                        id_log=False, capacity_log2=18)
        ref = alone["score"][req.event]
        got = by_event[req.event].score
        assert np.all(np.abs(got - ref) <= DEPOSIT_RTOL * np.abs(ref) + 1e-9)
        assert by_event[req.event].ledger["injected"] == alone["ledger"][req.event, 0]
    # and against the oracle for a few
    for req in reqs[:4]:
        o = oracle_run(geom, req.primaries, 64, idlog=False)
        ref = o["score"][req.event]
        got = by_event[req.event].score
        assert np.all(np.abs(got - ref) <= DEPOSIT_RTOL * np.abs(ref) + 1e-9)


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
