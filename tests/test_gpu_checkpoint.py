"""Checkpoint / resume: a snapshot taken between iterations, restored into a fresh context
of the same configuration, continues with exactly the histories of the original run
(every draw is keyed by event, id and step), for every form and driver; snapshots of
another configuration or damaged ones are refused."""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import assert_strict_parity, oracle_run

pytestmark = pytest.mark.gpu


def _collect(ctx, n_events, n_slabs):
    from paper_2302_08252_gb300 import et
    score, ledger = et.et_read_scoring_all(ctx, n_events, n_slabs)
    return {"score": score, "ledger": ledger, "counts": et.et_read_iteration_counts(ctx),
            "counters": et.et_read_counters(ctx), "idlog": et.et_read_id_log(ctx)}


@pytest.mark.parametrize("form,layout,driver", [("dense", "aosoa32", "persistent"),
                                                ("dense", "soa", "hostloop"),
                                                ("dense", "aos", "hybrid"),
                                                ("sparse", "aos", "graph")])
def test_resume_follows_the_same_histories(geom, form, layout, driver):
    from paper_2302_08252_gb300 import et
    p = W.small_electrons()
    o = oracle_run(geom, p, 16)
    n_slabs = len(geom["thickness"])
    kw = dict(max_events=16, capacity_log2=18, layout=layout, driver=driver, id_log=True,
              id_log_capacity=1 << 20, hybrid_tracks=300,
              form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE)
    a = et.make_context(geom, **kw)
    et.et_inject(a, p)
    first = et.et_run_until_empty(a, 40)
    assert first["iterations"] == 40 and sum(first["n_active"]) > 0
    snap = et.et_snapshot(a)
    et.et_run_until_empty(a)
    b = et.make_context(geom, **kw)
    et.et_restore(b, snap)
    rest = et.et_run_until_empty(b)
    assert rest["iterations"] > 0
    for ctx in (a, b):
        assert_strict_parity(_collect(ctx, 16, n_slabs), o)


def test_serving_snapshot_with_slot_reuse(geom):
    """Sparse form with slot reuse under serving: events injected, snapshot mid-shower,
    the restored context completes the same events with the same deposits."""
    from paper_2302_08252_gb300 import et
    p = W.uneven_events(6, 20)
    p["ekin"] = np.minimum(p["ekin"], np.float32(3000.0))
    o = oracle_run(geom, p, 8, idlog=False)
    kw = dict(max_events=8, capacity_log2=20, form=et.FORM_SPARSE, layout="aos",
              driver="persistent", serving=True, reuse_slots=True)
    a = et.make_context(geom, **kw)
    et.et_inject(a, p)
    et.et_run_until_empty(a, 25)
    done_before = set(int(e) for e in et.et_poll_completed(a))
    snap = et.et_snapshot(a)
    b = et.make_context(geom, **kw)
    et.et_restore(b, snap)
    et.et_run_until_empty(b)
    done_after = set(int(e) for e in et.et_poll_completed(b))
    assert done_before.isdisjoint(done_after)
    assert done_before | done_after == set(int(e) for e in np.unique(p["event"]))
    score, _ = et.et_read_scoring_all(b, 8, len(geom["thickness"]))
    ref = o["score"]
    assert np.all(np.abs(score - ref) <= 1e-6 * np.abs(ref) + 1e-9)


def test_restore_refuses_other_configurations(geom):
    from paper_2302_08252_gb300 import et
    a = et.make_context(geom, max_events=4, capacity_log2=12, form=et.FORM_DENSE)
    et.et_inject(a, W.gun(2, 100.0))
    et.et_run_until_empty(a, 3)
    snap = et.et_snapshot(a)
    other = et.make_context(geom, max_events=4, capacity_log2=13, form=et.FORM_DENSE)
    with pytest.raises(et.EtError):
        et.et_restore(other, snap)
    same = et.make_context(geom, max_events=4, capacity_log2=12, form=et.FORM_DENSE)
    with pytest.raises(et.EtError):
        et.et_restore(same, snap[: len(snap) // 2])  # truncated
    with pytest.raises(et.EtError):
        et.et_restore(same, b"not a snapshot" + snap[14:])
    et.et_restore(same, snap)
    assert et.et_run_until_empty(same)["steps"] > 0
