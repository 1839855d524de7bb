"""Helpers shared by the GPU parity tests: run a workload through the C ABI and compare it
with the oracle (strict mode: bit-exact counts, steps, secondaries, death records;
per-slab deposits within 1e-6 relative)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2302_08252_gb300 import workloads as W

DEPOSIT_RTOL = 1e-6


def run_gpu(geom, primaries, n_events, form="dense", layout="aos", driver="hostloop",
            capacity_log2=16, id_log=True, mode=0, seed=1, instrument=False, block_size=256,
            id_log_capacity=None, **ctx_kw):
    from paper_2302_08252_gb300 import et
    n_slabs = len(geom["thickness"])
    ctx = et.make_context(geom, max_events=n_events, capacity_log2=capacity_log2,
                          form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                          layout=layout, driver=driver, mode=mode, seed=seed,
                          id_log=id_log,
                          id_log_capacity=(id_log_capacity or (1 << capacity_log2) * 8) if id_log else 0,
                          instrument=instrument, block_size=block_size, **ctx_kw)
    et.et_inject(ctx, primaries)
    tot = et.et_run_until_empty(ctx)
    score, ledger = et.et_read_scoring_all(ctx, n_events, n_slabs)
    out = {
        "ctx": ctx,
        "score": score,
        "ledger": ledger,
        "counts": et.et_read_iteration_counts(ctx),
        "counters": et.et_read_counters(ctx),
        "totals": tot,
    }
    if id_log:
        out["idlog"] = et.et_read_id_log(ctx)
    return out


def oracle_run(geom, primaries, n_events, idlog=True, nthreads=8, mode=oracle.STRICT_FP32,
               msc=False):
    return oracle.run(geom, primaries, n_events=n_events, seed=1, idlog=idlog, nthreads=nthreads,
                      mode=mode, msc=msc)


def sorted_records(log):
    return np.sort(log, order=["id", "steps", "type_death"])


def assert_strict_parity(g, o, check_idlog=True):
    # per-iteration per-type counts, bit-exact
    gc = g["counts"].astype(np.int64)
    oc = o["counts"].astype(np.int64)
    assert gc.shape == oc.shape, (gc.shape, oc.shape)
    assert np.array_equal(gc, oc)
    # totals
    assert g["counters"]["steps"] == [int(x) for x in o["steps"]]
    assert g["counters"]["secondaries"] == [int(x) for x in o["secondaries"]]
    assert g["counters"]["reject_cap_hits"] == o["reject_cap_hits"]
    # sorted multiset of (id, steps, type | death << 8)
    if check_idlog:
        gl, ol = sorted_records(g["idlog"]), sorted_records(o["idlog"])
        assert len(gl) == len(ol)
        assert np.array_equal(gl["id"], ol["id"])
        assert np.array_equal(gl["steps"], ol["steps"])
        assert np.array_equal(gl["type_death"], ol["type_death"])
    # deposits: same per-step FP64 values, summed in another order
    ref = o["score"]
    err = np.abs(g["score"] - ref)
    assert np.all(err <= DEPOSIT_RTOL * np.abs(ref) + 1e-9), float(np.max(err))
    # ledger: injected exactly; the others to summation order
    gl_, ol_ = g["ledger"], o["ledger"]
    assert np.array_equal(gl_[:, 0], ol_[:, 0])
    for k in range(1, 6):
        assert np.allclose(gl_[:, k], ol_[:, k], rtol=1e-9, atol=1e-9), k


def ledger_residual(ledger):
    src = ledger[:, 0] + ledger[:, 4]
    snk = ledger[:, 1] + ledger[:, 2] + ledger[:, 3] + ledger[:, 5]
    ok = src > 0
    return float(np.max(np.abs(src[ok] - snk[ok]) / src[ok])) if ok.any() else 0.0
