"""Parity at the full sizes of the mixed and batched workloads, in the launch
configuration `bench.py --config 3` and `--config 4` time (dense, AoSoA-32, hybrid driver,
2^24 and 2^26 slots).

The 10,000 mixed primaries (1.29 G track-steps) are compared with the oracle on every
output but the death records.  For the 256 uneven events (5.36 G track-steps) the oracle
runs a sample of events on their own: an event's history does not depend on the other
events of the batch (every draw is keyed by event and track id), so each sampled event's
deposits and ledger must match.  Every event of the batch must close its energy ledger.
"""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import DEPOSIT_RTOL, assert_strict_parity, ledger_residual, oracle_run, run_gpu

pytestmark = pytest.mark.gpu


def test_full_mixed_primaries_hybrid(geom):
    p = W.mixed_primaries(10000)
    o = oracle_run(geom, p, 10000, idlog=False, nthreads=16)
    g = run_gpu(geom, p, 10000, form="dense", layout="aosoa32", driver="hybrid",
                capacity_log2=24, id_log=False)
    assert_strict_parity(g, o, check_idlog=False)
    assert ledger_residual(g["ledger"]) < 1e-12


def test_full_uneven_events_hybrid_sampled(geom):
    p = W.uneven_events(256, 1000)
    g = run_gpu(geom, p, 256, form="dense", layout="aosoa32", driver="hybrid",
                capacity_log2=26, id_log=False)
    assert ledger_residual(g["ledger"]) < 1e-12
    assert int(g["counters"]["steps"][0] + g["counters"]["steps"][1]
               + g["counters"]["steps"][2]) == 5_356_823_085
    # a sample across the event sizes: the smallest and largest events whose total energy
    # keeps the oracle (one thread per event) within seconds, and some in between
    e_tot = np.bincount(p["event"], weights=p["ekin"].astype(np.float64), minlength=256)
    n_prim = np.bincount(p["event"], minlength=256)
    ok = np.flatnonzero(e_tot <= 2.0e6)  # <= 2 TeV: at most about 2e7 track-steps
    by_size = ok[np.argsort(n_prim[ok], kind="stable")]
    sample = sorted(set(by_size[np.linspace(0, len(by_size) - 1, 8).astype(int)].tolist()))
    o = oracle_run(geom, W.select_events(p, sample), 256, idlog=False, nthreads=16)
    for ev in sample:
        ref, got = o["score"][ev], g["score"][ev]
        assert np.all(np.abs(got - ref) <= DEPOSIT_RTOL * np.abs(ref) + 1e-9), ev
        assert g["ledger"][ev, 0] == o["ledger"][ev, 0], ev
        assert np.allclose(g["ledger"][ev, 1:], o["ledger"][ev, 1:], rtol=1e-9, atol=1e-9), ev
