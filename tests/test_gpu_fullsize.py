"""Parity at the full sizes of the mixed and batched workloads, in the launch
configurations `bench.py --config 3` and `--config 4` time (dense; AoSoA-32 and the hybrid
driver with 2^24 slots for the mixed primaries; the autotuner's layout, block size and
driver with 2^26 slots for the batched events).

The 10,000 mixed primaries (1.29 G track-steps) and the 256 uneven events (5.36 G
track-steps) are compared with the oracle, run on the whole workload, on every output but
the death records (which would take gigabytes at these sizes).  Every event of each batch
must close its energy ledger.
"""
import os

import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import assert_strict_parity, ledger_residual, oracle_run, run_gpu

pytestmark = pytest.mark.gpu


def test_full_mixed_primaries_hybrid(geom):
    p = W.mixed_primaries(10000)
    o = oracle_run(geom, p, 10000, idlog=False, nthreads=16)
    g = run_gpu(geom, p, 10000, form="dense", layout="aosoa32", driver="hybrid",
                capacity_log2=24, id_log=False)
    assert_strict_parity(g, o, check_idlog=False)
    assert ledger_residual(g["ledger"]) < 1e-12


def test_full_uneven_events_tuned(geom):
    # the whole batch, in the launch configuration the bench times (the autotuner's pick),
    # against the oracle run on every event: per-iteration per-type counts, steps,
    # secondaries and sampler-cap hits bit-exact, every event's deposits to 1e-6 and its
    # ledger to 1e-9
    from paper_2302_08252_gb300 import tuned
    t = tuned.config("uneven")
    p = W.uneven_events(256, 1000)
    o = oracle_run(geom, p, 256, idlog=False, nthreads=os.cpu_count() or 16)
    g = run_gpu(geom, p, 256, form="dense", layout=t["layout"], driver=t["driver"],
                block_size=t["block_size"], capacity_log2=26, id_log=False)
    assert_strict_parity(g, o, check_idlog=False)
    assert ledger_residual(g["ledger"]) < 1e-12
