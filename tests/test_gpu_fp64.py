"""All-FP64 GPU transport against the FP64 reference oracle, and the FP32-stepping path
against both (the precision comparison of the mixed-primary workload).

The FP64 build and the FP64 oracle evaluate the same toy model in FP64 with the same keyed
draws; their log/exp/sin/cos come from different libraries and may differ in the last
bit, which changes a discrete decision only with probability ~1e-13 per step, so on these
sizes the histories are identical: step counts and iteration counts are compared exactly,
deposits to 1e-9 relative (FP64 rounding and atomic summation order).  The FP32 strict path
follows other histories (FP32 rounding changes decisions), so against FP64 only statistics
agree: per-layer mean deposits within 3 standard errors and 1% relative on the layers that
hold at least 1% of the deposit, as for the fast mode.
"""
import numpy as np
import pytest

import oracle
from paper_2302_08252_gb300 import workloads as W

from parity import oracle_run, run_gpu

pytestmark = pytest.mark.gpu


def _fp64_gpu(geom, p, n_events, capacity_log2=20):
    from paper_2302_08252_gb300 import et
    return et.et_run_fp64(geom, et.et_build_toy_tables_fp64(), p, 1, n_events, capacity_log2)


def test_fp64_gpu_follows_fp64_oracle_histories(geom):
    n = 120
    p = W.mixed_primaries(n)
    p["ekin"] = np.minimum(p["ekin"], np.float32(5000.0))
    score, ledger, steps, iters = _fp64_gpu(geom, p, n)
    o = oracle_run(geom, p, n, idlog=False, nthreads=16, mode=oracle.REF_FP64)
    assert steps == int(o["steps"].sum())
    assert iters == o["n_iters"]
    e = p["ekin"].astype(np.float64)
    np.testing.assert_array_equal(ledger[:, 0], o["ledger"][:, 0])
    tol = 1e-9 * e[:, None]
    assert np.all(np.abs(score - o["score"]) <= tol)
    for k_gpu, k_or in ((1, 2), (2, 3), (3, 4), (4, 5)):  # cut, escaped, mass created/consumed
        assert np.all(np.abs(ledger[:, k_gpu] - o["ledger"][:, k_or]) <= 1e-9 * e)
    # the ledger closes: deposits + escaped = injected + mass created - mass consumed
    lhs = score.sum(1) + ledger[:, 2]
    rhs = ledger[:, 0] + ledger[:, 3] - ledger[:, 4]
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * e)


def test_fp64_gpu_rejects_bad_input(geom):
    from paper_2302_08252_gb300 import et
    p = W.gun(2, 100.0)
    p["event"][1] = 5
    with pytest.raises(et.EtError):
        et.et_run_fp64(geom, et.et_build_toy_tables_fp64(), p, 1, 2)
    p = W.gun(100, 100.0)
    with pytest.raises(et.EtError):  # 100 primaries of one type exceed 2^6 slots
        et.et_run_fp64(geom, et.et_build_toy_tables_fp64(), p, 1, 100, capacity_log2=6)
    with pytest.raises(et.EtError):  # in flight: 2 GeV showers outgrow 2^6 slots
        et.et_run_fp64(geom, et.et_build_toy_tables_fp64(), W.gun(8, 2000.0), 1, 8,
                       capacity_log2=6)


def test_fp32_stepping_statistics_against_fp64(geom):
    n = 400
    p = W.gun(n, 1000.0)
    o = oracle_run(geom, p, n, idlog=False, nthreads=16, mode=oracle.REF_FP64)
    g = run_gpu(geom, p, n, form="dense", layout="aosoa32", driver="persistent", mode=0,
                id_log=False, capacity_log2=17)
    score64, _, _, _ = _fp64_gpu(geom, p, n, capacity_log2=17)
    lo = o["score"].reshape(n, 50, 2).sum(2)
    for other in (g["score"], score64):
        lg = other.reshape(n, 50, 2).sum(2)
        se = np.sqrt(lo.var(0, ddof=1) / n + lg.var(0, ddof=1) / n)
        diff = lg.mean(0) - lo.mean(0)
        assert np.all(np.abs(diff) <= 3 * se + 1e-12), np.max(np.abs(diff) / (se + 1e-30))
        tot = lo.mean(0)
        big = tot >= 0.01 * tot.sum()
        assert np.all(np.abs(diff[big]) <= 0.01 * tot[big])
