"""The instrumented build (per-field read/write counts and per-word heatmaps, the paper's
Sec. 5) against counts the oracle fixes exactly.

Per type t, with S_t steps, P_t primaries and Q_t secondaries from the oracle:
- every step reads each of the 15 leaves once: reads[t][f] = S_t;
- dense double buffer: every survivor and secondary is written whole, and every track
  dies once, so writes[t][f] = (S_t - P_t - Q_t) + Q_t = S_t - P_t;
- sparse single buffer: position, interaction lengths, step, time, length and flags are
  rewritten for each survivor and written for each secondary (S_t - P_t); id and event
  only for secondaries (Q_t);
- the heatmap counts 4-byte words: 16 per record read or written.
Instrumentation must not change the results, and the counts do not depend on the layout.
"""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import assert_strict_parity, oracle_run, run_gpu

pytestmark = pytest.mark.gpu

LEAVES_ALWAYS = [0, 1, 2, 7, 10, 12, 13, 14]   # x y z nia step time len flags
ID, EVENT = 8, 9


@pytest.fixture(scope="module")
def ref(geom):
    p = W.small_electrons(8, 500.0)
    return p, oracle_run(geom, p, 8)


def _trace(g):
    from paper_2302_08252_gb300 import et
    return et.et_read_field_trace(g["ctx"]).astype(np.int64)


@pytest.mark.parametrize("layout", ["aos", "soa", "aosoa32"])
def test_dense_trace_and_heatmap(geom, ref, layout):
    from paper_2302_08252_gb300 import et
    p, o = ref
    g = run_gpu(geom, p, 8, form="dense", layout=layout, driver="persistent", instrument=True,
                capacity_log2=14)
    assert_strict_parity(g, o)
    tr = _trace(g)
    S = o["steps"].astype(np.int64)
    P = np.bincount(p["type"], minlength=3).astype(np.int64)
    for t in range(3):
        assert np.all(tr[t, :, 0] == S[t]), (t, tr[t, :, 0], S[t])
        assert np.all(tr[t, :, 1] == S[t] - P[t]), (t, tr[t, :, 1], S[t] - P[t])
    cap = 1 << 14
    for t in range(3):
        heat = sum(et.et_read_heatmap(g["ctx"], t, h, cap).astype(np.int64).sum() for h in (0, 1))
        assert heat == 16 * (2 * S[t] - P[t])


def test_sparse_trace(geom, ref):
    p, o = ref
    g = run_gpu(geom, p, 8, form="sparse", layout="aos", driver="hostloop", instrument=True,
                capacity_log2=16)
    assert_strict_parity(g, o)
    tr = _trace(g)
    S = o["steps"].astype(np.int64)
    Q = o["secondaries"].astype(np.int64)
    P = np.bincount(p["type"], minlength=3).astype(np.int64)
    for t in range(3):
        assert np.all(tr[t, :, 0] == S[t])
        assert np.all(tr[t, LEAVES_ALWAYS, 1] == S[t] - P[t])
        assert tr[t, ID, 1] == Q[t] and tr[t, EVENT, 1] == Q[t]
        # writes skewed, reads uniform (paper Sec. 5)
        assert tr[t, :, 1].min() < tr[t, :, 1].max()


def test_trace_is_layout_independent(geom, ref):
    p, o = ref
    a = _trace(run_gpu(geom, p, 8, form="sparse", layout="aos", instrument=True, capacity_log2=16))
    b = _trace(run_gpu(geom, p, 8, form="sparse", layout="soa", instrument=True, capacity_log2=16))
    assert np.array_equal(a, b)
