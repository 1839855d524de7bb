"""GPU parity against the oracle, through the C ABI (strict mode: bit-exact histories).

Sizes: the 16 x 1 GeV electron case (~150k steps, 178 iterations, up to ~2,000 active
tracks: many warps per iteration with ragged tails) on every form x layout x driver; a
mixed-type case (e-, e+, photons); the full 1,000 x 10 GeV jittered case (92 M steps) in
the configuration the benchmark times, compared on everything the oracle produces.
"""
import numpy as np
import pytest

import oracle
from paper_2302_08252_gb300 import workloads as W

from parity import assert_strict_parity, ledger_residual, oracle_run, run_gpu

pytestmark = pytest.mark.gpu

FORMS = ["sparse", "dense"]
LAYOUTS = ["aos", "soa", "aosoa8", "aosoa16", "aosoa32", "aosoa64", "aosoa128", "hotcold"]
DRIVERS = ["hostloop", "graph", "persistent"]


@pytest.fixture(scope="module")
def small_ref(geom):
    p = W.small_electrons()
    return p, oracle_run(geom, p, 16)


@pytest.mark.parametrize("driver", DRIVERS)
@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("form", FORMS)
def test_small_electrons_bit_exact(geom, small_ref, form, layout, driver):
    p, o = small_ref
    g = run_gpu(geom, p, 16, form=form, layout=layout, driver=driver,
                capacity_log2=16 if form == "dense" else 18)
    assert_strict_parity(g, o)
    assert ledger_residual(g["ledger"]) < 1e-12
    assert g["totals"]["iterations"] == o["n_iters"]


@pytest.mark.parametrize("form", FORMS)
def test_mixed_types_bit_exact(geom, form):
    p = W.mixed_primaries(64)
    p["ekin"] = np.minimum(p["ekin"], np.float32(5000.0))
    o = oracle_run(geom, p, 64)
    g = run_gpu(geom, p, 64, form=form, layout="soa", driver="persistent", capacity_log2=19)
    assert_strict_parity(g, o)
    assert ledger_residual(g["ledger"]) < 1e-12


@pytest.mark.parametrize("block_size", [64, 128, 256])
def test_block_sizes_bit_exact(geom, small_ref, block_size):
    p, o = small_ref
    g = run_gpu(geom, p, 16, form="dense", layout="aosoa32", driver="persistent",
                block_size=block_size)
    assert_strict_parity(g, o)


def test_run_iteration_steps_one_at_a_time(geom, small_ref):
    from paper_2302_08252_gb300 import et
    p, o = small_ref
    ctx = et.make_context(geom, max_events=16, capacity_log2=16, form=et.FORM_DENSE)
    et.et_inject(ctx, p)
    counts = []
    while True:
        s = et.et_run_iteration(ctx)
        if s["steps"] == 0:
            break
        counts.append(s["steps"])
        if sum(s["n_active"]) == 0:
            break
    assert counts == [int(x) for x in o["counts"].sum(1)]


def test_score_reads_agree(geom, small_ref):
    """Scores read one event at a time, all at once and a second time give the same
    values; events injected after a completed run and a read add their deposits to their
    own rows; everything matches the oracle."""
    from paper_2302_08252_gb300 import et
    p, o = small_ref
    ns = len(geom["thickness"])
    ctx = et.make_context(geom, max_events=16, capacity_log2=16, form=et.FORM_DENSE,
                          driver="persistent")
    et.et_inject(ctx, p[p["event"] < 8])
    et.et_run_until_empty(ctx)
    first, _ = et.et_read_scoring_all(ctx, 16, ns)
    et.et_inject(ctx, p[p["event"] >= 8])   # a second batch adds to the folded scores
    et.et_run_until_empty(ctx)
    all1, _ = et.et_read_scoring_all(ctx, 16, ns)
    all2, _ = et.et_read_scoring_all(ctx, 16, ns)
    assert np.array_equal(all1, all2)
    assert np.array_equal(all1[:8], first[:8])
    for ev in (0, 9, 15):
        dep, _ = et.et_read_scoring(ctx, ev, ns)
        assert np.array_equal(dep, all1[ev])
    ref = o["score"]
    assert np.all(np.abs(all1 - ref) <= 1e-6 * np.abs(ref) + 1e-9)


def test_full_jittered_electrons(geom):
    """1,000 x 10 GeV electrons, dense AoSoA-32, persistent driver: all outputs vs oracle."""
    p = W.jittered_electrons()
    o = oracle_run(geom, p, 1000, nthreads=16)
    g = run_gpu(geom, p, 1000, form="dense", layout="aosoa32", driver="persistent",
                capacity_log2=21, id_log=True, id_log_capacity=1 << 25)
    assert_strict_parity(g, o)
    assert ledger_residual(g["ledger"]) < 1e-12


@pytest.mark.parametrize("threshold", [1, 300, 4000])
def test_hybrid_driver_bit_exact(geom, small_ref, threshold):
    """Persistent kernel below the threshold, graph of per-type kernels above it, switching
    back and forth as the showers grow and die out: the same histories."""
    from paper_2302_08252_gb300 import et
    p, o = small_ref
    ctx_kw = dict(hybrid_tracks=threshold)
    g = run_gpu(geom, p, 16, form="dense", layout="aosoa32", driver="hybrid", **ctx_kw)
    assert_strict_parity(g, o)


def test_hybrid_driver_full_jittered(geom):
    p = W.jittered_electrons()
    o = oracle_run(geom, p, 1000, nthreads=16)
    g = run_gpu(geom, p, 1000, form="dense", layout="aosoa32", driver="hybrid",
                capacity_log2=21, id_log=True, id_log_capacity=1 << 25)
    assert_strict_parity(g, o)


@pytest.mark.parametrize("driver", ["hostloop", "graph", "persistent", "hybrid"])
def test_dense_slot_high_water_is_the_peak_fill(geom, small_ref, driver):
    """Dense form: the reported high-water mark per type is the largest number of tracks any
    iteration wrote to the next buffer, i.e. the maximum of the counts log after the
    first (injected) row -- on every driver, also when the run is done in slices."""
    from paper_2302_08252_gb300 import et
    p, o = small_ref
    ctx = et.make_context(geom, max_events=16, capacity_log2=16, form=et.FORM_DENSE,
                          layout="aosoa32", driver=driver, hybrid_tracks=300)
    et.et_inject(ctx, p)
    et.et_run_until_empty(ctx, 17)
    et.et_run_until_empty(ctx, 40)
    et.et_run_until_empty(ctx)
    counts = et.et_read_iteration_counts(ctx).astype(np.int64)
    assert np.array_equal(counts, o["counts"].astype(np.int64))
    expect = counts[1:].max(axis=0)  # e-, e+, gamma
    assert et.et_read_counters(ctx)["slot_high_water"] == [int(x) for x in expect]


def test_empty_run_and_invalid_input(geom):
    from paper_2302_08252_gb300 import et
    ctx = et.make_context(geom, max_events=4, capacity_log2=10)
    t = et.et_run_until_empty(ctx)
    assert t["iterations"] == 0 and t["steps"] == 0
    bad = W.gun(1, 100.0)
    bad["pos"][0, 2] = -1.0
    with pytest.raises(et.EtError) as e:
        et.et_inject(ctx, bad)
    assert e.value.status == et.ET_ERR_INVALID
    bad = W.gun(1, 100.0)
    bad["event"] = 4
    with pytest.raises(et.EtError):
        et.et_inject(ctx, bad)


@pytest.mark.parametrize("form", FORMS)
def test_capacity_overflow_is_reported(geom, form):
    from paper_2302_08252_gb300 import et
    ctx = et.make_context(geom, max_events=16, capacity_log2=7,
                          form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE)
    et.et_inject(ctx, W.small_electrons())
    with pytest.raises(et.EtError) as e:
        et.et_run_until_empty(ctx)
    assert e.value.status == et.ET_ERR_CAPACITY
    # the context is reusable after a reset
    et.et_reset(ctx)
    et.et_inject(ctx, W.gun(1, 0.5, ptype=W.GAMMA))
    t = et.et_run_until_empty(ctx)
    assert t["steps"] > 0


def test_persistent_barrier_timeout_is_reported(geom, small_ref):
    """Host-side fault injection: one block never arrives at the grid barrier; the others
    give up after a bounded wait (0.2 s), record the timeout and return."""
    from paper_2302_08252_gb300 import et
    p, o = small_ref
    ctx = et.make_context(geom, max_events=16, capacity_log2=16, driver="persistent")
    et.et_debug_set_barrier_fault(ctx, 1, 200_000_000)
    et.et_inject(ctx, p)
    with pytest.raises(et.EtError) as e:
        et.et_run_until_empty(ctx)
    assert e.value.status == et.ET_ERR_TIMEOUT
    et.et_debug_set_barrier_fault(ctx, -1, 2_000_000_000)
    et.et_reset(ctx)
    et.et_inject(ctx, p)
    et.et_run_until_empty(ctx)
    assert et.et_read_counters(ctx)["steps"] == [int(x) for x in o["steps"]]
