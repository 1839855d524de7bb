"""The toy model v2 (multiple scattering of e+-) on the GPU against the oracle's v2,
through the C ABI: strict mode bit-exact (per-iteration counts, steps, secondaries, the
sorted death records; deposits to 1e-6), on the 16 x 1 GeV electrons for every layout of
the dense form and every driver, the sparse form, the split step kernels, a mixed-type
case, and the whole 1,000 x 10 GeV shower in the bench's launch configuration; fast mode
against the FP64 oracle within 3 standard errors and 1 %; a snapshot taken mid-run
resumes to the same histories; and the state rules of et_load_msc."""
import numpy as np
import pytest

import oracle
from paper_2302_08252_gb300 import workloads as W

from parity import assert_strict_parity, ledger_residual, oracle_run, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_v2(geom):
    p = W.small_electrons()
    return p, oracle_run(geom, p, 16, msc=True)


@pytest.mark.parametrize("driver", ["hostloop", "graph", "persistent", "hybrid"])
@pytest.mark.parametrize("layout", ["aos", "soa", "aosoa32", "aosoa64", "hotcold"])
def test_small_electrons_dense_bit_exact(geom, small_v2, layout, driver):
    p, o = small_v2
    kw = {"hybrid_tracks": 1 << 10} if driver == "hybrid" else {}
    g = run_gpu(geom, p, 16, form="dense", layout=layout, driver=driver, capacity_log2=17,
                msc=True, **kw)
    assert_strict_parity(g, o)
    assert ledger_residual(g["ledger"]) < 1e-12
    assert g["totals"]["iterations"] == o["n_iters"]


@pytest.mark.parametrize("driver", ["hostloop", "persistent"])
def test_small_electrons_sparse_bit_exact(geom, small_v2, driver):
    p, o = small_v2
    g = run_gpu(geom, p, 16, form="sparse", layout="aos", driver=driver, capacity_log2=20,
                msc=True)
    assert_strict_parity(g, o)


@pytest.mark.parametrize("form", ["dense", "sparse"])
def test_split_step_kernels_bit_exact(geom, small_v2, form):
    p, o = small_v2
    g = run_gpu(geom, p, 16, form=form, layout="aosoa32", driver="graph",
                capacity_log2=17 if form == "dense" else 20, msc=True, split=True)
    assert_strict_parity(g, o)


def test_mixed_types_bit_exact(geom):
    p = W.mixed_primaries(200)
    p["ekin"] = np.minimum(p["ekin"], np.float32(3000.0))
    o = oracle_run(geom, p, 200, msc=True)
    for form, layout, driver, cap in (("dense", "aosoa64", "hybrid", 20),
                                      ("sparse", "aos", "hostloop", 22)):
        g = run_gpu(geom, p, 200, form=form, layout=layout, driver=driver, capacity_log2=cap,
                    msc=True, id_log_capacity=1 << 24)
        assert_strict_parity(g, o)


def test_full_jittered_electrons(geom):
    """The whole 1,000 x 10 GeV shower under v2 (about 290 M track-steps), dense form,
    AoSoA-64 and the hybrid driver (AoSoA-32 is covered by the small cases): everything
    but the death records."""
    p = W.jittered_electrons()
    o = oracle_run(geom, p, 1000, idlog=False, nthreads=16, msc=True)
    g = run_gpu(geom, p, 1000, form="dense", layout="aosoa64", driver="hybrid",
                capacity_log2=22, id_log=False, msc=True)
    assert_strict_parity(g, o, check_idlog=False)
    assert ledger_residual(g["ledger"]) < 1e-12
    assert int(o["steps"].sum()) > 2.5e8


def test_fast_mode_statistics(geom):
    n = 600
    p = W.mixed_primaries(n)
    p["ekin"] = np.minimum(p["ekin"], np.float32(3000.0))
    o = oracle_run(geom, p, n, idlog=False, nthreads=16, mode=oracle.REF_FP64, msc=True)
    g = run_gpu(geom, p, n, form="dense", layout="aosoa32", driver="persistent",
                capacity_log2=21, id_log=False, mode=1, msc=True)
    a = g["score"].reshape(n, -1, 2).sum(2)
    b = o["score"].reshape(n, -1, 2).sum(2)
    se = np.sqrt(a.var(0, ddof=1) / n + b.var(0, ddof=1) / n)
    d = np.abs(a.mean(0) - b.mean(0))
    assert np.all(d <= 3 * se + 1e-9)
    big = b.mean(0) >= 0.01 * b.mean(0).sum()
    assert np.all(d[big] / b.mean(0)[big] <= 0.01)


def test_snapshot_resume(geom, small_v2):
    from paper_2302_08252_gb300 import et
    p, o = small_v2
    ctx = et.make_context(geom, max_events=16, capacity_log2=17, form=et.FORM_DENSE,
                          layout="aosoa32", driver="persistent", msc=True)
    et.et_inject(ctx, p)
    et.et_run_until_empty(ctx, 40)
    snap = et.et_snapshot(ctx)
    ctx2 = et.make_context(geom, max_events=16, capacity_log2=17, form=et.FORM_DENSE,
                           layout="aosoa32", driver="persistent", msc=True)
    et.et_restore(ctx2, snap)
    et.et_run_until_empty(ctx2)
    assert et.et_read_counters(ctx2)["steps"] == [int(x) for x in o["steps"]]
    v1 = et.make_context(geom, max_events=16, capacity_log2=17, form=et.FORM_DENSE,
                         layout="aosoa32", driver="persistent")
    with pytest.raises(et.EtError):
        et.et_restore(v1, snap)  # another configuration


def test_load_msc_state_rules(geom):
    from paper_2302_08252_gb300 import et
    x0 = et.et_toy_radiation_lengths()
    assert list(x0) == [np.float32(5.612), np.float32(140.0)]
    ctx = et.et_create(max_events=4, capacity_log2=10, msc=True)
    et.et_create_geometry(ctx, geom["thickness"], geom["material"], geom["half_xy"])
    t = et.et_build_toy_tables()
    with pytest.raises(et.EtError) as e:
        et.et_load_msc(ctx, x0)          # before the tables
    assert e.value.status == et.ET_ERR_STATE
    et.et_load_tables(ctx, t["sigma"], t["dedx"], t["log_emin"], t["inv_dlog"])
    with pytest.raises(et.EtError) as e:
        et.et_inject(ctx, W.small_electrons(4))   # radiation lengths missing
    assert e.value.status == et.ET_ERR_STATE
    with pytest.raises(et.EtError) as e:
        et.et_load_msc(ctx, np.array([5.6, -1.0], np.float32))
    assert e.value.status == et.ET_ERR_INVALID
    et.et_load_msc(ctx, x0)
    with pytest.raises(et.EtError) as e:
        et.et_load_msc(ctx, x0)          # once
    assert e.value.status == et.ET_ERR_STATE
    et.et_inject(ctx, W.small_electrons(4))
    v1 = et.make_context(geom, max_events=4, capacity_log2=10)
    with pytest.raises(et.EtError) as e:
        et.et_load_msc(v1, x0)           # not a multiple-scattering context
    assert e.value.status == et.ET_ERR_STATE
