"""The split step kernels against the oracle: per type, a transport pass that finishes the
steps without a discrete interaction and queues the others by process, then an interaction
pass over the queues (process-uniform warps).  The histories are those of the fused step,
so strict mode stays bit-exact on every form, layout and driver that runs the per-type
kernels (host loop, graph, and the graph phase of the hybrid driver)."""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import assert_strict_parity, ledger_residual, oracle_run, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_ref(geom):
    p = W.small_electrons()
    return p, oracle_run(geom, p, 16)


@pytest.mark.parametrize("driver", ["hostloop", "graph", "hybrid"])
@pytest.mark.parametrize("layout", ["aos", "soa", "aosoa32", "hotcold"])
@pytest.mark.parametrize("form", ["sparse", "dense"])
def test_split_small_electrons_bit_exact(geom, small_ref, form, layout, driver):
    p, o = small_ref
    g = run_gpu(geom, p, 16, form=form, layout=layout, driver=driver, split=True,
                hybrid_tracks=300, capacity_log2=16 if form == "dense" else 18)
    assert_strict_parity(g, o)
    assert ledger_residual(g["ledger"]) < 1e-12
    assert g["totals"]["iterations"] == o["n_iters"]


@pytest.mark.parametrize("form,reuse", [("sparse", False), ("sparse", True), ("dense", False)])
def test_split_mixed_types_bit_exact(geom, form, reuse):
    """e-, e+ and photons of 100 MeV-5 GeV: every one of the five process queues is used."""
    p = W.mixed_primaries(64)
    p["ekin"] = np.minimum(p["ekin"], np.float32(5000.0))
    o = oracle_run(geom, p, 64)
    g = run_gpu(geom, p, 64, form=form, layout="aosoa32", driver="graph", capacity_log2=19,
                split=True, reuse_slots=reuse)
    assert_strict_parity(g, o)
    assert ledger_residual(g["ledger"]) < 1e-12


def test_split_full_jittered_electrons(geom):
    """1,000 x 10 GeV electrons (92 M steps, queues of up to ~10^6 entries), dense AoSoA-32,
    graph driver: all outputs vs the oracle."""
    p = W.jittered_electrons()
    o = oracle_run(geom, p, 1000, nthreads=16)
    g = run_gpu(geom, p, 1000, form="dense", layout="aosoa32", driver="graph",
                capacity_log2=21, id_log=True, id_log_capacity=1 << 25, split=True)
    assert_strict_parity(g, o)
    assert ledger_residual(g["ledger"]) < 1e-12


def test_split_configurations_refused(geom):
    """The persistent kernel has no split form, and the split kernels are not instrumented."""
    from paper_2302_08252_gb300 import et
    for kw in (dict(driver="persistent"), dict(instrument=True)):
        with pytest.raises(et.EtError) as e:
            et.et_create(max_events=1, capacity_log2=10, split=True, **kw)
        assert e.value.status == et.ET_ERR_INVALID
