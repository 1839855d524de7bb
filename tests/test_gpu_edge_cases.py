"""Degenerate and boundary cases of the step, on the GPU against the oracle (strict mode,
bit-exact): directions parallel to the slab planes or the box faces (a limiter distance
of +inf), tracks on a plane or a box face, tracks leaving the box on their first step,
primaries below the tracking cut (e- and e+: annihilation at rest), photons just below
and just above the pair threshold, and energies at the ends of the cross-section tables.
Each primary is its own event; every form and driver runs the same list."""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import assert_strict_parity, ledger_residual, oracle_run, run_gpu

pytestmark = pytest.mark.gpu

E_M, E_P, G = W.E_MINUS, W.E_PLUS, W.GAMMA
S3 = np.float32(1.0 / np.sqrt(3.0))
# (type, MeV, position mm, direction)
CASES = [
    (E_M, 500.0, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0)),        # along +x: no plane ahead
    (G, 100.0, (0.0, 0.0, 1.0), (0.0, 1.0, 0.0)),           # photon along +y
    (E_M, 50.0, (0.0, 0.0, 0.0), (0.0, 0.0, -1.0)),         # leaves backwards at once
    (E_P, 0.005, (0.0, 0.0, 10.0), (0.0, 0.0, 1.0)),        # e+ below the cut: annihilates
    (E_M, 0.005, (0.0, 0.0, 10.0), (0.0, 0.0, 1.0)),        # e- below the cut
    (G, 1.0219, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0)),          # just below 2 m c^2
    (G, 1.0230, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0)),          # just above 2 m c^2
    (G, 0.001, (0.0, 0.0, 3.0), (0.0, 0.0, 1.0)),           # lowest table node
    (E_M, 1.0e5, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0)),         # highest table node
    (E_M, 1000.0, (199.9, 0.0, 0.0), (1.0, 0.0, 0.0)),      # next to the +x face, outwards
    (E_M, 1000.0, (-199.99, 5.0, 20.0), (-1.0, 0.0, 0.0)),  # next to the -x face, outwards
    (E_M, 300.0, (0.0, 0.0, 2.3), (0.0, 0.0, 1.0)),         # on a plane
    (G, 300.0, (200.0, 0.0, 0.0), (0.0, 0.0, 1.0)),         # on the +x face, parallel to it
    (E_M, 300.0, (0.0, 0.0, 399.0), (0.0, 0.0, 1.0)),       # last slab, forwards
    (G, 50.0, (0.0, 0.0, 0.0), (S3, S3, S3)),               # oblique
    (E_P, 200.0, (0.0, -200.0, 50.0), (0.0, -1.0, 0.0)),    # on the -y face, outwards
]


@pytest.fixture(scope="module")
def edge(geom):
    p = np.zeros(len(CASES), dtype=W.PRIMARY_DTYPE)
    for i, (ty, e, pos, d) in enumerate(CASES):
        p[i]["type"] = ty
        p[i]["event"] = i
        p[i]["ekin"] = np.float32(e)
        p[i]["pos"] = np.asarray(pos, dtype=np.float32)
        p[i]["dir"] = np.asarray(d, dtype=np.float32)
    p = W.assign_ids(p)
    return p, oracle_run(geom, p, len(CASES))


@pytest.mark.parametrize("driver", ["hostloop", "graph", "persistent"])
@pytest.mark.parametrize("form", ["sparse", "dense"])
def test_edge_cases_bit_exact(geom, edge, form, driver):
    p, o = edge
    g = run_gpu(geom, p, len(CASES), form=form, layout="aosoa32", driver=driver,
                capacity_log2=18 if form == "dense" else 21)
    assert_strict_parity(g, o)
    assert ledger_residual(g["ledger"]) < 1e-12
    assert g["totals"]["iterations"] == o["n_iters"]
