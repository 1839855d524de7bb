"""Autotuner: selection logic and sampling on CPU; on the GPU, tuning a batched workload of
uneven events and checking that the chosen configuration reproduces the oracle."""
import numpy as np
import pytest

from paper_2302_08252_gb300 import autotune
from paper_2302_08252_gb300 import workloads as W


def test_selection_picks_fastest_and_covers_all_candidates():
    cost = {"aos": 3.0, "soa": 2.0, "aosoa8": 1.8, "aosoa16": 1.4, "aosoa32": 1.0,
            "aosoa64": 1.5, "aosoa128": 1.7, "hotcold": 1.2}
    timer = lambda layout, block, driver: cost[layout] + {64: 0.3, 128: 0.1, 256: 0.2}[block] + \
        {"persistent": 0.0, "graph": 1.0, "hostloop": 2.0, "hybrid": 0.5}[driver]
    r = autotune.autotune(None, W.uneven_events(8, 5), 8, timer=timer)
    assert len(r["table"]) == 8 * 3 * 4
    assert r["best"]["layout"] == "aosoa32" and r["best"]["block_size"] == 128
    assert r["best"]["driver"] == "persistent"


def test_sampling_keeps_event_numbers():
    p = W.uneven_events(64, 20)
    s = autotune.sample_events(p, 10)
    assert len(np.unique(s["event"])) == 10
    for e in np.unique(s["event"]):
        assert np.array_equal(s[s["event"] == e]["id"], p[p["event"] == e]["id"])


def test_cache(tmp_path):
    calls = []
    f = lambda: calls.append(1) or {"x": 1}
    path = str(tmp_path / "tune.json")
    assert autotune.cached(path, "k", f) == {"x": 1}
    assert autotune.cached(path, "k", f) == {"x": 1}
    assert len(calls) == 1


@pytest.mark.gpu
def test_autotuned_batched_run_matches_oracle(geom):
    from parity import assert_strict_parity, oracle_run, run_gpu
    p = W.uneven_events(24, 6)
    p["ekin"] = np.minimum(p["ekin"], np.float32(2000.0))
    r = autotune.autotune(geom, p, 24, layouts=("aos", "aosoa32"), blocks=(128, 256),
                          drivers=("persistent", "graph"), reps=1, capacity_log2=18)
    b = r["best"]
    g = run_gpu(geom, p, 24, form="dense", layout=b["layout"], driver=b["driver"],
                block_size=b["block_size"], capacity_log2=18)
    assert_strict_parity(g, oracle_run(geom, p, 24))


def test_tuned_record_round_trip(tmp_path):
    from paper_2302_08252_gb300 import tuned
    path = str(tmp_path / "tuned.json")
    best = {"form": "dense", "layout": "aosoa64", "block_size": 256, "driver": "hybrid",
            "seconds": 0.1}
    tuned.write("uneven", best, "a sample", "cmd", path=path)
    tuned.write("mixed", dict(best, layout="aosoa32"), "a sample", "cmd", path=path)
    assert tuned.config("uneven", path=path) == {k: best[k] for k in tuned.KEYS}
    assert tuned.config("mixed", path=path)["layout"] == "aosoa32"
    assert tuned.config("jittered", path=path) is None
    # the committed record names a configuration the library accepts
    c = tuned.config("uneven")
    assert c["layout"] in autotune.LAYOUTS and c["driver"] in autotune.DRIVERS
    assert c["block_size"] in autotune.BLOCKS and c["form"] in ("dense", "sparse")
