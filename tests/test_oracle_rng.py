"""Pins of the oracle's random numbers and track ids against their published definitions."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_philox_known_answers():
    for row in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = oracle.philox(np.array([v[0:4]], np.uint32), v[4:6])[0]
        assert [int(x) for x in out] == v[6:10]


def test_splitmix64_finalizer_known_outputs():
    for n, state, out in _rows("splitmix64.txt"):
        assert int(state, 16) == (int(n) * 0x9E3779B97F4A7C15) % (1 << 64)
        assert oracle.mix64(int(state, 16)) == int(out, 16)


def test_u01_range_and_endpoints():
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFF) == 2.0 ** -24
    assert oracle.u01(0x100) == 2.0 * 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0


def test_philox_uniformity():
    # counters as the transport uses them: (id_lo, id_hi, step, block)
    n = 1 << 18
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = 7
    out = oracle.philox(ctr, [1, 3]).ravel()
    u = ((out >> 8).astype(np.float64) + 1.0) * 2.0 ** -24
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.002
    byte = (out & 0xFF).astype(np.int64)
    counts = np.bincount(byte, minlength=256)
    exp = out.size / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # chi2 with 255 dof: mean 255, sd ~22.6; 6 sd bound
    assert chi2 < 255 + 6 * 22.6
    # distinct keys give distinct streams
    other = oracle.philox(ctr[:16], [1, 4])
    assert not np.array_equal(other, out.reshape(-1, 4)[:16])


def test_secondary_ids_distinct():
    parent = (5 << 32) | 3
    ids = {oracle.secondary_id(parent, s, k) for s in range(200) for k in range(4)}
    assert len(ids) == 800
    assert parent not in ids
