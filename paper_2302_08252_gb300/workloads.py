"""Seeded synthetic inputs: calorimeter geometry and primary particles.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from.  It holds none of the transport arithmetic: it only draws
primaries (type, event, id, position, direction, energy) and lists the slab
thicknesses and materials.

Workloads stand in for the paper's benchmark (Sec. 4: a 10 GeV electron gun
into the 50 alternating absorber/gap layers of the TestEm3 geometry, run as
`-particles 10000 -batch 5000`; the heatmap run uses 25 particles in 5
batches).  Geometry: 50 layers of 2.3 mm lead then 5.7 mm liquid argon,
40 x 40 cm transverse, front face at z = 0, vacuum outside.

Primaries are drawn with numpy's Philox bit generator (seed 2 unless given).
"""
from __future__ import annotations

import numpy as np

# 48-byte primary record; the C-ABI's et_primary and the oracle's record match it.
PRIMARY_DTYPE = np.dtype(
    [
        ("type", "<u4"),
        ("event", "<u4"),
        ("id", "<u8"),
        ("pos", "<f4", (3,)),
        ("dir", "<f4", (3,)),
        ("ekin", "<f4"),
        ("pad", "<u4"),
    ],
    align=True,
)
assert PRIMARY_DTYPE.itemsize == 48

E_MINUS, E_PLUS, GAMMA = 0, 1, 2
N_LAYERS = 50
HALF_XY_MM = 200.0
PRIMARY_SEED = 2
PHYSICS_SEED = 1
ARRIVAL_SEED = 3


def calorimeter(n_layers: int = N_LAYERS, absorber_mm: float = 2.3, gap_mm: float = 5.7):
    """Slab thicknesses (FP64, mm), material per slab (0 lead, 1 liquid argon), half width."""
    thickness = np.empty(2 * n_layers, dtype=np.float64)
    thickness[0::2] = absorber_mm
    thickness[1::2] = gap_mm
    material = np.zeros(2 * n_layers, dtype=np.uint8)
    material[1::2] = 1
    return {"thickness": thickness, "material": material, "half_xy": HALF_XY_MM}


def single_slab(thickness_mm: float, material: int = 0, half_xy: float = 1.0e6):
    """One thick slab (used by the attenuation and range pins)."""
    return {
        "thickness": np.array([thickness_mm], dtype=np.float64),
        "material": np.array([material], dtype=np.uint8),
        "half_xy": float(half_xy),
    }


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=seed))


def _records(n: int) -> np.ndarray:
    p = np.zeros(n, dtype=PRIMARY_DTYPE)
    p["dir"][:, 2] = 1.0
    return p


def assign_ids(p: np.ndarray) -> np.ndarray:
    """id = (event << 32) | index of the primary within its event (in array order)."""
    ev = p["event"].astype(np.uint64)
    idx = np.zeros(len(p), dtype=np.uint64)
    seen: dict[int, int] = {}
    for i, e in enumerate(p["event"].tolist()):
        k = seen.get(e, 0)
        idx[i] = k
        seen[e] = k + 1
    p["id"] = (ev << np.uint64(32)) | idx
    return p


def gun(n: int, ekin_mev: float, ptype: int = E_MINUS, first_event: int = 0) -> np.ndarray:
    """n primaries of one type and energy at the origin along +z, one event each."""
    p = _records(n)
    p["type"] = ptype
    p["event"] = np.arange(first_event, first_event + n, dtype=np.uint32)
    p["ekin"] = np.float32(ekin_mev)
    return assign_ids(p)


def small_electrons(n: int = 16, ekin_mev: float = 1000.0) -> np.ndarray:
    """16 electrons of 1 GeV on the +z axis, one event each (the small plain-method case)."""
    return gun(n, ekin_mev)


def jittered_electrons(n: int = 1000, ekin_mev: float = 10000.0, jitter_rad: float = 1e-3,
                       seed: int = PRIMARY_SEED) -> np.ndarray:
    """n electrons of 10 GeV with directions uniform in solid angle inside a 1 mrad cone
    about +z (cos theta ~ U[cos 1e-3, 1], phi ~ U[0, 2 pi)), one event each."""
    r = _rng(seed)
    p = gun(n, ekin_mev)
    cost = r.uniform(np.cos(jitter_rad), 1.0, n)
    phi = r.uniform(0.0, 2.0 * np.pi, n)
    sint = np.sqrt(np.maximum(0.0, 1.0 - cost * cost))
    p["dir"][:, 0] = sint * np.cos(phi)
    p["dir"][:, 1] = sint * np.sin(phi)
    p["dir"][:, 2] = cost
    return p


def _mixed(r: np.random.Generator, n: int):
    u = r.uniform(0.0, 1.0, n)
    ptype = np.where(u < 0.5, E_MINUS, np.where(u < 0.75, E_PLUS, GAMMA)).astype(np.uint32)
    ekin = np.exp(r.uniform(np.log(100.0), np.log(1.0e5), n))
    x = r.uniform(-5.0, 5.0, n)
    y = r.uniform(-5.0, 5.0, n)
    return ptype, ekin, x, y


def mixed_primaries(n: int = 10000, seed: int = PRIMARY_SEED) -> np.ndarray:
    """50% e-, 25% e+, 25% photons; E log-uniform on [100 MeV, 100 GeV]; x, y ~ U[-5, 5] mm
    (1 cm^2 spot) at z = 0; direction +z; one event each."""
    r = _rng(seed)
    p = _records(n)
    ptype, ekin, x, y = _mixed(r, n)
    p["type"] = ptype
    p["ekin"] = ekin.astype(np.float32)
    p["pos"][:, 0] = x
    p["pos"][:, 1] = y
    p["event"] = np.arange(n, dtype=np.uint32)
    return assign_ids(p)


def uneven_events(n_events: int = 256, max_primaries: int = 1000, seed: int = PRIMARY_SEED):
    """n_events events; primaries per event clamp(floor(exp(u ln(max+1))), 1, max), each primary
    drawn like mixed_primaries.  Returns the primaries (grouped by event)."""
    r = _rng(seed)
    u = r.uniform(0.0, 1.0, n_events)
    sizes = np.clip(np.floor(np.exp(u * np.log(max_primaries + 1.0))), 1, max_primaries)
    sizes = sizes.astype(np.int64)
    n = int(sizes.sum())
    p = _records(n)
    ptype, ekin, x, y = _mixed(r, n)
    p["type"] = ptype
    p["ekin"] = ekin.astype(np.float32)
    p["pos"][:, 0] = x
    p["pos"][:, 1] = y
    p["event"] = np.repeat(np.arange(n_events, dtype=np.uint32), sizes)
    return assign_ids(p)


def poisson_arrivals(rate_per_s: float, n_events: int, seed: int = ARRIVAL_SEED) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    r = _rng(seed)
    return np.cumsum(r.exponential(1.0 / rate_per_s, n_events))


def select_events(p: np.ndarray, events) -> np.ndarray:
    """The primaries of the listed events, event numbers and ids unchanged (the random
    draws are keyed by event, so a sample must keep its original numbering)."""
    mask = np.isin(p["event"], np.asarray(list(events), dtype=np.uint32))
    return p[mask].copy()
