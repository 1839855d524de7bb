"""CPU oracle of the toy EM shower transport -- TEST INFRASTRUCTURE.

Plain, slow, obviously-correct CPU definition of the transport the CUDA path
implements (paper Sec. 2: sparse/dense track buffers stepped once per
iteration; Sec. 4: electron gun into a 50-layer calorimeter scoring energy per
layer).  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
may import this package.  It shares no code with the product package; inputs
come from the seeded generators in paper_2302_08252_gb300.workloads.

The C sources in this directory are the oracle; this module only marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

STRICT_FP32 = 0
REF_FP64 = 1
N_NODES = 257
N_MAT = 2
N_TAB = 5
TAB_COMPTON, TAB_PAIR, TAB_PHOT, TAB_TOT, TAB_BREM = range(5)
LIM_Z, LIM_X, LIM_Y, LIM_LOSS, LIM_PHYS, LIM_MSC = range(6)
PROC_NONE, PROC_COMPTON, PROC_PAIR, PROC_PHOT, PROC_BREM = range(5)
ALIVE, DEATH_ESCAPE, DEATH_CUT, DEATH_ABSORB = range(4)
LEDGER_FIELDS = ("injected", "deposited_cont", "below_cut", "escaped", "mass_created",
                 "mass_consumed")

IDREC_DTYPE = np.dtype([("id", "<u8"), ("steps", "<u4"), ("type_death", "<u4")])
TRACK32_DTYPE = np.dtype(
    [("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("dx", "<f4"), ("dy", "<f4"), ("dz", "<f4"),
     ("e", "<f4"), ("nia", "<f4"), ("id", "<u8"), ("event", "<u4"), ("step", "<u4"),
     ("slab", "<i4"), ("time", "<f4"), ("len", "<f4"), ("flags", "<u4")], align=True)
assert TRACK32_DTYPE.itemsize == 64


class _Track32(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("x", "y", "z", "dx", "dy", "dz", "e", "nia")] + [
        ("id", C.c_uint64), ("event", C.c_uint32), ("step", C.c_uint32), ("slab", C.c_int32),
        ("time", C.c_float), ("len", C.c_float), ("flags", C.c_uint32)]


class _StepResult(C.Structure):
    _fields_ = [("track", _Track32), ("alive", C.c_int32), ("death", C.c_int32),
                ("lim", C.c_int32), ("proc", C.c_int32), ("nsec", C.c_int32),
                ("sec_type", C.c_int32 * 4), ("sec", _Track32 * 4), ("dep_cont", C.c_double),
                ("cut", C.c_double), ("esc", C.c_double), ("mc", C.c_double),
                ("mcr", C.c_double), ("slab_cont", C.c_int32), ("slab_cut", C.c_int32),
                ("reject_cap_hit", C.c_int32), ("pad", C.c_int32)]


class _World(C.Structure):
    _fields_ = [("n_slabs", C.c_int32), ("n_mat", C.c_int32), ("n_nodes", C.c_int32),
                ("pad0", C.c_int32), ("thickness", C.c_void_p), ("material", C.c_void_p),
                ("half_xy", C.c_float), ("log_emin32", C.c_float), ("inv_dlog32", C.c_float),
                ("pad1", C.c_float), ("log_emin64", C.c_double), ("inv_dlog64", C.c_double),
                ("sig32", C.c_void_p), ("sig64", C.c_void_p), ("dedx32", C.c_void_p),
                ("dedx64", C.c_void_p), ("seed", C.c_uint64), ("msc", C.c_int32),
                ("pad2", C.c_int32), ("x0_32", C.c_void_p), ("x0_64", C.c_void_p)]


class _Totals(C.Structure):
    _fields_ = [("steps", C.c_uint64 * 3), ("tracks", C.c_uint64 * 3),
                ("secondaries", C.c_uint64 * 3), ("reject_cap_hits", C.c_uint64),
                ("n_iters", C.c_uint64), ("idlog_n", C.c_uint64), ("errors", C.c_uint64)]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, sz = C.c_void_p, C.c_size_t
        L.oracle_philox_n.argtypes = [vp, vp, vp, sz]
        L.oracle_u01.argtypes = [C.c_uint32]
        L.oracle_u01.restype = C.c_float
        L.oracle_mix64.argtypes = [C.c_uint64]
        L.oracle_mix64.restype = C.c_uint64
        L.oracle_secondary_id.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        L.oracle_secondary_id.restype = C.c_uint64
        for n in ("oracle_spec_log_n", "oracle_spec_exp_n"):
            getattr(L, n).argtypes = [vp, vp, sz]
        L.oracle_spec_sincos2pi_n.argtypes = [vp, vp, vp, sz]
        for n in ("oracle_sigma_compton", "oracle_sigma_pair", "oracle_sigma_phot",
                  "oracle_sigma_brem"):
            getattr(L, n).argtypes = [C.c_int, C.c_double]
            getattr(L, n).restype = C.c_double
        L.oracle_dedx.argtypes = [C.c_int]
        L.oracle_dedx.restype = C.c_double
        L.oracle_x0.argtypes = [C.c_int]
        L.oracle_x0.restype = C.c_double
        L.oracle_kn_per_electron_cm2.argtypes = [C.c_double]
        L.oracle_kn_per_electron_cm2.restype = C.c_double
        L.oracle_electron_density_cm3.argtypes = [C.c_int]
        L.oracle_electron_density_cm3.restype = C.c_double
        L.oracle_build_tables.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_run.argtypes = [vp, vp, sz, C.c_uint32, C.c_int, C.c_int, vp, vp, vp,
                                 C.c_uint64, vp, C.c_uint64, vp]
        L.oracle_step_one.argtypes = [vp, C.c_int, vp, vp]
        L.oracle_sample_compton_eps_n.argtypes = [C.c_float, C.c_uint64, C.c_uint32, vp,
                                                  C.c_uint32, vp, vp, sz]
        _LIB = L
    return _LIB


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- building blocks

def philox(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr[n, 4] (uint32) under key (k0, k1)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.asarray(key, dtype=np.uint32)
    out = np.empty_like(ctr)
    lib().oracle_philox_n(_p(ctr), _p(k), _p(out), len(ctr))
    return out


def u01(x: int) -> float:
    return float(lib().oracle_u01(int(x)))


def mix64(z: int) -> int:
    return int(lib().oracle_mix64(int(z)))


def secondary_id(parent: int, step: int, ordinal: int) -> int:
    return int(lib().oracle_secondary_id(int(parent), int(step), int(ordinal)))


def spec_log(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().oracle_spec_log_n(_p(x), _p(y), x.size)
    return y


def spec_exp(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().oracle_spec_exp_n(_p(x), _p(y), x.size)
    return y


def spec_sincos2pi(u):
    u = np.ascontiguousarray(u, dtype=np.float32)
    s = np.empty_like(u)
    c = np.empty_like(u)
    lib().oracle_spec_sincos2pi_n(_p(u), _p(s), _p(c), u.size)
    return s, c


def sigma(kind: str, mat: int, e_mev: float) -> float:
    """Closed-form cross section (1/mm): kind in compton, pair, phot, brem."""
    return float(getattr(lib(), f"oracle_sigma_{kind}")(int(mat), float(e_mev)))


def kn_per_electron_cm2(k: float) -> float:
    return float(lib().oracle_kn_per_electron_cm2(float(k)))


def electron_density_cm3(mat: int) -> float:
    return float(lib().oracle_electron_density_cm3(int(mat)))


def dedx(mat: int) -> float:
    return float(lib().oracle_dedx(int(mat)))


def build_tables(n_nodes: int = N_NODES, n_mat: int = N_MAT) -> dict:
    """The oracle's own tables: sig32/sig64 [n_mat][5][n_nodes], dedx32/dedx64, lookup constants."""
    sig32 = np.zeros((n_mat, N_TAB, n_nodes), dtype=np.float32)
    sig64 = np.zeros((n_mat, N_TAB, n_nodes), dtype=np.float64)
    d32 = np.zeros(n_mat, dtype=np.float32)
    d64 = np.zeros(n_mat, dtype=np.float64)
    le32 = np.zeros(1, np.float32)
    id32 = np.zeros(1, np.float32)
    le64 = np.zeros(1, np.float64)
    id64 = np.zeros(1, np.float64)
    rc = lib().oracle_build_tables(n_mat, n_nodes, _p(sig32), _p(sig64), _p(d32), _p(d64),
                                   _p(le32), _p(id32), _p(le64), _p(id64))
    if rc:
        raise ValueError("oracle_build_tables failed")
    return {"sig32": sig32, "sig64": sig64, "dedx32": d32, "dedx64": d64,
            "log_emin32": float(le32[0]), "inv_dlog32": float(id32[0]),
            "log_emin64": float(le64[0]), "inv_dlog64": float(id64[0]), "n_nodes": n_nodes,
            "n_mat": n_mat}


def radiation_lengths(n_mat: int = N_MAT) -> np.ndarray:
    """Radiation length X0 (mm) per material (FP64)."""
    return np.array([lib().oracle_x0(m) for m in range(n_mat)], dtype=np.float64)


class World:
    """Geometry + tables + seed, kept alive for the C side.  msc=True selects the toy
    model v2 (multiple scattering of e+-) with the materials' radiation lengths."""

    def __init__(self, geom: dict, tables: dict | None = None, seed: int = 1, msc: bool = False):
        self.tables = tables if tables is not None else build_tables()
        t = self.tables
        self._keep = [np.ascontiguousarray(geom["thickness"], np.float64),
                      np.ascontiguousarray(geom["material"], np.uint8),
                      np.ascontiguousarray(t["sig32"], np.float32),
                      np.ascontiguousarray(t["sig64"], np.float64),
                      np.ascontiguousarray(t["dedx32"], np.float32),
                      np.ascontiguousarray(t["dedx64"], np.float64)]
        th, mat, s32, s64, d32, d64 = self._keep
        w = _World()
        w.n_slabs = len(th)
        w.n_mat = int(t["n_mat"])
        w.n_nodes = int(t["n_nodes"])
        w.thickness = th.ctypes.data
        w.material = mat.ctypes.data
        w.half_xy = float(geom["half_xy"])
        w.log_emin32 = t["log_emin32"]
        w.inv_dlog32 = t["inv_dlog32"]
        w.log_emin64 = t["log_emin64"]
        w.inv_dlog64 = t["inv_dlog64"]
        w.sig32 = s32.ctypes.data
        w.sig64 = s64.ctypes.data
        w.dedx32 = d32.ctypes.data
        w.dedx64 = d64.ctypes.data
        w.seed = int(seed)
        x0 = radiation_lengths(int(t["n_mat"]))
        self._keep += [x0.astype(np.float32), x0]
        w.msc = int(bool(msc))
        w.x0_32 = self._keep[-2].ctypes.data
        w.x0_64 = self._keep[-1].ctypes.data
        self.c = w
        self.n_slabs = len(th)


def run(geom: dict, primaries: np.ndarray, n_events: int | None = None, seed: int = 1,
        mode: int = STRICT_FP32, nthreads: int = 1, max_iters: int = 1 << 16,
        idlog: bool = False, tables: dict | None = None, world: World | None = None,
        msc: bool = False) -> dict:
    """Run primaries (workloads.PRIMARY_DTYPE) to completion; returns numpy results.
    msc=True runs the toy model v2 (multiple scattering)."""
    w = world if world is not None else World(geom, tables, seed, msc=msc)
    prim = np.ascontiguousarray(primaries)
    assert prim.dtype.itemsize == 48
    if n_events is None:
        n_events = int(prim["event"].max()) + 1 if len(prim) else 0
    score = np.zeros((n_events, w.n_slabs), dtype=np.float64)
    ledger = np.zeros((n_events, 6), dtype=np.float64)
    counts = np.zeros((max_iters, 3), dtype=np.uint64)
    tot = _Totals()
    idl = None
    cap = 0
    if idlog:
        # first pass to size the log is avoided: grow until it fits
        cap = max(1024, 64 * len(prim))
        while True:
            idl = np.zeros(cap, dtype=IDREC_DTYPE)
            rc = lib().oracle_run(C.byref(w.c), _p(prim), len(prim), n_events, mode, nthreads,
                                  _p(score), _p(ledger), _p(counts), max_iters, _p(idl), cap,
                                  C.byref(tot))
            if rc & 2:
                cap = int(tot.idlog_n) + 16
                continue
            break
    else:
        rc = lib().oracle_run(C.byref(w.c), _p(prim), len(prim), n_events, mode, nthreads,
                              _p(score), _p(ledger), _p(counts), max_iters, None, 0,
                              C.byref(tot))
    if rc:
        raise RuntimeError(f"oracle_run failed with error mask {rc}")
    n_iters = int(tot.n_iters)
    out = {
        "score": score,
        "ledger": ledger,
        "counts": counts[:n_iters].copy(),
        "n_iters": n_iters,
        "steps": np.array(tot.steps[:], dtype=np.uint64),
        "tracks": np.array(tot.tracks[:], dtype=np.uint64),
        "secondaries": np.array(tot.secondaries[:], dtype=np.uint64),
        "reject_cap_hits": int(tot.reject_cap_hits),
    }
    if idlog:
        out["idlog"] = idl[: int(tot.idlog_n)].copy()
    return out


def make_track(x=0.0, y=0.0, z=0.0, d=(0.0, 0.0, 1.0), e=1.0, nia=-1.0, id=0, event=0, step=0,
               slab=0, time=0.0, length=0.0) -> np.ndarray:
    t = np.zeros(1, dtype=TRACK32_DTYPE)
    t["x"], t["y"], t["z"] = x, y, z
    t["dx"], t["dy"], t["dz"] = d
    t["e"], t["nia"], t["id"], t["event"] = e, nia, id, event
    t["step"], t["slab"], t["time"], t["len"] = step, slab, time, length
    return t


def step_one(world: World, ptype: int, track: np.ndarray) -> dict:
    """One strict FP32 step of one track (TRACK32_DTYPE record)."""
    tin = _Track32.from_buffer_copy(np.ascontiguousarray(track).tobytes())
    res = _StepResult()
    rc = lib().oracle_step_one(C.byref(world.c), int(ptype), C.byref(tin), C.byref(res))
    if rc:
        raise ValueError("oracle_step_one rejected its input")

    def rec(t):
        return np.frombuffer(bytes(t), dtype=TRACK32_DTYPE)[0].copy()

    return {
        "track": rec(res.track), "alive": res.alive, "death": res.death, "lim": res.lim,
        "proc": res.proc, "nsec": res.nsec, "sec_type": list(res.sec_type[: res.nsec]),
        "sec": [rec(res.sec[k]) for k in range(res.nsec)], "dep_cont": res.dep_cont,
        "cut": res.cut, "esc": res.esc, "mc": res.mc, "mcr": res.mcr,
        "slab_cont": res.slab_cont, "slab_cut": res.slab_cut,
        "reject_cap_hit": res.reject_cap_hit,
    }


def compton_eps(k: float, ids: np.ndarray, seed: int = 1, event: int = 0, step: int = 0):
    """Klein-Nishina eps samples for each track id (strict FP32 sampler)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    eps = np.empty(len(ids), dtype=np.float32)
    att = np.empty(len(ids), dtype=np.int32)
    lib().oracle_sample_compton_eps_n(float(k), int(seed), int(event), _p(ids), int(step),
                                      _p(eps), _p(att), len(ids))
    return eps, att
