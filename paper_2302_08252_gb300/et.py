"""Python binding of the C ABI in include/et.h (argument marshalling only).

Every transport step runs in the CUDA library libet.so built in-tree by
paper_2302_08252_gb300/build.py; importing this module fails loudly when the
library is missing.  PyTorch provides device memory (its caching allocator,
through the et_config allocator callbacks) and the CUDA stream.

Functions carry the C names; each raises EtError when the C call does not
return ET_OK.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .workloads import PRIMARY_DTYPE

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libet.so")

ET_OK, ET_ERR_INVALID, ET_ERR_CAPACITY, ET_ERR_CUDA, ET_ERR_TIMEOUT, ET_ERR_STATE, ET_ERR_NOMEM = \
    range(7)
FORM_SPARSE, FORM_DENSE = 0, 1
LAYOUT_AOS, LAYOUT_SOA, LAYOUT_AOSOA32, LAYOUT_AOSOA64, LAYOUT_AOSOA8, LAYOUT_AOSOA16, \
    LAYOUT_AOSOA128, LAYOUT_HOTCOLD = range(8)
LAYOUTS = {"aos": 0, "soa": 1, "aosoa32": 2, "aosoa64": 3, "aosoa8": 4, "aosoa16": 5,
           "aosoa128": 6, "hotcold": 7}
MODE_STRICT, MODE_FAST = 0, 1
DRIVER_HOSTLOOP, DRIVER_GRAPH, DRIVER_PERSISTENT, DRIVER_HYBRID = range(4)
DRIVERS = {"hostloop": 0, "graph": 1, "persistent": 2, "hybrid": 3}
N_LEAVES = 15
N_TAB, N_NODES = 5, 257   # tables: [material][Compton, pair, photoelectric, total, brems][node]
LEAF_NAMES = ("x", "y", "z", "dx", "dy", "dz", "ekin", "num_ia_left", "id", "event", "step",
              "slab", "time", "track_len", "flags")
IDREC_DTYPE = np.dtype([("id", "<u8"), ("steps", "<u4"), ("type_death", "<u4")])

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class EtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"et status {status}: {msg}")
        self.status = status


class et_config(C.Structure):
    _fields_ = [("capacity_log2", C.c_uint32), ("form", C.c_int32), ("layout", C.c_int32),
                ("mode", C.c_int32), ("driver", C.c_int32), ("block_size", C.c_int32),
                ("seed", C.c_uint64), ("max_events", C.c_uint32), ("max_iters", C.c_uint32),
                ("instrument", C.c_int32), ("id_log", C.c_int32),
                ("id_log_capacity", C.c_uint64), ("cuda_stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("serving", C.c_int32), ("reuse_slots", C.c_int32), ("hybrid_tracks", C.c_uint32),
                ("split_interactions", C.c_int32), ("msc", C.c_int32)]


class et_iter_stats(C.Structure):
    _fields_ = [("n_active", C.c_uint32 * 3), ("pad", C.c_uint32), ("steps", C.c_uint64),
                ("secondaries", C.c_uint64)]


class et_ledger(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("injected", "deposited_cont", "below_cut", "escaped",
                                          "mass_created", "mass_consumed")]


class et_counters(C.Structure):
    _fields_ = [("steps", C.c_uint64 * 3), ("secondaries", C.c_uint64 * 3),
                ("iterations", C.c_uint64), ("slot_high_water", C.c_uint64 * 3),
                ("reject_cap_hits", C.c_uint64), ("kernel_launches", C.c_uint64),
                ("status", C.c_uint32), ("pad", C.c_uint32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2302_08252_gb300/build.py)")
    L = C.CDLL(LIB_PATH)
    vp, st = C.c_void_p, C.c_int
    sig = {
        "et_create": ([C.POINTER(et_config), C.POINTER(vp)], st),
        "et_destroy": ([vp], st),
        "et_last_error": ([vp], C.c_char_p),
        "et_create_geometry": ([vp, C.c_uint32, vp, vp, C.c_float], st),
        "et_load_tables": ([vp, C.c_uint32, C.c_uint32, C.c_float, C.c_float, vp, vp], st),
        "et_build_toy_tables": ([C.c_uint32, C.c_uint32, vp, vp, vp, vp], st),
        "et_load_msc": ([vp, C.c_uint32, vp], st),
        "et_toy_radiation_lengths": ([C.c_uint32, vp], st),
        "et_build_toy_tables_fp64": ([C.c_uint32, C.c_uint32, vp, vp, vp, vp], st),
        "et_run_fp64": ([C.c_uint32, vp, vp, C.c_double, C.c_uint32, C.c_double, C.c_double, vp,
                         vp, vp, C.c_size_t, C.c_uint64, C.c_uint32, C.c_uint32, vp, vp,
                         C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], st),
        "et_inject": ([vp, vp, C.c_size_t], st),
        "et_inject_device": ([vp, vp, C.c_size_t], st),
        "et_run_iteration": ([vp, C.POINTER(et_iter_stats)], st),
        "et_run_until_empty": ([vp, C.c_uint64, C.POINTER(et_iter_stats), C.POINTER(C.c_uint64)], st),
        "et_read_scoring": ([vp, C.c_uint32, vp, C.c_size_t, C.POINTER(et_ledger)], st),
        "et_read_scoring_all": ([vp, vp, vp], st),
        "et_read_iteration_counts": ([vp, vp, C.c_uint64, C.POINTER(C.c_uint64)], st),
        "et_read_id_log": ([vp, vp, C.c_uint64, C.POINTER(C.c_uint64)], st),
        "et_read_field_trace": ([vp, vp], st),
        "et_read_heatmap": ([vp, C.c_uint32, C.c_uint32, vp, C.c_uint64], st),
        "et_read_counters": ([vp, C.POINTER(et_counters)], st),
        "et_reset": ([vp], st),
        "et_snapshot_size": ([vp, C.POINTER(C.c_uint64)], st),
        "et_snapshot": ([vp, vp, C.c_uint64, C.POINTER(C.c_uint64)], st),
        "et_restore": ([vp, vp, C.c_uint64], st),
        "et_poll_completed": ([vp, vp, C.c_uint64, C.POINTER(C.c_uint64)], st),
        "et_release_event": ([vp, C.c_uint32], st),
        "et_serve_submit": ([vp, vp, C.c_size_t, C.c_uint32, vp], st),
        "et_serve_round": ([vp, C.c_uint32, vp, vp, C.c_uint64, C.POINTER(C.c_uint64),
                            C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)], st),
        "et_serve_flush": ([vp, vp, vp, C.c_uint64, C.POINTER(C.c_uint64),
                            C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)], st),
        "et_serve_capacity": ([vp, C.POINTER(C.c_uint32)], st),
        "et_set_timing": ([vp, C.c_int], st),
        "et_read_timing": ([vp, C.POINTER(C.c_double), C.POINTER(C.c_uint64)], st),
        "et_transport_noalloc": ([C.c_uint32, vp, vp, C.c_float, C.c_uint32, C.c_float, C.c_float,
                                  vp, vp, vp, C.c_size_t, C.c_uint64, C.c_uint32, vp, vp,
                                  C.POINTER(C.c_uint64), vp, C.c_char_p, C.c_size_t], st),
        "et_debug_set_barrier_fault": ([vp, C.c_int, C.c_uint64], st),
        "et_debug_eval": ([C.c_int, vp, vp, C.c_size_t, vp], st),
        "et_debug_score_columns": ([C.c_uint32, vp], st),
        "et_debug_iteration_times": ([vp, C.c_int], st),
        "et_debug_read_iteration_times": ([vp, vp, C.c_uint64, C.POINTER(C.c_uint64)], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Context:
    """Owns an et_ctx* and keeps the allocator callbacks alive."""

    def __init__(self, handle, callbacks):
        self.handle = handle
        self._callbacks = callbacks

    def __del__(self):
        if getattr(self, "handle", None):
            lib.et_destroy(self.handle)
            self.handle = None


def _check(ctx, status):
    if status != ET_OK:
        h = ctx.handle if isinstance(ctx, Context) else ctx
        msg = lib.et_last_error(h).decode() if h else ""
        raise EtError(status, msg)


def _torch_callbacks():
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def free(ptr, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(alloc), FREE_FN(free)


def et_create(capacity_log2=20, form=FORM_DENSE, layout=LAYOUT_AOS, mode=MODE_STRICT,
              driver=DRIVER_HOSTLOOP, block_size=256, seed=1, max_events=1, max_iters=1 << 16,
              instrument=False, id_log=False, id_log_capacity=0, stream=None,
              use_torch_allocator=True, serving=False, reuse_slots=False,
              allocator=None, hybrid_tracks=0, split=False, msc=False) -> Context:
    """Create a context.  stream: a torch.cuda.Stream, an int cudaStream_t, or None for
    torch's current stream.  allocator: optional (alloc(nbytes, stream) -> int address,
    free(address)) pair of Python callables for the library's device buffers; default
    PyTorch's caching allocator."""
    import torch
    if not torch.cuda.is_available():
        raise EtError(ET_ERR_CUDA, "no CUDA device")
    if stream is None:
        s = torch.cuda.current_stream().cuda_stream
    elif isinstance(stream, int):
        s = stream
    else:
        s = stream.cuda_stream
    cfg = et_config()
    cfg.capacity_log2 = capacity_log2
    cfg.form = form
    cfg.layout = LAYOUTS[layout] if isinstance(layout, str) else layout
    cfg.mode = mode
    cfg.driver = DRIVERS[driver] if isinstance(driver, str) else driver
    cfg.block_size = block_size
    cfg.seed = seed
    cfg.max_events = max_events
    cfg.max_iters = max_iters
    cfg.instrument = int(bool(instrument))
    cfg.id_log = int(bool(id_log))
    cfg.id_log_capacity = id_log_capacity
    cfg.cuda_stream = s
    cfg.serving = int(bool(serving))
    cfg.reuse_slots = int(bool(reuse_slots))
    cfg.hybrid_tracks = int(hybrid_tracks)
    cfg.split_interactions = int(bool(split))
    cfg.msc = int(bool(msc))
    cbs = None
    if allocator is not None:
        fa, ff = allocator

        def alloc(nbytes, stream, user):
            try:
                return fa(int(nbytes), int(stream or 0))
            except Exception:
                return None

        cbs = (ALLOC_FN(alloc), FREE_FN(lambda ptr, user: ff(int(ptr))))
        cfg.alloc, cfg.free = cbs
    elif use_torch_allocator:
        cbs = _torch_callbacks()
        cfg.alloc, cfg.free = cbs
    h = C.c_void_p()
    st = lib.et_create(C.byref(cfg), C.byref(h))
    ctx = Context(h, cbs)
    _check(ctx, st)
    return ctx


def et_destroy(ctx: Context):
    if ctx.handle:
        st = lib.et_destroy(ctx.handle)
        ctx.handle = None
        if st != ET_OK:
            raise EtError(st, "et_destroy")


def et_create_geometry(ctx, thickness_mm, material, half_xy_mm):
    th = np.ascontiguousarray(thickness_mm, dtype=np.float64)
    mat = np.ascontiguousarray(material, dtype=np.uint8)
    _check(ctx, lib.et_create_geometry(ctx.handle, len(th), _p(th), _p(mat), float(half_xy_mm)))


def et_build_toy_tables(n_materials=2, n_nodes=257):
    sig = np.zeros((n_materials, 5, n_nodes), dtype=np.float32)
    dedx = np.zeros(n_materials, dtype=np.float32)
    le = np.zeros(1, np.float32)
    idl = np.zeros(1, np.float32)
    st = lib.et_build_toy_tables(n_materials, n_nodes, _p(sig), _p(dedx), _p(le), _p(idl))
    if st != ET_OK:
        raise EtError(st, "et_build_toy_tables")
    return {"sigma": sig, "dedx": dedx, "log_emin": float(le[0]), "inv_dlog": float(idl[0])}


def et_toy_radiation_lengths(n_materials=2) -> np.ndarray:
    x0 = np.zeros(n_materials, dtype=np.float32)
    st = lib.et_toy_radiation_lengths(n_materials, _p(x0))
    if st != ET_OK:
        raise EtError(st, "et_toy_radiation_lengths")
    return x0


def et_load_msc(ctx, x0_mm):
    x0 = np.ascontiguousarray(x0_mm, dtype=np.float32)
    _check(ctx, lib.et_load_msc(ctx.handle, len(x0), _p(x0)))


def et_build_toy_tables_fp64(n_materials=2, n_nodes=257):
    sig = np.zeros((n_materials, 5, n_nodes), dtype=np.float64)
    dedx = np.zeros(n_materials, dtype=np.float64)
    le = np.zeros(1, np.float64)
    idl = np.zeros(1, np.float64)
    st = lib.et_build_toy_tables_fp64(n_materials, n_nodes, _p(sig), _p(dedx), _p(le), _p(idl))
    if st != ET_OK:
        raise EtError(st, "et_build_toy_tables_fp64")
    return {"sigma": sig, "dedx": dedx, "log_emin": float(le[0]), "inv_dlog": float(idl[0])}


def et_load_tables(ctx, sigma, dedx, log_emin, inv_dlog):
    sig = np.ascontiguousarray(sigma, dtype=np.float32)
    d = np.ascontiguousarray(dedx, dtype=np.float32)
    _check(ctx, lib.et_load_tables(ctx.handle, sig.shape[0], sig.shape[2], float(log_emin),
                                   float(inv_dlog), _p(sig), _p(d)))


def et_inject(ctx, primaries: np.ndarray):
    p = np.ascontiguousarray(primaries)
    assert p.dtype == PRIMARY_DTYPE
    _check(ctx, lib.et_inject(ctx.handle, _p(p), len(p)))


def et_inject_device(ctx, primaries_device, n: int):
    """primaries_device: a CUDA torch.uint8 tensor holding n 48-byte records (or an int
    device address)."""
    ptr = primaries_device if isinstance(primaries_device, int) else primaries_device.data_ptr()
    _check(ctx, lib.et_inject_device(ctx.handle, C.c_void_p(ptr), n))


def et_run_iteration(ctx):
    s = et_iter_stats()
    _check(ctx, lib.et_run_iteration(ctx.handle, C.byref(s)))
    return {"n_active": list(s.n_active), "steps": s.steps, "secondaries": s.secondaries}


def et_run_until_empty(ctx, max_iters=1 << 30):
    s = et_iter_stats()
    n = C.c_uint64()
    _check(ctx, lib.et_run_until_empty(ctx.handle, max_iters, C.byref(s), C.byref(n)))
    return {"n_active": list(s.n_active), "steps": s.steps, "secondaries": s.secondaries,
            "iterations": n.value}


def et_read_scoring(ctx, event, n_slabs):
    dep = np.zeros(n_slabs, dtype=np.float64)
    lg = et_ledger()
    _check(ctx, lib.et_read_scoring(ctx.handle, event, _p(dep), n_slabs, C.byref(lg)))
    return dep, {f: getattr(lg, f) for f, _ in et_ledger._fields_}


def et_read_scoring_all(ctx, max_events, n_slabs, out=None):
    """Per-slab deposits [max_events][n_slabs] and ledgers [max_events][6].  `out`: an
    optional (score, ledger) pair of float64 arrays to fill (e.g. views of pinned memory,
    which the device copies into directly)."""
    if out is None:
        score = np.zeros((max_events, n_slabs), dtype=np.float64)
        ledger = np.zeros((max_events, 6), dtype=np.float64)
    else:
        score, ledger = out
        assert score.dtype == np.float64 and score.shape == (max_events, n_slabs)
        assert ledger.dtype == np.float64 and ledger.shape == (max_events, 6)
        assert score.flags.c_contiguous and ledger.flags.c_contiguous
    _check(ctx, lib.et_read_scoring_all(ctx.handle, _p(score), _p(ledger)))
    return score, ledger


def et_read_iteration_counts(ctx):
    n = C.c_uint64()
    _check(ctx, lib.et_read_iteration_counts(ctx.handle, None, 0, C.byref(n)))
    out = np.zeros((n.value, 3), dtype=np.uint64)
    if n.value:
        _check(ctx, lib.et_read_iteration_counts(ctx.handle, _p(out), n.value, C.byref(n)))
    return out


def et_read_id_log(ctx):
    n = C.c_uint64()
    _check(ctx, lib.et_read_id_log(ctx.handle, None, 0, C.byref(n)))
    out = np.zeros(n.value, dtype=IDREC_DTYPE)
    if n.value:
        _check(ctx, lib.et_read_id_log(ctx.handle, _p(out), n.value, C.byref(n)))
    return out


def et_read_field_trace(ctx):
    out = np.zeros((3, N_LEAVES, 2), dtype=np.uint64)
    _check(ctx, lib.et_read_field_trace(ctx.handle, _p(out)))
    return out


def et_read_heatmap(ctx, ptype, half, capacity):
    out = np.zeros(capacity * 16, dtype=np.uint32)
    _check(ctx, lib.et_read_heatmap(ctx.handle, ptype, half, _p(out), out.size))
    return out


def et_read_counters(ctx):
    c = et_counters()
    _check(ctx, lib.et_read_counters(ctx.handle, C.byref(c)))
    return {"steps": list(c.steps), "secondaries": list(c.secondaries),
            "iterations": c.iterations, "slot_high_water": list(c.slot_high_water),
            "reject_cap_hits": c.reject_cap_hits, "kernel_launches": c.kernel_launches,
            "status": c.status}


def et_reset(ctx):
    _check(ctx, lib.et_reset(ctx.handle))


def et_poll_completed(ctx, cap=1 << 16):
    out = np.zeros(cap, dtype=np.uint32)
    n = C.c_uint64()
    _check(ctx, lib.et_poll_completed(ctx.handle, _p(out), cap, C.byref(n)))
    return out[: n.value].copy()


def et_release_event(ctx, event):
    _check(ctx, lib.et_release_event(ctx.handle, event))


def et_serve_submit(ctx, primaries: np.ndarray, event: int, reserve):
    """Queue one event's primaries for the native serving loop (see et.h)."""
    p = np.ascontiguousarray(primaries)
    assert p.dtype == PRIMARY_DTYPE
    r = np.ascontiguousarray(reserve, dtype=np.uint32)
    assert r.shape == (3,)
    _check(ctx, lib.et_serve_submit(ctx.handle, _p(p), len(p), int(event), _p(r)))


class ServeBuffers:
    """Host result buffers of the serving loop: events and [n_slabs + 5] rows."""

    def __init__(self, ctx, n_slabs: int):
        m = C.c_uint32()
        _check(ctx, lib.et_serve_capacity(ctx.handle, C.byref(m)))
        self.cap = m.value
        self.events = np.zeros(self.cap, dtype=np.uint32)
        self.rows = np.zeros((self.cap, n_slabs + 5), dtype=np.float64)


def _serve_out(buf, n, steps, inflight):
    k = int(n.value)
    return (buf.events[:k].copy(), buf.rows[:k].copy(), int(steps.value), int(inflight.value))


def et_serve_round(ctx, buf: ServeBuffers, iters: int):
    """One round; returns (events, rows, steps, in_flight) of the previous round."""
    n, steps, inflight = C.c_uint64(), C.c_uint64(), C.c_uint32()
    _check(ctx, lib.et_serve_round(ctx.handle, int(iters), _p(buf.events), _p(buf.rows), buf.cap,
                                   C.byref(n), C.byref(steps), C.byref(inflight)))
    return _serve_out(buf, n, steps, inflight)


def et_serve_flush(ctx, buf: ServeBuffers):
    n, steps, inflight = C.c_uint64(), C.c_uint64(), C.c_uint32()
    _check(ctx, lib.et_serve_flush(ctx.handle, _p(buf.events), _p(buf.rows), buf.cap,
                                   C.byref(n), C.byref(steps), C.byref(inflight)))
    return _serve_out(buf, n, steps, inflight)


def et_set_timing(ctx, on=True):
    _check(ctx, lib.et_set_timing(ctx.handle, int(bool(on))))


def et_read_timing(ctx):
    ms = C.c_double()
    n = C.c_uint64()
    _check(ctx, lib.et_read_timing(ctx.handle, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def et_debug_set_barrier_fault(ctx, skip_block=-1, timeout_ns=0):
    _check(ctx, lib.et_debug_set_barrier_fault(ctx.handle, skip_block, timeout_ns))


def et_debug_iteration_times(ctx, enable=True):
    _check(ctx, lib.et_debug_iteration_times(ctx.handle, int(bool(enable))))


def et_debug_read_iteration_times(ctx):
    n = C.c_uint64()
    _check(ctx, lib.et_debug_read_iteration_times(ctx.handle, None, 0, C.byref(n)))
    out = np.zeros(n.value, dtype=np.uint64)
    if n.value:
        _check(ctx, lib.et_debug_read_iteration_times(ctx.handle, _p(out), n.value, C.byref(n)))
    return out


NOALLOC_MAX_TRACKS = 32768
NOALLOC_MAX_ITERS = 4096


def _noalloc_check_tensor(name, t, dtype, min_elems):
    """Refuse a device buffer the library would read or write out of bounds."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"et_transport_noalloc: {name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"et_transport_noalloc: {name} must be {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"et_transport_noalloc: {name} must be contiguous")
    if t.numel() < min_elems:
        raise ValueError(f"et_transport_noalloc: {name} holds {t.numel()} elements,"
                         f" {min_elems} needed")


def _noalloc_check_device(name, t, device):
    if not t.is_cuda:
        raise ValueError(f"et_transport_noalloc: {name} is not in device memory")
    if device is not None and t.device != device:
        raise ValueError(f"et_transport_noalloc: {name} is on {t.device}, not {device}")


def et_transport_noalloc(geom, tables, primaries_device, n_primaries, seed, n_events,
                         score_device, ledger_device, stream=None):
    """The allocation-free transport of one batch (see et.h).  primaries_device: CUDA uint8
    tensor holding n_primaries 48-byte records; score_device: CUDA float64
    [n_events][n_slabs]; ledger_device: CUDA float64 [n_events][5], both on the primaries'
    device.  Every buffer is checked (type, device, contiguity, size) before the library
    is called, since the kernels write score[event][slab] and ledger[event][k] for every
    event below n_events.  Returns the steps."""
    import torch
    th = np.ascontiguousarray(geom["thickness"], dtype=np.float64)
    mat = np.ascontiguousarray(geom["material"], dtype=np.uint8)
    sig = np.ascontiguousarray(tables["sigma"], dtype=np.float32)
    dedx = np.ascontiguousarray(tables["dedx"], dtype=np.float32)
    if sig.ndim != 3 or sig.shape[1:] != (N_TAB, N_NODES):
        raise ValueError(f"et_transport_noalloc: sigma must be [n_materials][{N_TAB}]"
                         f"[{N_NODES}], not {list(sig.shape)}")
    if dedx.shape != (sig.shape[0],):
        raise ValueError("et_transport_noalloc: dedx must hold one value per material")
    if len(mat) != len(th):
        raise ValueError("et_transport_noalloc: thickness and material differ in length")
    n_primaries, n_events = int(n_primaries), int(n_events)
    if n_primaries < 0 or n_events < 1:
        raise ValueError("et_transport_noalloc: n_primaries >= 0 and n_events >= 1 needed")
    if not 0 <= int(seed) < (1 << 32):
        raise ValueError("et_transport_noalloc: the seed keys Philox with 32 bits")
    _noalloc_check_tensor("primaries_device", primaries_device, torch.uint8,
                          n_primaries * PRIMARY_DTYPE.itemsize)
    _noalloc_check_tensor("score_device", score_device, torch.float64, n_events * len(th))
    _noalloc_check_tensor("ledger_device", ledger_device, torch.float64, n_events * 5)
    dev = primaries_device.device
    for name, t in (("primaries_device", primaries_device), ("score_device", score_device),
                    ("ledger_device", ledger_device)):
        _noalloc_check_device(name, t, dev)
    if stream is None:
        s = torch.cuda.current_stream(dev).cuda_stream
    else:
        s = stream if isinstance(stream, int) else stream.cuda_stream
    steps = C.c_uint64()
    err = C.create_string_buffer(256)
    with torch.cuda.device(dev):
        st = lib.et_transport_noalloc(len(th), _p(th), _p(mat), float(geom["half_xy"]),
                                      sig.shape[0], float(tables["log_emin"]),
                                      float(tables["inv_dlog"]), _p(sig), _p(dedx),
                                      C.c_void_p(primaries_device.data_ptr()), n_primaries,
                                      int(seed), n_events, C.c_void_p(score_device.data_ptr()),
                                      C.c_void_p(ledger_device.data_ptr()), C.byref(steps),
                                      C.c_void_p(s), err, len(err))
    if st != ET_OK:
        raise EtError(st, err.value.decode())
    return steps.value


def et_run_fp64(geom, tables64, primaries: np.ndarray, seed, n_events, capacity_log2=22):
    """The all-FP64 transport of one batch (see et.h).  tables64: et_build_toy_tables_fp64().
    Returns (score[n_events][n_slabs], ledger[n_events][5], steps, iterations)."""
    th = np.ascontiguousarray(geom["thickness"], dtype=np.float64)
    mat = np.ascontiguousarray(geom["material"], dtype=np.uint8)
    sig = np.ascontiguousarray(tables64["sigma"], dtype=np.float64)
    dedx = np.ascontiguousarray(tables64["dedx"], dtype=np.float64)
    p = np.ascontiguousarray(primaries)
    assert p.dtype == PRIMARY_DTYPE
    score = np.zeros((n_events, len(th)), np.float64)
    ledger = np.zeros((n_events, 5), np.float64)
    steps, iters = C.c_uint64(), C.c_uint64()
    st = lib.et_run_fp64(len(th), _p(th), _p(mat), float(geom["half_xy"]), sig.shape[0],
                         float(tables64["log_emin"]), float(tables64["inv_dlog"]), _p(sig),
                         _p(dedx), _p(p), len(p), seed, n_events, capacity_log2, _p(score),
                         _p(ledger), C.byref(steps), C.byref(iters))
    if st != ET_OK:
        raise EtError(st, "et_run_fp64")
    return score, ledger, steps.value, iters.value


def make_context(geom: dict, max_events: int, tables: dict | None = None, **kw) -> Context:
    """Create a context and load the calorimeter and the toy tables (convenience); with
    msc=True also the toy radiation lengths (toy model v2)."""
    ctx = et_create(max_events=max_events, **kw)
    et_create_geometry(ctx, geom["thickness"], geom["material"], geom["half_xy"])
    t = tables if tables is not None else et_build_toy_tables()
    et_load_tables(ctx, t["sigma"], t["dedx"], t["log_emin"], t["inv_dlog"])
    if kw.get("msc"):
        et_load_msc(ctx, et_toy_radiation_lengths(len(t["dedx"])))
    return ctx


EVAL_PHILOX, EVAL_U01, EVAL_LOG, EVAL_EXP, EVAL_SINCOS2PI = range(5)


def et_debug_eval(what: int, inputs, outputs):
    """Evaluate a device primitive (et_debug.h) on CUDA tensors: inputs uint32 [n, 6]
    (Philox), uint32 [n] (u01) or float32 [n]; outputs sized accordingly."""
    import torch
    n = inputs.shape[0]
    st = lib.et_debug_eval(what, C.c_void_p(inputs.data_ptr()), C.c_void_p(outputs.data_ptr()), n,
                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != ET_OK:
        raise EtError(st, "et_debug_eval")
    return outputs


def et_snapshot(ctx) -> bytes:
    """The context's state between iterations (see et.h) as bytes."""
    n = C.c_uint64()
    _check(ctx, lib.et_snapshot_size(ctx.handle, C.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    w = C.c_uint64()
    _check(ctx, lib.et_snapshot(ctx.handle, _p(buf), n.value, C.byref(w)))
    return buf[: w.value].tobytes()


def et_restore(ctx, snapshot: bytes):
    buf = np.frombuffer(snapshot, dtype=np.uint8)
    _check(ctx, lib.et_restore(ctx.handle, _p(buf), len(buf)))

