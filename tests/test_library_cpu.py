"""Host-side checks of the CUDA library that need no GPU: it builds, loads, exports every
entry point include/et.h declares, and its host-side table builder reproduces the oracle's
tables bit for bit (the two are written independently from the same closed forms)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libet():
    from paper_2302_08252_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(et_\w+)\s*\(", text, re.M))
    return sorted(names)


def test_exports_every_declared_symbol(libet):
    names = declared_symbols()
    for core in ("et_create_geometry", "et_load_tables", "et_inject", "et_run_iteration",
                 "et_run_until_empty", "et_read_scoring"):
        assert core in names
    assert len(names) >= 19
    for n in names:
        assert hasattr(libet, n), n


def test_toy_tables_match_oracle_bit_for_bit(libet):
    import oracle
    from paper_2302_08252_gb300 import et
    mine = et.et_build_toy_tables()
    ref = oracle.build_tables()
    assert np.array_equal(mine["sigma"].view(np.uint32), ref["sig32"].view(np.uint32))
    assert np.array_equal(mine["dedx"], ref["dedx32"])
    assert mine["log_emin"] == ref["log_emin32"]
    assert mine["inv_dlog"] == ref["inv_dlog32"]


def test_fp64_toy_tables_match_oracle(libet):
    import oracle
    from paper_2302_08252_gb300 import et
    mine = et.et_build_toy_tables_fp64()
    ref = oracle.build_tables()
    assert np.allclose(mine["sigma"], ref["sig64"], rtol=1e-14, atol=0.0)
    assert np.array_equal(mine["dedx"], ref["dedx64"])
    assert mine["log_emin"] == ref["log_emin64"]
    assert mine["inv_dlog"] == ref["inv_dlog64"]


def test_create_without_gpu_fails_cleanly(libet):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2302_08252_gb300 import et

    class Cfg(ctypes.Structure):
        _fields_ = et.et_config._fields_

    cfg = et.et_config()
    cfg.capacity_log2 = 10
    cfg.form = 1
    cfg.max_events = 4
    cfg.block_size = 256
    h = ctypes.c_void_p()
    st = et.lib.et_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == et.ET_ERR_CUDA
    assert b"CUDA" in et.lib.et_last_error(h)
    assert et.lib.et_destroy(h) == et.ET_OK


def test_invalid_config_rejected(libet):
    from paper_2302_08252_gb300 import et
    cfg = et.et_config()
    cfg.capacity_log2 = 3     # too small
    cfg.max_events = 1
    h = ctypes.c_void_p()
    assert et.lib.et_create(ctypes.byref(cfg), ctypes.byref(h)) == et.ET_ERR_INVALID
    assert not h.value


def test_score_columns_interleave_each_32_slab_group(libet):
    """The deposit rows' column order (host mirror of the device's): a permutation of the
    slabs; within a complete group of 32, slab s sits at 16 (s mod 2) + (s mod 32) / 2,
    so neighbouring slabs are 16 doubles (one 128-byte half) apart; the last incomplete
    group keeps its order; bad counts are refused."""
    out = (ctypes.c_uint32 * 128)()
    for ns in range(1, 129):
        assert libet.et_debug_score_columns(ns, out) == 0
        col = list(out)[:ns]
        assert sorted(col) == list(range(ns))
        full = (ns // 32) * 32
        for s in range(full):
            assert col[s] == (s & ~31) + 16 * (s & 1) + (s & 31) // 2
        for s in range(full, ns):
            assert col[s] == s
        for s in range(full - 1):
            if (s + 1) % 32:
                assert abs(col[s + 1] - col[s]) in (15, 16)
    assert libet.et_debug_score_columns(0, out) == 1
    assert libet.et_debug_score_columns(129, out) == 1
    assert libet.et_debug_score_columns(4, None) == 1


def test_aosoa128_needs_a_full_block(libet):
    from paper_2302_08252_gb300 import et
    cfg = et.et_config()
    cfg.capacity_log2 = 6     # 64 slots: less than one AoSoA-128 block
    cfg.layout = et.LAYOUT_AOSOA128
    cfg.max_events = 1
    cfg.block_size = 256
    h = ctypes.c_void_p()
    assert et.lib.et_create(ctypes.byref(cfg), ctypes.byref(h)) == et.ET_ERR_INVALID
    cfg.layout = 8            # no such layout
    cfg.capacity_log2 = 10
    assert et.lib.et_create(ctypes.byref(cfg), ctypes.byref(h)) == et.ET_ERR_INVALID


def test_split_interactions_validation(libet):
    """The split step kernels exist for the host-loop, graph and hybrid drivers, without
    instrumentation: other combinations are refused before any device work."""
    import torch
    from paper_2302_08252_gb300 import et

    def status(**kw):
        cfg = et.et_config()
        cfg.capacity_log2 = 10
        cfg.form = 1
        cfg.max_events = 1
        cfg.block_size = 256
        for k, v in kw.items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        st = et.lib.et_create(ctypes.byref(cfg), ctypes.byref(h))
        if h.value:
            et.lib.et_destroy(h)
        return st

    assert status(split_interactions=1, driver=et.DRIVER_PERSISTENT) == et.ET_ERR_INVALID
    assert status(split_interactions=1, instrument=1) == et.ET_ERR_INVALID
    assert status(split_interactions=2) == et.ET_ERR_INVALID
    if not torch.cuda.is_available():  # accepted: creation goes on to the (missing) device
        for d in (et.DRIVER_HOSTLOOP, et.DRIVER_GRAPH, et.DRIVER_HYBRID):
            assert status(split_interactions=1, driver=d) == et.ET_ERR_CUDA


@pytest.mark.parametrize("layout", ["aos", "soa", "aosoa8", "aosoa16", "aosoa32", "aosoa64",
                                    "aosoa128", "hotcold"])
def test_layout_mappings_tile_the_buffer(layout):
    """Every layout places the 15 leaves of `cap` records at distinct, naturally aligned
    byte ranges that exactly tile the cap * 64-byte buffer (the address formulas the
    device layout layer and the heatmap plotter share in form)."""
    from paper_2302_08252_gb300 import heatmap
    cap = 256
    used = np.zeros(cap * 64, dtype=np.int32)
    for i in range(cap):
        for f, (_, _, size) in enumerate(heatmap.LEAVES):
            a = heatmap.leaf_address(layout, i, f, cap)
            assert a % size == 0 and 0 <= a and a + size <= cap * 64
            used[a:a + size] += 1
    assert np.all(used == 1)


def test_noalloc_wrapper_refuses_bad_buffers(libet, geom):
    # every refusal happens on the host, before the library is called
    import torch

    from paper_2302_08252_gb300 import et
    from paper_2302_08252_gb300 import workloads as W
    tables = et.et_build_toy_tables()
    n_slabs, n_ev = len(geom["thickness"]), 4
    prim = torch.zeros(3 * 48, dtype=torch.uint8)
    score = torch.zeros((n_ev, n_slabs), dtype=torch.float64)
    ledger = torch.zeros((n_ev, 5), dtype=torch.float64)

    def call(t=tables, p=prim, n=3, seed=1, ev=n_ev, s=score, lg=ledger):
        return et.et_transport_noalloc(geom, t, p, n, seed, ev, s, lg)

    cases = [
        (dict(t=dict(tables, sigma=tables["sigma"][:, :, :256])), "sigma"),
        (dict(t=dict(tables, dedx=tables["dedx"][:1])), "dedx"),
        (dict(seed=1 << 32), "seed"),
        (dict(ev=0), "n_events"),
        (dict(p=np.zeros(3 * 48, np.uint8)), "primaries_device must be a CUDA tensor"),
        (dict(p=torch.zeros(3 * 48, dtype=torch.int8)), "primaries_device must be torch.uint8"),
        (dict(n=4), "primaries_device holds 144"),
        (dict(s=torch.zeros((n_ev, n_slabs), dtype=torch.float32)), "score_device must be"),
        (dict(s=torch.zeros((n_ev - 1, n_slabs), dtype=torch.float64)), "score_device holds"),
        (dict(s=torch.zeros((n_slabs, 2 * n_ev), dtype=torch.float64).t()), "contiguous"),
        (dict(lg=torch.zeros((n_ev, 4), dtype=torch.float64)), "ledger_device holds"),
        ({}, "primaries_device is not in device memory"),
    ]
    for kw, msg in cases:
        with pytest.raises((TypeError, ValueError), match=msg):
            call(**kw)
    assert W.PRIMARY_DTYPE.itemsize == 48
