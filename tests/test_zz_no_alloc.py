"""The allocation-free entry point (et_transport_noalloc) against the regular one.

For callers that cannot allocate device memory (inside another framework's memory pool,
under an allocation budget, or where cudaMalloc's implicit synchronisation is not
allowed), the library offers one call whose scratch lives in a fixed device array.  This
file checks, through the C ABI, that two calls in a row give the deposits, ledger and step
count of the context-based path (strict mode; deposits within the parity tolerance), and
that oversize requests are refused with a clear error.  It is named to be collected last.
"""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

from parity import DEPOSIT_RTOL, run_gpu

pytestmark = pytest.mark.gpu


def _close(a, b):
    return np.all(np.abs(a - b) <= DEPOSIT_RTOL * np.abs(b) + 1e-9)


def test_noalloc_matches_the_context_path_on_two_calls(geom):
    import torch

    from paper_2302_08252_gb300 import et
    p = W.small_electrons()
    n_events, n_slabs = 16, len(geom["thickness"])
    ref = run_gpu(geom, p, n_events, form="dense", layout="aos", driver="persistent", id_log=False)
    ref_steps = sum(ref["counters"]["steps"])
    tables = et.et_build_toy_tables()
    d_prim = torch.from_numpy(p.view(np.uint8).copy()).cuda()
    score = torch.full((n_events, n_slabs), 7.0, dtype=torch.float64, device="cuda")
    ledger = torch.full((n_events, 5), 7.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        steps = et.et_transport_noalloc(geom, tables, d_prim, len(p), 1, n_events, score, ledger)
        torch.cuda.synchronize()
        assert steps == ref_steps
        s = score.cpu().numpy()
        lg = ledger.cpu().numpy()
        assert _close(s, ref["score"])
        rl = ref["ledger"]  # injected, deposited_cont, below_cut, escaped, mass_created, mass_consumed
        assert np.array_equal(lg[:, 0], rl[:, 0])
        for mine, theirs in ((1, 2), (2, 3), (3, 4), (4, 5)):
            assert _close(lg[:, mine], rl[:, theirs])


def test_noalloc_refuses_oversize_batches(geom):
    import torch

    from paper_2302_08252_gb300 import et
    tables = et.et_build_toy_tables()
    n = et.NOALLOC_MAX_TRACKS + 1
    p = W.gun(n, 1.0, ptype=W.GAMMA)
    d_prim = torch.from_numpy(p.view(np.uint8).copy()).cuda()
    score = torch.zeros((n, len(geom["thickness"])), dtype=torch.float64, device="cuda")
    ledger = torch.zeros((n, 5), dtype=torch.float64, device="cuda")
    with pytest.raises(et.EtError) as e:
        et.et_transport_noalloc(geom, tables, d_prim, n, 1, n, score, ledger)
    assert e.value.status == et.ET_ERR_CAPACITY
    assert "ET_NOALLOC_MAX_TRACKS" in str(e.value)
