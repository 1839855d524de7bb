"""Bounds checks without a sanitizer: every device buffer the library allocates comes from
a test allocator that surrounds it with guard bytes of a known pattern.  Runs that end
normally and runs that overflow the track buffers (which the library reports as
ET_ERR_CAPACITY) must leave every guard byte intact: no write lands outside a buffer."""
import numpy as np
import pytest

from paper_2302_08252_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 4096
PATTERN = 0xA5


class GuardedAllocator:
    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.bad = []  # buffers whose guards were found overwritten (callbacks cannot raise)

    def alloc(self, nbytes, stream):
        t = self.torch.full((nbytes + 2 * GUARD,), PATTERN, dtype=self.torch.uint8, device="cuda")
        ptr = t.data_ptr() + GUARD
        self.live[ptr] = (t, nbytes)
        return ptr

    def free(self, ptr):
        t, n = self.live.pop(ptr)
        if not self._intact(t, n):
            self.bad.append((ptr, n))

    def _intact(self, t, n):
        self.torch.cuda.synchronize()
        head = t[:GUARD].cpu().numpy()
        tail = t[GUARD + n:].cpu().numpy()
        return bool(np.all(head == PATTERN) and np.all(tail == PATTERN))

    def check_all(self):
        for ptr, (t, n) in self.live.items():
            assert self._intact(t, n), f"guard bytes around a {n}-byte buffer overwritten"


@pytest.mark.parametrize("form", ["dense", "sparse"])
@pytest.mark.parametrize("driver", ["persistent", "hostloop"])
def test_no_write_outside_buffers(geom, form, driver):
    from paper_2302_08252_gb300 import et
    ga = GuardedAllocator()
    ctx = et.make_context(geom, max_events=16, capacity_log2=7, driver=driver, layout="aosoa32",
                          form=et.FORM_DENSE if form == "dense" else et.FORM_SPARSE,
                          allocator=(ga.alloc, ga.free), id_log=True, id_log_capacity=256)
    assert len(ga.live) > 5
    # a run that fits
    et.et_inject(ctx, W.gun(2, 2.0))
    et.et_run_until_empty(ctx)
    ga.check_all()
    # a run that overflows the track buffers and the id log
    et.et_reset(ctx)
    et.et_inject(ctx, W.small_electrons())
    with pytest.raises(et.EtError) as e:
        et.et_run_until_empty(ctx)
    assert e.value.status == et.ET_ERR_CAPACITY
    ga.check_all()
    et.et_destroy(ctx)
    assert not ga.live and not ga.bad
