"""Failure handling without a GPU fault: device-allocation failures injected on
the host through the library's allocator hook (an allocator that refuses
after a set number of calls).  The library must report G6_ENOMEM, give back
everything it had allocated, and stay usable: the same context (or a new one)
works once allocations succeed again."""
import numpy as np
import pytest

from paper_0902_4463_gb300 import g6gb as g6
from paper_0902_4463_gb300 import ics
from tests.gpu_helpers import load_j, rel_err_vec, sweep

pytestmark = pytest.mark.gpu

CID = 11


class RefusingAllocator:
    """Device memory from PyTorch's caching allocator; refuses every call
    after `allow` successful ones."""

    def __init__(self):
        import torch
        self.torch = torch
        self.allow = 10 ** 9
        self.calls = 0
        self.live = {}
        self.hooks = (g6.ALLOC_FN(self._alloc), g6.FREE_FN(self._free))

    def _alloc(self, nbytes, user):
        self.calls += 1
        if self.calls > self.allow:
            return None
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, user):
        self.live.pop(ptr, None)


@pytest.fixture()
def refusing():
    from paper_0902_4463_gb300 import build
    build.build()
    ra = RefusingAllocator()
    assert g6.lib().g6x_set_allocator(ra.hooks[0], ra.hooks[1], None) == 0
    try:
        yield ra
    finally:
        g6.lib().g6_close(CID)
        g6.g6x_use_cuda_allocator()


def test_open_fails_cleanly_and_the_next_open_works(refusing, orc):
    for allow in (0, 1, 3, 6):
        refusing.calls, refusing.allow = 0, allow
        assert g6.lib().g6x_open_ex(CID, 4096, 4096) == g6.G6_ENOMEM
        assert not refusing.live, allow            # everything given back
    refusing.allow = 10 ** 9
    assert g6.lib().g6x_open_ex(CID, 4096, 4096) == 0
    n, eps2 = 1024, 1e-4
    m, x, v = ics.plummer(n, 1)
    idx = np.arange(n)
    load_j(CID, x, v, m)
    acc, *_ = sweep(CID, n, x, v, idx, eps2, 0.0)
    oa, *_ = orc.force(x, v, idx, x, v, m, idx, eps2)
    assert np.median(rel_err_vec(acc, oa)) <= 1e-6


def test_calculation_that_must_grow_fails_then_succeeds(refusing, orc):
    n, eps2 = 32768, 1e-5
    assert g6.lib().g6x_open_ex(CID, n, n) == 0
    m, x, v = ics.plummer(n, 2)
    idx = np.arange(n)
    load_j(CID, x, v, m)
    small = np.arange(64)
    sweep(CID, n, x[small], v[small], small, eps2, 0.0)   # partial buffers for 64
    refusing.allow = refusing.calls                        # no more device memory
    with pytest.raises(g6.G6Error) as e:
        sweep(CID, n, x, v, idx, eps2, 0.0)                # needs larger partial buffers
    assert e.value.code == g6.G6_ENOMEM
    # the context is intact: small calls still work, and the large one once
    # memory is available again
    acc, *_ = sweep(CID, n, x[small], v[small], small, eps2, 0.0)
    refusing.allow = 10 ** 9
    acc, *_ = sweep(CID, n, x, v, idx, eps2, 0.0)
    sel = idx[:512]
    oa, *_ = orc.force(x[sel], v[sel], sel, x, v, m, idx, eps2)
    ea = rel_err_vec(acc[:512], oa)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5


def test_batch_creation_fails_cleanly(refusing):
    for allow in (0, 5, 10, 13):           # the batch makes 14 device allocations
        refusing.calls, refusing.allow = 0, allow
        with pytest.raises(g6.G6Error) as e:
            g6.G6Batch([300, 1000, 70])
        assert e.value.code == g6.G6_ENOMEM
        assert not refusing.live, allow
    refusing.allow = 10 ** 9
    b = g6.G6Batch([300, 1000, 70])
    assert b.launch_count() == 0
    b.close()
    assert not refusing.live
