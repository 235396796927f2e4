"""The allocation-free force entry point, g6x_calc_dev_noalloc.

Callers that may not allocate device memory when they need a force (their
memory belongs to another framework's pool, or their loop cannot take the
device-wide synchronisation of cudaMalloc/cudaFree) use this call; its partial
sums live in one fixed device array instead of context memory that grows.
Checked here against g6x_calc_dev, through the C ABI, on two calls in a row
with different active blocks, so that anything the first call leaves in the
shared array would show up in the second.  Collected last on purpose."""
import numpy as np
import pytest

from paper_0902_4463_gb300 import g6gb as g6
from paper_0902_4463_gb300 import ics

pytestmark = pytest.mark.gpu

CID = 5


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_noalloc_matches_calc_dev_on_two_calls_in_a_row():
    import torch
    from paper_0902_4463_gb300 import build
    build.build()
    n, eps2, t_blk = 20000, 1e-5, 0.125
    st = ics.taylor_state(n, 17, t_blk)
    addr = np.arange(n, dtype=np.int32)
    g6.g6x_open_ex(CID, n, g6.G6X_NOALLOC_NI_MAX)
    stream = torch.cuda.Stream()
    try:
        g6.g6x_set_stream(CID, stream.cuda_stream)
        g6.g6x_set_j_particles(CID, addr, addr, st["tj"], st["m"], st["j0"] / 6.0,
                               st["a0"] / 2.0, st["v0"], st["x0"])
        perm = ics.permutation(n, 17)
        for m_act in (5000, 777):
            act = perm[:m_act]
            rec = np.zeros(m_act, dtype=g6.IREC)
            rec["x"], rec["v"], rec["index"] = st["x0"][act], st["v0"][act], act
            with torch.cuda.stream(stream):
                d_rec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
                nb = m_act * g6.OUT.itemsize
                d_ref = torch.empty(nb, dtype=torch.uint8, device="cuda")
                d_out = torch.full((nb,), 255, dtype=torch.uint8, device="cuda")
            g6.g6x_calc_dev(CID, t_blk, n, m_act, d_rec.data_ptr(), eps2, 0, d_ref.data_ptr())
            g6.g6x_calc_dev_noalloc(CID, t_blk, n, m_act, d_rec.data_ptr(), eps2,
                                    d_out.data_ptr())
            g6.g6x_sync(CID)
            ref = d_ref.cpu().numpy().view(g6.OUT)
            out = d_out.cpu().numpy().view(g6.OUT)
            for f in ("acc", "jerk"):
                e = _rel(out[f], ref[f])
                assert np.median(e) <= 1e-6 and e.max() <= 1e-5, (f, m_act)
            assert np.allclose(out["pot"], ref["pot"], rtol=1e-6, atol=0)
            assert np.array_equal(out["nnb"], ref["nnb"])
        # requests beyond the fixed maximum are refused before any work
        lib = g6.lib()
        assert lib.g6x_calc_dev_noalloc(CID, t_blk, n, g6.G6X_NOALLOC_NI_MAX + 1,
                                        d_rec.data_ptr(), eps2, d_out.data_ptr()) == g6.G6_EINVAL
    finally:
        g6.g6x_set_stream(CID, 0)
        g6.g6_close(CID)
