"""The allocation-free force entry point, g6x_calc_dev_noalloc.

Callers that may not allocate device memory when they need a force (their
memory belongs to another framework's pool, or their loop cannot take the
device-wide synchronisation of cudaMalloc/cudaFree) use this call; its partial
sums live in one fixed device array instead of context memory that grows.
Checked here against g6x_calc_dev and against the FP64 oracle, through the C
ABI, on two calls in a row with different active blocks, so that anything the
first call leaves in the shared array would show up in the second; and at the
largest block it accepts against N = 2^20, where the launch must shrink its
grid so that the partial sums fit the array.  Collected last on purpose."""
import numpy as np
import pytest

from paper_0902_4463_gb300 import g6gb as g6
from paper_0902_4463_gb300 import ics

pytestmark = pytest.mark.gpu

CID = 5


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def _oracle_check(orc, out, st, act, t_blk, eps2, sample):
    """Sampled i-particles of one call against the FP64 oracle (median
    relative error <= 1e-6, max <= 1e-5 for acceleration and potential)."""
    n = st["m"].shape[0]
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t_blk)
    s = act[sample]
    oa, oj, op, onn, onr = orc.force(st["x0"][s], st["v0"][s], s, xp, vp, st["m"],
                                     np.arange(n), eps2)
    ea = _rel(out["acc"][sample], oa)
    ep = np.abs(out["pot"][sample] - op) / np.abs(op)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5, (np.median(ea), ea.max())
    assert np.median(ep) <= 1e-6 and ep.max() <= 1e-5, (np.median(ep), ep.max())
    assert np.mean(out["nnb"][sample] == onn) >= 0.99


def test_noalloc_matches_calc_dev_on_two_calls_in_a_row(orc):
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
            _oracle_check(orc, out, st, act, t_blk, eps2, np.arange(0, m_act, 7))
        # requests beyond the fixed maximum are refused before any work
        lib = g6.lib()
        assert lib.g6x_calc_dev_noalloc(CID, t_blk, n, g6.G6X_NOALLOC_NI_MAX + 1,
                                        d_rec.data_ptr(), eps2, d_out.data_ptr()) == g6.G6_EINVAL
    finally:
        g6.g6x_set_stream(CID, 0)
        g6.g6_close(CID)


def test_noalloc_largest_block_shrinks_its_grid(orc):
    # ni = G6X_NOALLOC_NI_MAX against N = 2^20: the launch g6x_calc_dev would
    # use writes more partial sums than the array holds, so the call must run
    # on a smaller grid whose partials fit, and still give the right forces.
    import torch
    from paper_0902_4463_gb300 import build
    build.build()
    n, eps2, t_blk = 1 << 20, 1e-6, 2.0 ** -10
    ni = g6.G6X_NOALLOC_NI_MAX
    st = ics.taylor_state(n, 3, t_blk, dt_levels=None)
    addr = np.arange(n, dtype=np.int32)
    g6.g6x_open_ex(CID, n, ni)
    stream = torch.cuda.Stream()
    try:
        g6.g6x_set_stream(CID, stream.cuda_stream)
        g6.g6x_set_j_particles(CID, addr, addr, st["tj"], st["m"], st["j0"] / 6.0,
                               st["a0"] / 2.0, st["v0"], st["x0"])
        act = np.sort(ics.permutation(n, 9)[:ni])
        rec = np.zeros(ni, dtype=g6.IREC)
        rec["x"], rec["v"], rec["index"] = st["x0"][act], st["v0"][act], act
        with torch.cuda.stream(stream):
            d_rec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
            d_ref = torch.empty(ni * g6.OUT.itemsize, dtype=torch.uint8, device="cuda")
            d_out = torch.full((ni * g6.OUT.itemsize,), 255, dtype=torch.uint8, device="cuda")
        g6.g6x_calc_dev(CID, t_blk, n, ni, d_rec.data_ptr(), eps2, 0, d_ref.data_ptr())
        g6.g6x_sync(CID)
        full = g6.g6x_last_config(CID)
        g6.g6x_calc_dev_noalloc(CID, t_blk, n, ni, d_rec.data_ptr(), eps2, d_out.data_ptr())
        g6.g6x_sync(CID)
        small = g6.g6x_last_config(CID)
        itile = small["ti"] * small["ni_per"]
        n_itile = -(-ni // itile)
        slots = g6.G6X_NOALLOC_SCRATCH_BYTES // 72
        assert (full["grid"] + n_itile) * itile > slots      # would not fit
        assert small["grid"] < full["grid"]
        assert (small["grid"] + n_itile) * itile <= slots    # the shrunken launch fits
        ref = d_ref.cpu().numpy().view(g6.OUT)
        out = d_out.cpu().numpy().view(g6.OUT)
        e = _rel(out["acc"], ref["acc"])
        assert np.median(e) <= 1e-6 and e.max() <= 1e-5
        assert np.mean(out["nnb"] == ref["nnb"]) >= 0.999
        _oracle_check(orc, out, st, act, t_blk, eps2, np.arange(0, ni, 64))
    finally:
        g6.g6x_set_stream(CID, 0)
        g6.g6_close(CID)
