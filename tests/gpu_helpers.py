"""Shared helpers of the GPU parity tests: drive the C ABI and compare with
the oracle.  The oracle computes every expected value from the same seeded
inputs; nothing here feeds a CUDA result into the oracle."""
import numpy as np

from paper_0902_4463_gb300 import g6gb as g6


def load_j(cid, x0, v0, m, a0=None, j0=None, tj=0.0, index=None):
    """Store n j-particles in slots 0..n-1 (a0, j0 unscaled; stored as a/2, j/6)."""
    n = m.shape[0]
    a0 = np.zeros((n, 3)) if a0 is None else a0
    j0 = np.zeros((n, 3)) if j0 is None else j0
    addr = np.arange(n, dtype=np.int32)
    index = addr if index is None else np.asarray(index, dtype=np.int32)
    g6.g6x_set_j_particles(cid, addr, index, tj, m, j0 / 6.0, a0 / 2.0, v0, x0)


def sweep(cid, nj, xi, vi, idx_i, eps2, ti, h2=None):
    ni = xi.shape[0]
    g6.g6_set_ti(cid, ti)
    g6.g6calc_firsthalf(cid, nj, ni, idx_i, xi, vi, eps2, h2)
    return g6.g6calc_lasthalf2(cid, nj, ni, eps2)


def rel_err_vec(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def abs_scale_err(a, b, scale):
    """|a - b| / scale: error relative to the sum of magnitudes of the terms."""
    return np.linalg.norm(a - b, axis=1) / scale


def check_nn(orc_nnb, orc_nnr2, gpu_nnb, xi, xj, idx_j, rtol=1e-5):
    """Nearest-neighbour parity: the GPU's choice must be a valid nearest
    neighbour: its FP64 distance within rtol of the oracle minimum.  Returns
    the fraction of exact index matches."""
    pos_of = {int(k): p for p, k in enumerate(idx_j)}
    for i in range(xi.shape[0]):
        if orc_nnb[i] < 0:
            assert gpu_nnb[i] == -1
            continue
        assert gpu_nnb[i] >= 0
        p = pos_of[int(gpu_nnb[i])]
        d2 = float(np.sum((xj[p] - xi[i]) ** 2))
        assert d2 <= orc_nnr2[i] * (1 + rtol) + 1e-300, (i, d2, orc_nnr2[i])
    return float(np.mean(idx_j[orc_nnb] == gpu_nnb))
