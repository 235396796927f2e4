"""Host side of the path (row a6): the C++ driver's block corrector and
time-step choice against the oracle, on the CPU (no GPU call)."""
import numpy as np

from paper_0902_4463_gb300 import build, g6gb


def test_correct_block_matches_oracle(orc):
    build.build()
    rng = np.random.default_rng(7)
    n = 500
    t_blk = 0.375
    dt = np.ldexp(1.0, -rng.integers(3, 12, n))
    t0 = t_blk - dt
    xp, vp = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    a0, j0 = rng.normal(size=(n, 3)), rng.normal(size=(n, 3)) * 3
    a1 = a0 + j0 * dt[:, None] + rng.normal(size=(n, 3)) * dt[:, None] ** 2
    j1 = j0 + rng.normal(size=(n, 3)) * dt[:, None]
    eta, dt_max, dt_min = 0.01, 2.0 ** -2, 2.0 ** -40
    x1, v1, dtn, small = g6gb.g6h_correct_block(t_blk, t0, dt, eta, dt_max, dt_min,
                                                xp, vp, a0, j0, a1, j1)
    assert small == 0
    agree = 0
    for k in range(n):
        ox, ov, o2, o3 = orc.hermite_correct(dt[k], xp[k], vp[k], a0[k], j0[k], a1[k], j1[k])
        assert np.allclose(x1[k], ox, rtol=1e-13, atol=1e-13)
        assert np.allclose(v1[k], ov, rtol=1e-13, atol=1e-13)
        req = orc.aarseth_dt(a1[k], j1[k], o2 + dt[k] * o3, o3, eta)
        odt = orc.block_dt(dt[k], req, t_blk, dt_max, dt_min)
        agree += dtn[k] == odt
        # a step decision can only differ where the request sits on a power of 2
        if dtn[k] != odt:
            assert abs(np.log2(req) - np.round(np.log2(req))) < 1e-12
    assert agree == n


def test_correct_block_flags_steps_below_minimum():
    build.build()
    z = np.zeros((1, 3))
    a = np.array([[1.0, 0, 0]])
    j = np.array([[0, 1e9, 0]])
    x1, v1, dtn, small = g6gb.g6h_correct_block(1e-9, 0.0, 1e-9, 1e-6, 2.0 ** -4, 1e-3,
                                                z, z, a, j, a, j)
    assert small == 1 and dtn[0] == -1.0


# ------------------------------------------------ checkpoint file parser
# The layout written by g6h_checkpoint (host byte order, little-endian):
# magic, int64 n, nbuckets, nblocks, nactive, hist[64], 6 doubles of
# parameters, the particle arrays, the scheduler buckets, an FNV-1a hash.
# On a host without a GPU a consistent file gets as far as the first library
# call (the cluster id is not open); an inconsistent one is refused before.

def _fnv1a(b):
    h = 1469598103934665603
    for c in b:
        h ^= c
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _ckpt_bytes(n=3, dt=(0.125, 0.25, 0.125), t=(0.0, 0.0, 0.0), buckets=None, magic=b"G6HCKPT1",
                hash_fix=0):
    import struct
    dt, t = np.asarray(dt, float), np.asarray(t, float)
    if buckets is None:
        due = {}
        for k in range(n):
            due.setdefault(t[k] + dt[k], []).append(k)
        buckets = sorted(due.items())
    b = bytearray(magic)
    b += struct.pack("<4q", n, len(buckets), 7, 21)
    b += np.zeros(64, dtype="<i8").tobytes()
    b += struct.pack("<6d", 1e-4, 0.01, 0.001, 0.0625, 2.0 ** -40, 0.0)
    rng = np.random.default_rng(1)
    b += np.full(n, 1.0 / n).astype("<f8").tobytes()
    for _ in range(4):
        b += rng.normal(size=(n, 3)).astype("<f8").tobytes()
    b += t.astype("<f8").tobytes() + dt.astype("<f8").tobytes()
    for tb, ids in buckets:
        b += struct.pack("<dq", tb, len(ids)) + np.asarray(ids, dtype="<i4").tobytes()
    b += struct.pack("<Q", (_fnv1a(bytes(b)) + hash_fix) & 0xFFFFFFFFFFFFFFFF)
    return bytes(b)


def _restore(tmp_path, data, name="c.ckpt"):
    import ctypes
    build.build()
    p = tmp_path / name
    if data is not None:
        p.write_bytes(data)
    err = ctypes.c_int(0)
    h = g6gb.lib().g6h_restore(7, str(p).encode(), ctypes.byref(err))
    assert not h
    return err.value


def test_checkpoint_parser_accepts_a_consistent_file(tmp_path):
    # consistent: refused only by the library call (cluster 7 is not open)
    assert _restore(tmp_path, _ckpt_bytes()) in (g6gb.G6_ENOTOPEN, g6gb.G6_ENODEV)


def test_checkpoint_parser_rejects_damage(tmp_path):
    good = _ckpt_bytes()
    assert _restore(tmp_path, None, "missing.ckpt") == g6gb.G6_EIO
    assert _restore(tmp_path, _ckpt_bytes(magic=b"G6HCKPT0")) == g6gb.G6_EINVAL
    assert _restore(tmp_path, good[:-9]) == g6gb.G6_EINVAL            # truncated
    assert _restore(tmp_path, good + b"\0") == g6gb.G6_EINVAL         # trailing bytes
    flipped = bytearray(good)
    flipped[700] ^= 1
    assert _restore(tmp_path, bytes(flipped)) == g6gb.G6_EINVAL       # hash
    assert _restore(tmp_path, _ckpt_bytes(hash_fix=1)) == g6gb.G6_EINVAL
    # scheduler inconsistent with t + dt, a particle filed twice or never
    assert _restore(tmp_path, _ckpt_bytes(buckets=[(0.125, [0, 2]), (0.5, [1])])) == g6gb.G6_EINVAL
    assert _restore(tmp_path, _ckpt_bytes(buckets=[(0.125, [0, 0]), (0.25, [1])])) == g6gb.G6_EINVAL
    assert _restore(tmp_path, _ckpt_bytes(buckets=[(0.125, [0, 2])])) == g6gb.G6_EINVAL
    assert _restore(tmp_path, _ckpt_bytes(dt=(0.125, 0.0, 0.125))) == g6gb.G6_EINVAL
