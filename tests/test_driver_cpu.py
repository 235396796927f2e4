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


def _circular(t):
    """Acceleration and jerk on the unit circular orbit of unit angular
    frequency: a = -(cos t, sin t, 0), j = (sin t, -cos t, 0); every
    derivative has magnitude 1, so Aarseth's request is sqrt(eta)."""
    a = -np.array([[np.cos(t), np.sin(t), 0.0]])
    j = np.array([[np.sin(t), -np.cos(t), 0.0]])
    return a, j


def test_noise_aware_step_with_zero_noise_is_the_plain_criterion():
    build.build()
    rng = np.random.default_rng(11)
    n = 300
    dt = np.ldexp(1.0, -rng.integers(3, 12, n))
    t_blk = 0.5
    xp, vp = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    a0, j0 = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    a1 = a0 + j0 * dt[:, None] + rng.normal(size=(n, 3)) * dt[:, None] ** 2
    j1 = j0 + rng.normal(size=(n, 3)) * dt[:, None]
    args = (t_blk, t_blk - dt, dt, 0.02, 0.5, 2.0 ** -40, xp, vp, a0, j0, a1, j1)
    # the wrapper calls g6h_correct_block_ex; call g6h_correct_block itself too
    x1, v1, dtn, small = g6gb.g6h_correct_block(*args, force_noise=0.0)
    xr, vr, dtr = xp.copy(), vp.copy(), np.empty(n)
    p = g6gb._p
    nsmall = g6gb.lib().g6h_correct_block(n, t_blk, p(np.ascontiguousarray(t_blk - dt)), p(dt),
                                          0.02, 0.5, 2.0 ** -40, p(xr), p(vr), p(a0), p(j0),
                                          p(a1), p(j1), p(dtr))
    assert nsmall == small == 0
    assert np.array_equal(x1, xr) and np.array_equal(v1, vr) and np.array_equal(dtn, dtr)
    with np.testing.assert_raises(g6gb.G6Error):
        g6gb.g6h_correct_block(*args, force_noise=-1e-7)


def test_noise_aware_step_does_not_collapse_on_force_noise():
    """Sect. 3.1: with low-precision forces the step sizes of a small eta
    shrink further.  On a smooth orbit whose forces carry a relative error of
    1e-7, the plain criterion reads the noise as a large third derivative and halves a
    step that the orbit itself allows; allowing for that error keeps it."""
    build.build()
    eta, h, t_blk = 1e-4, 2.0 ** -10, 1.0
    a0, j0 = _circular(t_blk - h)
    a1, j1 = _circular(t_blk)
    z = np.zeros((1, 3))
    rng = np.random.default_rng(5)
    worst = []
    for _ in range(20):
        na = a1 * (1 + 1e-7 * rng.choice([-1.0, 1.0], size=(1, 3)))
        nj = j1 * (1 + 1e-7 * rng.choice([-1.0, 1.0], size=(1, 3)))
        args = (t_blk, [t_blk - h], [h], eta, 2.0 ** -3, 2.0 ** -40, z, z, a0, j0, na, nj)
        _, _, plain, _ = g6gb.g6h_correct_block(*args)
        _, _, aware, _ = g6gb.g6h_correct_block(*args, force_noise=1e-7)
        worst.append(plain[0])
        assert aware[0] >= h
    assert min(worst) < h                  # the plain criterion does shrink the step
    # without noise both keep the step (the orbit allows sqrt(eta) = 0.01)
    args = (t_blk, [t_blk - h], [h], eta, 2.0 ** -3, 2.0 ** -40, z, z, a0, j0, a1, j1)
    assert g6gb.g6h_correct_block(*args)[2][0] >= h
    assert g6gb.g6h_correct_block(*args, force_noise=1e-7)[2][0] >= h


def test_noise_aware_step_never_shortens_a_step():
    """The allowance takes the larger of the plain and the reduced request:
    on random states (including near-zero jerks, where a reduced second
    derivative of 0 alone would collapse the request) no step comes out
    shorter than the plain criterion gives."""
    build.build()
    rng = np.random.default_rng(13)
    n = 4000
    dt = np.ldexp(1.0, -rng.integers(2, 30, n))
    t_blk = 1.0
    z = np.zeros((n, 3))
    a0 = rng.normal(size=(n, 3))
    j0 = rng.normal(size=(n, 3)) * np.where(rng.random(n) < 0.3, 1e-9, 1.0)[:, None]
    a1 = a0 * (1 + 1e-6 * rng.normal(size=(n, 3))) + j0 * dt[:, None]
    j1 = j0 * (1 + 1e-3 * rng.normal(size=(n, 3)))
    args = (t_blk, t_blk - dt, dt, 1e-3, 0.5, 2.0 ** -60, z, z, a0, j0, a1, j1)
    plain = g6gb.g6h_correct_block(*args)[2]
    for noise in (1e-9, 1e-7, 1e-5, 0.5):
        aware = g6gb.g6h_correct_block(*args, force_noise=noise)[2]
        assert np.all(aware >= plain), noise
    assert np.any(g6gb.g6h_correct_block(*args, force_noise=1e-7)[2] > plain)


def test_noise_aware_step_still_shrinks_on_real_structure():
    """A step too long for the orbit (eta = 0.01 allows 0.1) is halved with and
    without the noise allowance: at h = 1/4 the allowance is ~1e-5 of the third derivative."""
    build.build()
    eta, h, t_blk = 0.01, 0.25, 1.0
    a0, j0 = _circular(t_blk - h)
    a1, j1 = _circular(t_blk)
    z = np.zeros((1, 3))
    args = (t_blk, [t_blk - h], [h], eta, 0.5, 2.0 ** -40, z, z, a0, j0, a1, j1)
    plain = g6gb.g6h_correct_block(*args)[2][0]
    aware = g6gb.g6h_correct_block(*args, force_noise=1e-7)[2][0]
    assert plain == aware == 0.0625


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


def test_large_blocks_on_host_threads_match_the_serial_corrector():
    """Blocks of 8192 and more particles are corrected on the host thread
    pool; the results equal those of the same particles corrected in serial
    pieces, bit for bit (steps below the minimum counted the same way)."""
    build.build()
    rng = np.random.default_rng(21)
    n = 30000
    dt = np.ldexp(1.0, -rng.integers(3, 20, n))
    t_blk = 0.75
    xp, vp = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    a0, j0 = rng.normal(size=(n, 3)), rng.normal(size=(n, 3)) * 3
    a1 = a0 + j0 * dt[:, None] + rng.normal(size=(n, 3)) * dt[:, None] ** 2
    j1 = j0 + rng.normal(size=(n, 3)) * dt[:, None] * 50
    args = (t_blk, t_blk - dt, dt, 0.01, 0.5, 2.0 ** -12, xp, vp, a0, j0, a1, j1)
    x1, v1, dtn, small = g6gb.g6h_correct_block(*args)
    assert small > 0                         # some steps fall below the floor
    xs, vs, ds, ss = [], [], [], 0
    for k0 in range(0, n, 5000):
        sl = slice(k0, k0 + 5000)
        part = g6gb.g6h_correct_block(t_blk, (t_blk - dt)[sl], dt[sl], 0.01, 0.5, 2.0 ** -12,
                                      xp[sl], vp[sl], a0[sl], j0[sl], a1[sl], j1[sl])
        xs.append(part[0]); vs.append(part[1]); ds.append(part[2]); ss += part[3]
    assert np.array_equal(x1, np.concatenate(xs)) and np.array_equal(v1, np.concatenate(vs))
    assert np.array_equal(dtn, np.concatenate(ds)) and small == ss


# ------------------------------------------------ host thread pool
def test_host_thread_pool(tmp_path):
    """The library's host pool (g6gb_pool.h) in a standalone C++ test: every
    index once, back-to-back runs, sleeping workers, nested and concurrent
    callers (a deadlock would trip the timeout)."""
    import os
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = str(tmp_path / "pool_test")
    r = subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-pthread",
                        "-I", os.path.join(root, "paper_0902_4463_gb300", "csrc"),
                        os.path.join(root, "tests", "cpp", "pool_test.cpp"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "pool ok" in r.stdout, r.stderr
