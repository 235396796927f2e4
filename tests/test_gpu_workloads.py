"""GPU parity at the benchmark's sizes and through the Hermite driver.

* Plummer N = 32768 (eps2 = 1e-5): every i-particle against all j, DS and FP64,
  compared element by element with the oracle.
* Plummer N = 2^20 (eps2 = 1e-6), m = N, in the launch configuration the
  benchmark times: 256 sampled i-particles checked against the oracle.
* Neighbour lists (Sect. 4) on a Plummer sphere with binaries, h2 = 1e-4.
* The C++ Hermite block-time-step driver (Sect. 2) on a Kepler orbit against
  the closed-form solution, and on Plummer N = 1024 to t = 0.25 with eta = 0.01
  against the oracle's integrator: energy drift within 2x the oracle's.
"""
import math

import numpy as np
import pytest

from paper_0902_4463_gb300 import g6gb as g6
from paper_0902_4463_gb300 import ics
from tests.gpu_helpers import check_nn, load_j, rel_err_vec, sweep

pytestmark = pytest.mark.gpu

CID = 3


@pytest.fixture()
def open_ctx():
    from paper_0902_4463_gb300 import build
    build.build()
    opened = []

    def _open(nj, ni):
        g6.g6x_open_ex(CID, nj, ni)
        opened.append(CID)
        return CID

    yield _open
    for c in opened:
        g6.g6_close(c)


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_plummer_32768_full_sweep(open_ctx, orc, prec):
    n, eps2 = 32768, 1e-5
    m, x, v = ics.plummer(n, 2)
    idx = np.arange(n)
    cid = open_ctx(n, n)
    g6.g6x_set_precision(cid, prec)
    load_j(cid, x, v, m)
    acc, jerk, pot, nnb = sweep(cid, n, x, v, idx, eps2, 0.0)
    oa, oj, op, onn, onr = orc.force(x, v, idx, x, v, m, idx, eps2)
    med, mx = (1e-6, 1e-5) if prec == g6.G6X_PREC_DS else (1e-12, 1e-10)
    ea, ej = rel_err_vec(acc, oa), rel_err_vec(jerk, oj)
    ep = np.abs(pot - op) / np.abs(op)
    assert np.median(ea) <= med and ea.max() <= mx, (np.median(ea), ea.max())
    assert np.median(ej) <= med and ej.max() <= mx, (np.median(ej), ej.max())
    assert np.median(ep) <= med and ep.max() <= mx
    assert check_nn(onn, onr, nnb, x, x, idx) > 0.999


def test_full_size_sampled_in_bench_configuration(open_ctx, orc):
    # N = 2^20, every particle active, j predicted from t_j = 0 to 2^-10
    n, eps2, t_blk = 1 << 20, 1e-6, 2.0 ** -10
    st = ics.taylor_state(n, 3, t_blk, dt_levels=None)
    cid = open_ctx(n, n)
    load_j(cid, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    idx = np.arange(n)
    acc, jerk, pot, nnb = sweep(cid, n, st["x0"], st["v0"], idx, eps2, t_blk)
    cfg = g6.g6x_last_config(cid)
    assert cfg["variant"] == 9 and cfg["grid"] == 152 * 4 * 8
    sample = ics.permutation(n, 99)[:256]
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t_blk)
    oa, oj, op, onn, onr = orc.force(st["x0"][sample], st["v0"][sample], sample, xp, vp,
                                     st["m"], idx, eps2)
    ea, ej = rel_err_vec(acc[sample], oa), rel_err_vec(jerk[sample], oj)
    ep = np.abs(pot[sample] - op) / np.abs(op)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5, (np.median(ea), ea.max())
    assert np.median(ej) <= 1e-6 and ej.max() <= 1e-5, (np.median(ej), ej.max())
    assert np.median(ep) <= 1e-6 and ep.max() <= 1e-5
    check_nn(onn, onr, nnb[sample], st["x0"][sample], xp, idx)
    # properties that hold at any size: finite, attractive on average
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(jerk)) and np.all(pot < 0)


def _list_ok(gpu_ids, orc_pos, idx_j, xi, xj, h2, tol=1e-6):
    """Lists agree as sets, except members within tol of the radius."""
    g = set(int(k) for k in gpu_ids)
    o = set(int(idx_j[p]) for p in orc_pos)
    for k in g ^ o:
        r2 = float(np.sum((xj[k] - xi) ** 2))
        assert abs(r2 - h2) <= tol * h2, (k, r2, h2)


@pytest.mark.parametrize("maxnb", [64, 256, 1024])
@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_neighbour_lists_plummer_with_binaries(open_ctx, orc, prec, maxnb):
    # Sect. 4 lists at the list lengths 64, 256 (the paper's) and 1024
    # against the oracle's lists truncated at the same length: contents,
    # ascending order, overflow flags.  The list parts start with room for a
    # few entries, so the first read computes the lists once more with
    # larger parts; a second calculation of the same block needs no more.
    n, eps2 = 8192, 1e-8
    m, x, v, pairs = ics.plummer_with_binaries(n, 5)
    idx = np.arange(n)
    cid = open_ctx(n, n)
    g6.g6x_set_precision(cid, prec)
    g6.g6x_set_max_neighbours(cid, maxnb)
    assert g6.g6x_max_neighbours(cid) == maxnb
    load_j(cid, x, v, m)
    act = np.sort(ics.permutation(n, 5)[:600])
    h2 = np.full(act.size, 1e-4)
    h2[::7] = 0.05 ** 2                       # some long lists
    h2[::11] = 0.3 ** 2                       # some that overflow 64 and 256
    h2[::13] = 1.0                            # some that overflow 1024
    nblen, nbl, nov = orc.neighbours(x[act], act, x, idx, h2, maxnb=maxnb)
    for rep in range(2):
        acc, jerk, pot, nnb = sweep(cid, n, x[act], v[act], act, eps2, 0.0, h2=h2)
        rc = g6.g6_read_neighbour_list(cid)
        assert g6.g6x_list_reruns(cid) == 1          # only the first read ran again
        assert rc == (g6.G6_EOVERFLOW if nov else 0) and nov > 0
        for q in range(act.size):
            rc_q, ln, ids = g6.g6_get_neighbour_list(cid, q)
            if nblen[q] <= maxnb:
                assert abs(ln - nblen[q]) <= 2
                _list_ok(ids, nbl[q, :nblen[q]], idx, x[act[q]], x, h2[q])
                assert list(ids) == sorted(ids)            # ascending j-slot
            else:
                assert ln > maxnb and rc_q == g6.G6_EOVERFLOW
                assert len(ids) == maxnb and list(ids) == sorted(ids)
                # truncation keeps the lowest j-slots: the oracle's first maxnb
                # up to members within rounding of the radius
                _list_ok(ids, nbl[q, :maxnb], idx, x[act[q]], x, h2[q])
    # forces are unchanged by list building
    oa, *_ = orc.force(x[act], v[act], act, x, v, m, idx, eps2)
    ea = rel_err_vec(acc, oa)
    lim = (1e-6, 1e-5) if prec == g6.G6X_PREC_DS else (1e-12, 1e-10)
    assert np.median(ea) <= lim[0] and ea.max() <= lim[1]


@pytest.mark.parametrize("m", [16, 300])
@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_neighbour_lists_every_list_shape(open_ctx, orc, m, prec):
    # Every DS list shape, forced, against the oracle's lists: the split-j
    # shapes merge the ascending runs of their j-groups at the end of each
    # segment, so contents, order, truncation at the list length (the lowest
    # j-slots) and the counts must match whatever the shape.  Each shape runs
    # twice: with its own grid (many partials per i-tile: the separate
    # reduction concatenates the lists) and with two CTAs per i-tile (the
    # last CTA of each i-tile concatenates them inside the force launch; the
    # all-FP64 kernel always has the separate reduction).  At m = 16 the
    # separate reduction takes one CTA per i-particle (more than 64 partials
    # each), at m = 300 one warp for most shapes.
    n, eps2, maxnb = 32768, 1e-8, 256
    m_, x, v, pairs = ics.plummer_with_binaries(n, 6)
    idx = np.arange(n)
    cid = open_ctx(n, n)
    g6.g6x_set_precision(cid, prec)
    load_j(cid, x, v, m_)
    act = np.sort(ics.permutation(n, 6)[:m])
    h2 = np.full(act.size, 1e-4)
    h2[::5] = 0.05 ** 2
    h2[::7] = 0.3 ** 2                        # past the list length
    h2[::9] = 1.0
    nblen, nbl, nov = orc.neighbours(x[act], act, x, idx, h2, maxnb=maxnb)
    oa, *_ = orc.force(x[act], v[act], act, x, v, m_, idx, eps2)
    shapes = [k for k in range(g6.g6x_variant_count())
              if g6.g6x_variant_info(k)["list"] == 1 and g6.g6x_variant_info(k)["prec"] == prec]
    assert len(shapes) >= (7 if prec == g6.G6X_PREC_DS else 1)
    fusable = prec == g6.G6X_PREC_DS
    lim = (1e-6, 1e-5) if prec == g6.G6X_PREC_DS else (1e-12, 1e-10)
    sweep(cid, n, x[act], v[act], act, eps2, 0.0, h2=h2)     # the prediction, once
    try:
        for k, fused in ((k, f) for k in shapes for f in (False, True)):
            info = g6.g6x_variant_info(k)
            n_itile = -(-m // (info["ti"] * info["ni_per"]))
            g6.g6x_set_variant(cid, k, 2 * n_itile if fused else 0)
            l0 = g6.g6x_launch_count(cid)
            acc, jerk, pot, nnb = sweep(cid, n, x[act], v[act], act, eps2, 0.0, h2=h2)
            launches = g6.g6x_launch_count(cid) - l0
            cfg = g6.g6x_last_config(cid)
            assert cfg["variant"] == k
            if fused:
                assert cfg["grid"] == 2 * n_itile, (k, cfg)
                assert launches == base - (1 if fusable else 0), (k, launches)
            else:
                base = launches
                if m == 16:
                    assert cfg["grid"] // n_itile + 1 >= 64      # the wide reduction
            rc = g6.g6_read_neighbour_list(cid)
            assert rc == (g6.G6_EOVERFLOW if nov else 0), k
            for q in range(act.size):
                rc_q, ln, ids = g6.g6_get_neighbour_list(cid, q)
                assert list(ids) == sorted(ids), (k, q)
                if nblen[q] <= maxnb:
                    assert abs(ln - nblen[q]) <= 2, (k, q)
                    _list_ok(ids, nbl[q, :nblen[q]], idx, x[act[q]], x, h2[q])
                else:
                    assert ln > maxnb and rc_q == g6.G6_EOVERFLOW and len(ids) == maxnb
                    _list_ok(ids, nbl[q, :maxnb], idx, x[act[q]], x, h2[q])
            ea = rel_err_vec(acc, oa)
            assert np.median(ea) <= lim[0] and ea.max() <= lim[1], k
    finally:
        g6.g6x_set_variant(cid, -1, 0)


def test_list_length_setting_is_validated(open_ctx):
    cid = open_ctx(1024, 64)
    assert g6.g6x_max_neighbours(cid) == g6.G6_MAXNB
    for bad in (0, -1, g6.G6X_MAXNB_LIMIT + 1):
        with pytest.raises(g6.G6Error):
            g6.g6x_set_max_neighbours(cid, bad)
    assert g6.g6x_max_neighbours(cid) == g6.G6_MAXNB


def test_lists_with_all_radii_zero_are_empty(open_ctx):
    n = 1000
    m, x, v = ics.plummer(n, 8)
    cid = open_ctx(n, n)
    load_j(cid, x, v, m)
    sweep(cid, n, x[:50], v[:50], np.arange(50), 1e-4, 0.0, h2=np.zeros(50))
    assert g6.g6_read_neighbour_list(cid) == 0
    for q in range(50):
        rc, ln, ids = g6.g6_get_neighbour_list(cid, q)
        assert rc == 0 and ln == 0 and ids.size == 0


def _kepler_relative(t, a=1.0, e=0.5, mtot=1.0):
    nmean = math.sqrt(mtot / a ** 3)
    M = nmean * t
    E = M
    for _ in range(100):
        E -= (E - e * math.sin(E) - M) / (1.0 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_hermite_driver_kepler_orbit(open_ctx, prec):
    rp, vpk = 0.5, math.sqrt(3.0)
    m = np.array([0.5, 0.5])
    x = np.array([[-rp / 2, 0, 0], [rp / 2, 0, 0]])
    v = np.array([[0, -vpk / 2, 0], [0, vpk / 2, 0]])
    cid = open_ctx(256, 256)
    g6.g6x_set_precision(cid, prec)
    sim = g6.G6HSim(cid, m, x, v, 0.0, 0.005)
    sim.run(2.0)
    st = sim.state()
    assert np.all(st["t"] == 2.0)
    err = np.linalg.norm((st["x"][1] - st["x"][0]) - _kepler_relative(2.0))
    assert err < 2e-4
    ek, ep = sim.energy()
    assert abs((ek + ep) / -0.125 - 1) < 1e-6
    sim.close()


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_hermite_driver_plummer_1024_energy_drift(open_ctx, orc, prec):
    n, eps2, eta, t_end = 1024, 1e-4, 0.01, 0.25
    m, x, v = ics.plummer(n, 1)
    E0 = orc.energy(m, x, v, eps2)
    ref = orc.hermite_run(m, x, v, eps2, eta, t_end)
    assert ref["err"] == 0
    dE_orc = abs(orc.energy(m, ref["x"], ref["v"], eps2) / E0 - 1)
    cid = open_ctx(n, n)
    g6.g6x_set_precision(cid, prec)
    sim = g6.G6HSim(cid, m, x, v, eps2, eta)
    sim.run(t_end)
    st = sim.state()
    assert np.all(st["t"] == t_end)
    dE_gpu = abs(orc.energy(m, st["x"], st["v"], eps2) / E0 - 1)
    ek, ep = sim.energy()                        # the library's own energy sweep
    assert abs((ek + ep) / E0 - 1 - (orc.energy(m, st["x"], st["v"], eps2) / E0 - 1)) < 1e-7
    stats = sim.stats()
    assert stats["nblocks"] > 10 and stats["hist"].sum() == stats["nblocks"]
    assert dE_gpu <= 2 * max(dE_orc, 1e-12), (dE_gpu, dE_orc)
    sim.close()


def test_autotuner_table_is_used_and_results_stay_correct(open_ctx, orc, tmp_path):
    n, eps2 = 8192, 1e-4
    m, x, v = ics.plummer(n, 31)
    idx = np.arange(n)
    cid = open_ctx(n, n)
    load_j(cid, x, v, m)
    path = tmp_path / "tune.txt"
    try:
        tuned = g6.g6x_autotune(cid, n, 512, path)
        assert tuned == 6                                 # m = 16 .. 512
        assert g6.g6x_load_tuning(path) == tuned
        for m_act in (16, 100, 512, 3000):
            act = ics.permutation(n, m_act)[:m_act]
            acc, jerk, pot, nnb = sweep(cid, n, x[act], v[act], act, eps2, 0.0)
            oa, oj, op, onn, onr = orc.force(x[act], v[act], act, x, v, m, idx, eps2)
            ea = rel_err_vec(acc, oa)
            assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5
            check_nn(onn, onr, nnb, x[act], x, idx)
    finally:
        g6.g6x_clear_tuning()


def _oracle_drift(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_drift.txt")
    for line in open(path):
        if line.startswith(name + " "):
            f = line.split()
            return float(f[6]), int(f[7]), int(f[8])
    raise KeyError(name)


@pytest.mark.parametrize("name,t_end", [("plummer_n32768_t0.25", 0.25), ("plummer_n32768_t1", 1.0)])
def test_hermite_driver_plummer_32768_drift_vs_stored_oracle(name, t_end):
    # Plummer N = 32768, eps2 = 1e-5, eta = 0.01: the DS path's energy drift is
    # within 2x the FP64 oracle's drift, written by tests/golden/make_oracle_drift.py
    from paper_0902_4463_gb300 import hermite_run
    d_orc, nb_orc, na_orc = _oracle_drift(name)
    r = hermite_run.run(32768, 2, 1e-5, 0.01, t_end, "ds", cid=4)
    assert r["synchronised"]
    assert abs(r["dE_over_E"]) <= 2 * max(abs(d_orc), 1e-12), (r["dE_over_E"], d_orc)
    # the block structure follows the oracle's closely
    assert abs(r["nactive"] / na_orc - 1) < 0.02


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_hermite_checkpoint_resume_reproduces_the_run(orc, tmp_path, prec):
    # Plummer N = 1024 to t = 0.125, checkpoint, continue to t = 0.25; a
    # driver restored from the checkpoint on another cluster id reaches the
    # same state bit for bit (same library settings, same block order).
    from paper_0902_4463_gb300 import build
    build.build()
    n, eps2, eta = 1024, 1e-4, 0.01
    m, x, v = ics.plummer(n, 1)
    ck = str(tmp_path / "run.ckpt")
    g6.g6x_open_ex(5, n, n)
    try:
        g6.g6x_set_precision(5, prec)
        a = g6.G6HSim(5, m, x, v, eps2, eta)
        a.run(0.125)
        a.checkpoint(ck)
        a.run(0.25)
        sa, ta = a.state(), a.stats()
        a.close()
    finally:
        g6.g6_close(5)
    g6.g6x_open_ex(6, n, n)
    try:
        g6.g6x_set_precision(6, prec)
        b = g6.G6HSim.restore(6, ck)
        assert b.n == n
        b.run(0.25)
        sb, tb = b.state(), b.stats()
        b.close()
    finally:
        g6.g6_close(6)
    for k in ("x", "v", "acc", "jerk", "t", "dt"):
        assert np.array_equal(sa[k], sb[k]), k
    assert ta["nblocks"] == tb["nblocks"] and ta["nactive"] == tb["nactive"]
    assert np.array_equal(ta["hist"], tb["hist"])
    assert np.all(sb["t"] == 0.25)


def test_config5_full_size_binary_members_and_lists(open_ctx, orc):
    # Plummer N = 131072 with 10 % of the stars in binaries, eps2 = 1e-8,
    # h2 = 1e-4 (radius 0.01): DS forces on binary members, where the DS
    # separations matter, and their neighbour lists against the oracle.
    n, eps2, h2 = 131072, 1e-8, 1e-4
    m, x, v, pairs = ics.plummer_with_binaries(n, 5)
    idx = np.arange(n)
    cid = open_ctx(n, 4096)
    load_j(cid, x, v, m)
    rng = np.random.default_rng(5)
    members = pairs[rng.choice(len(pairs), 192, replace=False)].reshape(-1)
    act = np.concatenate([members, ics.permutation(n, 55)[:128]])
    hv = np.full(act.size, h2)
    acc, jerk, pot, nnb = sweep(cid, n, x[act], v[act], act, eps2, 0.0, h2=hv)
    rc = g6.g6_read_neighbour_list(cid)
    oa, oj, op, onn, onr = orc.force(x[act], v[act], act, x, v, m, idx, eps2)
    ea, ep = rel_err_vec(acc, oa), np.abs(pot - op) / np.abs(op)
    assert np.median(ea[:members.size]) <= 1e-6 and ea.max() <= 1e-5, (np.median(ea), ea.max())
    assert np.median(ep) <= 1e-6 and ep.max() <= 1e-5
    assert np.array_equal(nnb, onn)
    nblen, nbl, nov = orc.neighbours(x[act], act, x, idx, hv, maxnb=g6.G6_MAXNB)
    assert rc == (g6.G6_EOVERFLOW if nov else 0)
    for q in range(act.size):
        rc_q, ln, ids = g6.g6_get_neighbour_list(cid, q, g6.G6_MAXNB)
        assert abs(ln - nblen[q]) <= 2
        _list_ok(ids, nbl[q, :min(nblen[q], g6.G6_MAXNB)], idx, x[act[q]], x, h2)
    # most binary members list their companion (softened pairs can be wider)
    comp = pairs[np.isin(pairs[:, 0], members)]
    assert np.mean([int(b) in set(g6.g6_get_neighbour_list(cid, int(np.where(act == a)[0][0]),
                                                          g6.G6_MAXNB)[2])
                    for a, b in comp]) > 0.5


def test_hermite_driver_reads_neighbour_lists(open_ctx):
    n = 2048
    m, x, v, pairs = ics.plummer_with_binaries(n, 9)
    cid = open_ctx(n, n)
    sim = g6.G6HSim(cid, m, x, v, 1e-8, 0.01)
    sim.set_neighbour_radius(1e-4)
    sim.run(0.0625)
    st = sim.stats()
    nb = sim.neighbour_stats()
    assert nb["lists"] == st["nactive"] and nb["entries"] > 0 and nb["overflowed"] == 0
    with pytest.raises(g6.G6Error):
        sim.set_neighbour_radius(-1.0)
    sim.close()


def test_config2_force_errors_at_natural_block_steps(orc):
    # Plummer N = 32768, eps2 = 1e-5, eta = 0.01: the DS driver runs to
    # t = 1/4; at 20 points of the run its j-state (every particle at its own
    # last block time, with its a and jerk) is taken as it is, and the next
    # natural block (uneven size, 1 .. N) is evaluated both by the library
    # (j predicted on the GPU) and by the oracle (j predicted in FP64), with
    # the i-particles predicted on the host as the driver does.
    from paper_0902_4463_gb300 import build
    build.build()
    n, eps2, eta, t_end = 32768, 1e-5, 0.01, 0.25
    m, x, v = ics.plummer(n, 2)
    idx = np.arange(n)
    g6.g6x_open_ex(7, n, n)
    g6.g6x_open_ex(8, n, n)
    rows = []
    try:
        sim = g6.G6HSim(7, m, x, v, eps2, eta)
        for snap in range(20):
            if sim.run_blocks(t_end, 229 if snap else 1) == 0:
                break
            st = sim.state()
            tn = st["t"] + st["dt"]
            tb = tn.min()
            act = np.where(tn == tb)[0]
            h = (tb - st["t"][act])[:, None]
            a0, j0 = st["acc"][act], st["jerk"][act]
            xi = st["x"][act] + h * (st["v"][act] + h * (a0 / 2.0 + h * j0 / 6.0))
            vi = st["v"][act] + h * (a0 + h * j0 / 2.0)
            load_j(8, st["x"], st["v"], m, st["acc"], st["jerk"], st["t"])
            acc, jerk, pot, nnb = sweep(8, n, xi, vi, act, eps2, tb)
            xp, vp = orc.predict(st["x"], st["v"], st["acc"], st["jerk"], st["t"], tb)
            oa, oj, op, onn, onr = orc.force(xi, vi, act, xp, vp, m, idx, eps2)
            ea, ej = rel_err_vec(acc, oa), rel_err_vec(jerk, oj)
            ep = np.abs(pot - op) / np.abs(op)
            rows.append((float(tb), act.size, np.median(ea), ea.max(), np.median(ej), ej.max(),
                         np.median(ep), float(np.mean(nnb == onn))))
            assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5, rows[-1]
            assert np.median(ej) <= 1e-6 and ej.max() <= 1e-5, rows[-1]
            assert np.median(ep) <= 1e-6 and ep.max() <= 1e-5, rows[-1]
            check_nn(onn, onr, nnb, xi, xp, idx)
        sim.close()
    finally:
        g6.g6_close(7)
        g6.g6_close(8)
    assert len(rows) == 20 and len({r[1] for r in rows}) > 3     # uneven block sizes
    print("\nconfig2 block errors (t, m, acc med, acc max, jerk med, jerk max, pot med, nn):")
    for r in rows:
        print("%.6f %6d %.2e %.2e %.2e %.2e %.2e %.4f" % r)


def test_hermite_driver_noise_allowance_takes_fewer_blocks(open_ctx, orc):
    # Plummer N = 4096, eps = 4/N, eta = 1e-3 to t = 1/16: the DS driver with
    # the noise-aware step choice (relative force error 1e-6) takes fewer
    # blocks than with the plain criterion, and its energy error stays within
    # 3x the larger of the plain DS and the FP64 runs' (plus 1e-10 absolute).
    n, t_end, eta = 4096, 0.0625, 1e-3
    eps2 = (4.0 / n) ** 2
    m, x, v = ics.plummer(n, 1)
    E0 = orc.energy(m, x, v, eps2)
    cid = open_ctx(n, n)
    out = {}
    for name, prec, noise in (("plain", g6.G6X_PREC_DS, 0.0), ("aware", g6.G6X_PREC_DS, 1e-6),
                              ("fp64", g6.G6X_PREC_FP64, 0.0)):
        g6.g6x_set_precision(cid, prec)
        sim = g6.G6HSim(cid, m, x, v, eps2, eta)
        try:
            for bad in (-1e-7, 1.0, float("nan")):
                with pytest.raises(g6.G6Error):
                    sim.set_force_noise(bad)
            sim.set_force_noise(noise)
            sim.run(t_end)
            st = sim.state()
            assert np.all(st["t"] == t_end)
            out[name] = (sim.stats()["nblocks"],
                         abs(orc.energy(m, st["x"], st["v"], eps2) / E0 - 1))
        finally:
            sim.close()
    assert out["aware"][0] < out["plain"][0], out
    assert out["aware"][1] <= 3 * max(out["plain"][1], out["fp64"][1]) + 1e-10, out


@pytest.mark.parametrize("variant", [-1, 17])
def test_config3_block_sizes_sampled_at_full_size(open_ctx, orc, variant):
    # N = 2^20 (j predicted from t_j = 0 to 2^-10), active sets = the first m
    # entries of the seeded permutation for m = 16 ... 65536, in the launch
    # configuration the built-in heuristic picks (variant -1) and, for the
    # small sizes, in the 16 x 16 x 1 shape that predicts its own j-tiles
    # (variant 17): up to 128 sampled i per size against the oracle.
    n, eps2, t_blk = 1 << 20, 1e-6, 2.0 ** -10
    st = ics.taylor_state(n, 3, t_blk, dt_levels=None)
    cid = open_ctx(n, 65536)
    load_j(cid, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    idx = np.arange(n)
    perm = ics.permutation(n, 7)
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t_blk)
    sizes = (16, 64) if variant == 17 else (16, 128, 1024, 8192, 65536)
    g6.g6x_set_variant(cid, variant)
    try:
        for m in sizes:
            act = perm[:m]
            acc, jerk, pot, nnb = sweep(cid, n, st["x0"][act], st["v0"][act], act, eps2, t_blk)
            if variant >= 0:
                assert g6.g6x_last_config(cid)["variant"] == variant
            s = np.linspace(0, m - 1, min(m, 128)).astype(int)
            oa, oj, op, onn, onr = orc.force(st["x0"][act[s]], st["v0"][act[s]], act[s], xp, vp,
                                             st["m"], idx, eps2)
            ea, ej = rel_err_vec(acc[s], oa), rel_err_vec(jerk[s], oj)
            ep = np.abs(pot[s] - op) / np.abs(op)
            assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5, (m, np.median(ea), ea.max())
            assert np.median(ej) <= 1e-6 and ej.max() <= 1e-5, (m, np.median(ej), ej.max())
            assert np.median(ep) <= 1e-6 and ep.max() <= 1e-5, (m, np.median(ep), ep.max())
            check_nn(onn, onr, nnb[s], st["x0"][act[s]], xp, idx)
    finally:
        g6.g6x_set_variant(cid, -1)


def test_launch_plan_matches_the_launch(open_ctx):
    # g6x_plan_launch names the variant and grid that a calculation of the
    # same size then uses (built-in choice, no tuning table)
    import torch
    g6.g6x_clear_tuning()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 32768
    m, x, v = ics.plummer(n, 2)
    cid = open_ctx(n, n)
    load_j(cid, x, v, m)
    for ni in (1, 16, 256, 1024, 4096, n):
        sel = np.arange(ni)
        sweep(cid, n, x[sel], v[sel], sel, 1e-5, 0.0)
        got = g6.g6x_last_config(cid)
        plan = g6.g6x_plan_launch(g6.G6X_PREC_DS, n, ni, False, sms)
        assert (got["variant"], got["grid"], got["jtiles"]) == \
            (plan["variant"], plan["grid"], plan["jtiles"]), (ni, got, plan)
