"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances (stated for the FP32 + double-single path at N = 32768: median
relative force error <= 1e-6, max <= 1e-5) are applied to acceleration, jerk
and potential.  Nearest neighbours must be valid (FP64 distance within 1e-5
relative of the oracle minimum; floating point decides near-ties).  The
all-FP64 path must agree to 1e-11."""
import numpy as np
import pytest

from paper_0902_4463_gb300 import g6gb as g6
from paper_0902_4463_gb300 import ics
from tests.gpu_helpers import check_nn, load_j, rel_err_vec, sweep

pytestmark = pytest.mark.gpu

CID = 2


@pytest.fixture()
def ctx():
    from paper_0902_4463_gb300 import build
    build.build()
    g6.g6x_open_ex(CID, 1 << 20 | 4096, 1 << 20)
    yield CID
    g6.g6_close(CID)


def _tol(prec):
    return (1e-12, 1e-10) if prec == g6.G6X_PREC_FP64 else (1e-6, 1e-5)


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_full_sweep_plummer_1024(ctx, orc, prec):
    # Plummer N = 1024, eps2 = 1e-4, every particle active at t = 0.
    n, eps2 = 1024, 1e-4
    m, x, v = ics.plummer(n, 1)
    idx = np.arange(n)
    g6.g6x_set_precision(ctx, prec)
    load_j(ctx, x, v, m)
    acc, jerk, pot, nnb = sweep(ctx, n, x, v, idx, eps2, 0.0)
    oa, oj, op, onn, onr = orc.force(x, v, idx, x, v, m, idx, eps2)
    med, mx = _tol(prec)
    ea, ej = rel_err_vec(acc, oa), rel_err_vec(jerk, oj)
    ep = np.abs(pot - op) / np.abs(op)
    assert np.median(ea) <= med and ea.max() <= mx
    assert np.median(ej) <= med and ej.max() <= mx, (np.median(ej), ej.max())
    assert np.median(ep) <= med and ep.max() <= mx
    assert check_nn(onn, onr, nnb, x, x, idx) > 0.99


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64, g6.G6X_PREC_DS_X64])
def test_predictor_matches_eq1_eq2(ctx, orc, prec):
    # j-particles last updated at varied block times; predicted to t_blk.
    n, t_blk = 3001, 0.375
    st = ics.taylor_state(n, 7, t_blk)
    g6.g6x_set_precision(ctx, prec)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    g6.g6_set_ti(ctx, t_blk)
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t_blk)
    h = (t_blk - st["tj"])[:, None]
    inc = np.abs(st["v0"] * h) + np.abs(st["a0"] * h * h / 2) + np.abs(st["j0"] * h ** 3 / 6)
    vinc = np.abs(st["v0"]) + np.abs(st["a0"] * h) + np.abs(st["j0"] * h * h / 2)
    if prec != g6.G6X_PREC_FP64:
        hi, lo, vel = g6.g6x_get_predicted(ctx, n)
        x_gpu = hi[:, :3].astype(np.float64) + lo[:, :3].astype(np.float64)
        assert np.all(np.abs(x_gpu - xp) <= 8 * 2.0 ** -24 * inc + 2.0 ** -46 * np.abs(xp))
        assert np.all(np.abs(vel[:, :3] - vp) <= 8 * 2.0 ** -24 * vinc)
        # hi is the nearest float of the position (DS split of Sect. 2.2)
        assert np.all(np.abs(hi[:, :3] - xp) <= 2.0 ** -23 * np.abs(xp) + 8 * 2.0 ** -24 * inc)
        assert np.array_equal(hi[:, 3], st["m"].astype(np.float32))
        assert np.array_equal(vel[:, 3].view(np.int32), np.arange(n, dtype=np.int32))
    else:
        x64, v64 = g6.g6x_get_predicted(ctx, n, fp64=True)
        assert np.allclose(x64[:, :3], xp, rtol=0, atol=1e-15 * (1 + np.abs(xp)).max())
        assert np.allclose(v64[:, :3], vp, rtol=0, atol=1e-14 * (1 + np.abs(vp)).max())
        assert np.array_equal(x64[:, 3], st["m"])


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64, g6.G6X_PREC_DS_X64])
def test_subset_of_predicted_particles_ragged(ctx, orc, prec):
    # n and m not multiples of any tile; i-particles are a seeded subset that
    # sit at their generator positions while the j-particles are predicted.
    n, m_act, t_blk, eps2 = 3001, 777, 0.25, 1e-5
    st = ics.taylor_state(n, 11, t_blk)
    g6.g6x_set_precision(ctx, prec)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    act = ics.permutation(n, 11)[:m_act]
    xi, vi = st["x0"][act], st["v0"][act]
    acc, jerk, pot, nnb = sweep(ctx, n, xi, vi, act, eps2, t_blk)
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t_blk)
    idx = np.arange(n)
    oa, oj, op, onn, onr = orc.force(xi, vi, act, xp, vp, st["m"], idx, eps2)
    med, mx = _tol(prec)
    ea, ej = rel_err_vec(acc, oa), rel_err_vec(jerk, oj)
    ep = np.abs(pot - op) / np.abs(op)
    assert np.median(ea) <= med and ea.max() <= mx
    assert np.median(ej) <= med and ej.max() <= mx, (np.median(ej), ej.max())
    assert np.median(ep) <= med and ep.max() <= mx
    check_nn(onn, onr, nnb, xi, xp, idx)


@pytest.mark.parametrize("n,m_act", [(1, 1), (7, 7), (33, 5), (255, 255), (257, 256),
                                     (513, 33), (2049, 17), (300, 1)])
def test_odd_sizes(ctx, orc, n, m_act):
    eps2 = 1e-3
    m, x, v = ics.plummer(n, 100 + n)
    idx = np.arange(n)
    load_j(ctx, x, v, m)
    act = ics.permutation(n, n)[:m_act]
    acc, jerk, pot, nnb = sweep(ctx, n, x[act], v[act], act, eps2, 0.0)
    oa, oj, op, onn, onr = orc.force(x[act], v[act], act, x, v, m, idx, eps2)
    if n == 1:
        assert np.all(acc == 0) and np.all(jerk == 0) and np.all(pot == 0)
        assert nnb[0] == -1
        return
    ea = rel_err_vec(acc, oa)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5
    assert np.allclose(pot, op, rtol=1e-6)
    check_nn(onn, onr, nnb, x[act], x, idx)


def test_i_not_in_j_memory_feels_every_particle(ctx, orc):
    # An i-particle whose index matches no j-slot is not self-excluded.
    n, eps2 = 500, 1e-2
    m, x, v = ics.plummer(n, 5)
    load_j(ctx, x, v, m)
    xi = x[:3] + 0.01
    acc, jerk, pot, nnb = sweep(ctx, n, xi, v[:3], [10 ** 6, 10 ** 6 + 1, 10 ** 6 + 2],
                                eps2, 0.0)
    oa, oj, op, onn, onr = orc.force(xi, v[:3], [10 ** 6, 10 ** 6 + 1, 10 ** 6 + 2], x, v, m,
                                     np.arange(n), eps2)
    assert np.all(rel_err_vec(acc, oa) < 1e-5)
    assert np.array_equal(nnb, onn)


def test_two_body_without_softening(ctx, orc):
    x = np.array([[-0.25, 0.0, 0.0], [0.25, 0.0, 0.0]])
    v = np.array([[0.0, -0.8, 0.0], [0.0, 0.8, 0.0]])
    m = np.array([0.5, 0.5])
    load_j(ctx, x, v, m)
    acc, jerk, pot, nnb = sweep(ctx, 2, x, v, [0, 1], 0.0, 0.0)
    oa, oj, op, onn, _ = orc.force(x, v, [0, 1], x, v, m, [0, 1], 0.0)
    assert np.allclose(acc, oa, rtol=1e-6, atol=1e-7)
    assert np.allclose(jerk, oj, rtol=1e-6, atol=1e-7)
    assert np.allclose(pot, op, rtol=1e-6)
    assert list(nnb) == [1, 0]


def test_close_binaries_need_double_single(ctx, orc):
    # Binaries with separations 1e-4..1e-2 inside a Plummer sphere
    # (Sect. 2.3: DS separations keep the digits FP32 positions would lose).
    n = 4096
    m, x, v, pairs = ics.plummer_with_binaries(n, 5)
    idx = np.arange(n)
    eps2 = 1e-8
    load_j(ctx, x, v, m)
    act = pairs[:64].reshape(-1)
    acc, jerk, pot, nnb = sweep(ctx, n, x[act], v[act], act, eps2, 0.0)
    oa, oj, op, onn, onr = orc.force(x[act], v[act], act, x, v, m, idx, eps2)
    ea = rel_err_vec(acc, oa)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5
    # nearest neighbours agree with the oracle; almost all are the companion
    # (a wide pair can have a closer third star)
    assert np.array_equal(nnb, onn)
    assert np.mean(nnb == pairs[:64][:, ::-1].reshape(-1)) > 0.9


def test_device_resident_path_matches_host_path(ctx):
    import torch
    n, eps2, t_blk = 5000, 1e-4, 0.125
    st = ics.taylor_state(n, 3, t_blk)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    act = ics.permutation(n, 3)[:1234]
    xi, vi = st["x0"][act], st["v0"][act]
    acc, jerk, pot, nnb = sweep(ctx, n, xi, vi, act, eps2, t_blk)
    rec = np.zeros(act.size, dtype=g6.IREC)
    rec["x"], rec["v"], rec["index"] = xi, vi, act
    d_rec = torch.from_numpy(rec.view(np.uint8)).cuda()
    d_out = torch.empty(act.size * g6.OUT.itemsize, dtype=torch.uint8, device="cuda")
    g6.g6x_set_stream(ctx, torch.cuda.current_stream().cuda_stream)
    g6.g6x_calc_dev(ctx, t_blk, n, act.size, d_rec.data_ptr(), eps2, 0, d_out.data_ptr())
    g6.g6x_sync(ctx)
    out = d_out.cpu().numpy().view(g6.OUT)
    g6.g6x_set_stream(ctx, 0)
    assert np.array_equal(out["acc"], acc) and np.array_equal(out["jerk"], jerk)
    assert np.array_equal(out["pot"], pot) and np.array_equal(out["nnb"], nnb)


def test_j_updates_between_calls(ctx, orc):
    # set_j_particle after a calculation replaces slots; repeated writes to
    # one slot keep the last; the prediction is redone.
    n, eps2 = 1000, 1e-3
    m, x, v = ics.plummer(n, 9)
    idx = np.arange(n)
    load_j(ctx, x, v, m)
    sweep(ctx, n, x[:10], v[:10], idx[:10], eps2, 0.0)
    x2 = x.copy()
    x2[:50] += 0.05
    z = np.zeros(3)
    for k in range(50):
        g6.g6_set_j_particle(ctx, k, k, 0.0, 0.0, m[k], z, z, z, v[k], x[k] - 1.0)
        g6.g6_set_j_particle(ctx, k, k, 0.0, 0.0, m[k], z, z, z, v[k], x2[k])
    acc, jerk, pot, nnb = sweep(ctx, n, x2[:100], v[:100], idx[:100], eps2, 0.0)
    oa, oj, op, onn, onr = orc.force(x2[:100], v[:100], idx[:100], x2, v, m, idx, eps2)
    assert np.median(rel_err_vec(acc, oa)) < 1e-6
    assert np.allclose(pot, op, rtol=1e-6)


def test_argument_errors_are_reported(ctx):
    lib = g6.lib()
    z = np.zeros(3)
    zp = z.ctypes.data_as(g6.C.c_void_p)
    assert lib.g6_set_j_particle(ctx, -1, 0, 0.0, 0.0, 1.0, zp, zp, zp, zp, zp) == g6.G6_EINVAL
    assert lib.g6_set_j_particle(ctx, 0, -5, 0.0, 0.0, 1.0, zp, zp, zp, zp, zp) == g6.G6_EINVAL
    assert lib.g6_open(ctx) == g6.G6_EBUSY
    # lasthalf without firsthalf
    assert lib.g6calc_lasthalf(ctx, 1, 1, None, None, None, 0.0, None, None, None,
                               None) == g6.G6_EBUSY
    # negative softening is latched by firsthalf and returned by lasthalf
    g6.g6calc_firsthalf(ctx, 10, 1, [0], np.zeros((1, 3)), np.zeros((1, 3)), -1.0)
    with pytest.raises(g6.G6Error):
        g6.g6calc_lasthalf(ctx, 10, 1)
    # the context stays usable
    m, x, v = ics.plummer(64, 2)
    load_j(ctx, x, v, m)
    acc, *_ = sweep(ctx, 64, x, v, np.arange(64), 1e-2, 0.0)
    assert np.all(np.isfinite(acc))


def test_bounded_wait_that_nothing_completes_is_reported(ctx, orc):
    # Failure detection without a fault: one bounded wait on an mbarrier that
    # nothing completes runs out after the set limit and is reported as the
    # force kernels report it; the context stays usable.
    import time
    g6.g6x_set_wait_limit(0.05)
    try:
        t0 = time.perf_counter()
        rc = g6.g6x_probe_wait_timeout(ctx)
        dt = time.perf_counter() - t0
    finally:
        g6.g6x_set_wait_limit(2.0)
    assert rc == g6.G6_ETIMEDOUT
    assert 0.04 <= dt < 1.5, dt
    n, eps2 = 1024, 1e-4
    m, x, v = ics.plummer(n, 1)
    idx = np.arange(n)
    load_j(ctx, x, v, m)
    acc, jerk, pot, nnb = sweep(ctx, n, x, v, idx, eps2, 0.0)
    oa, *_ = orc.force(x, v, idx, x, v, m, idx, eps2)
    assert np.median(rel_err_vec(acc, oa)) <= 1e-6


def test_force_kernel_timeout_path_leaves_the_context_usable(ctx, orc):
    # With a 1 us limit the force kernel's waits for staged j-tiles may run
    # out (the hardware wait can also complete first): the call then reports
    # G6_ETIMEDOUT after draining its copies; either way the next call with
    # the normal limit gives correct forces.
    n, eps2, mi = 65536, 1e-5, 8192
    m, x, v = ics.plummer(n, 2)
    idx = np.arange(n)
    load_j(ctx, x, v, m)
    act = np.sort(ics.permutation(n, 3)[:mi])
    outcome = 0
    g6.g6x_set_wait_limit(1e-6)
    try:
        for _ in range(3):
            try:
                sweep(ctx, n, x[act], v[act], act, eps2, 0.0)
            except g6.G6Error as e:
                outcome = e.code
                break
    finally:
        g6.g6x_set_wait_limit(2.0)
    assert outcome in (0, g6.G6_ETIMEDOUT)
    acc, jerk, pot, nnb = sweep(ctx, n, x[act], v[act], act, eps2, 0.0)
    oa, *_ = orc.force(x[act[:256]], v[act[:256]], act[:256], x, v, m, idx, eps2)
    ea = rel_err_vec(acc[:256], oa)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5


@pytest.mark.parametrize("fv,twin,m", [(17, 4, 16), (18, 14, 100), (19, 15, 256),
                                       (20, 16, 1000)])
def test_fused_prediction_is_identical_to_separate(ctx, orc, fv, twin, m):
    # A force kernel that predicts its j-tiles itself (Eq. 1, Eq. 2 with the
    # predictor's own arithmetic) gives bit-identical results to the separate
    # predictor + force kernel of the same shape, also after j-updates
    # between calls; both agree with the oracle.
    n, eps2, t_blk = 50001, 1e-5, 0.375
    st = ics.taylor_state(n, 21, t_blk)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    act = np.sort(ics.permutation(n, 21)[:m])
    xi, vi = st["x0"][act], st["v0"][act]

    def run(v, t):
        g6.g6x_set_variant(ctx, v, 0)
        r = sweep(ctx, n, xi, vi, act, eps2, t)
        assert g6.g6x_last_config(ctx)["variant"] == v
        return r

    try:
        a = run(twin, t_blk)
        b = run(fv, t_blk)
        for u, w in zip(a, b):
            assert np.array_equal(u, w)
        # j-updates: new Taylor data for some particles, then the fused
        # shape first (it stores the records and predicts itself)
        q = ics.permutation(n, 5)[:777]
        st["x0"][q] += 1e-3
        st["tj"][q] = t_blk
        g6.g6x_set_j_particles(ctx, q.astype(np.int32), q.astype(np.int32), st["tj"][q],
                               st["m"][q], st["j0"][q] / 6.0, st["a0"][q] / 2.0, st["v0"][q],
                               st["x0"][q])
        t2 = t_blk + 2.0 ** -6
        b2 = run(fv, t2)
        a2 = run(twin, t2)
        for u, w in zip(a2, b2):
            assert np.array_equal(u, w)
    finally:
        g6.g6x_set_variant(ctx, -1, 0)
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t2)
    idx = np.arange(n)
    oa, oj, op, onn, onr = orc.force(xi, vi, act, xp, vp, st["m"], idx, eps2)
    ea = rel_err_vec(b2[0], oa)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5
    check_nn(onn, onr, b2[3], xi, xp, idx)


@pytest.mark.parametrize("m", [16, 3001])
def test_full_ds_subtraction_ablation(ctx, orc, m):
    # Separations by the full DS subtraction instead of Eq. 3's form: the
    # same tolerances on close binaries and on a Plummer subset; the DS forms
    # agree with each other far more closely than with FP32 positions.
    n = 4096
    mm, x, v, pairs = ics.plummer_with_binaries(n, 5)
    idx = np.arange(n)
    eps2 = 1e-8
    load_j(ctx, x, v, mm)
    act = np.sort(np.concatenate([pairs[:8].reshape(-1),
                                  ics.permutation(n, 6)[:max(0, min(m, n) - 16)]]))[:m]
    act = np.unique(act)
    res = {}
    for prec in (g6.G6X_PREC_DS, g6.G6X_PREC_DS_DSSUB):
        g6.g6x_set_precision(ctx, prec)
        res[prec] = sweep(ctx, n, x[act], v[act], act, eps2, 0.0)
    cfg = g6.g6x_last_config(ctx)
    assert cfg["variant"] in (21, 22)
    oa, oj, op, onn, onr = orc.force(x[act], v[act], act, x, v, mm, idx, eps2)
    for prec, (acc, jerk, pot, nnb) in res.items():
        ea, ep = rel_err_vec(acc, oa), np.abs(pot - op) / np.abs(op)
        assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5, (prec, np.median(ea), ea.max())
        assert np.median(ep) <= 1e-6 and ep.max() <= 1e-5
        check_nn(onn, onr, nnb, x[act], x, idx)
    g6.g6x_set_precision(ctx, g6.G6X_PREC_DS)


def test_large_bulk_staging_keeps_the_last_values(ctx, orc):
    # A bulk j-update above the threaded size that names every address twice
    # (first with wrong data) stages the last values, as the per-particle
    # calls do; a large update without repeats equals per-particle staging.
    n, eps2, t_blk = 20000, 1e-5, 0.375
    st = ics.taylor_state(n, 31, t_blk)
    addr = np.arange(n, dtype=np.int32)
    both = np.concatenate([addr, addr])
    junk = st["x0"] + 1.0
    g6.g6x_set_j_particles(ctx, both, both, np.concatenate([st["tj"], st["tj"]]),
                           np.concatenate([st["m"], st["m"]]),
                           np.concatenate([st["j0"], st["j0"]]) / 6.0,
                           np.concatenate([st["a0"], st["a0"]]) / 2.0,
                           np.concatenate([st["v0"], st["v0"]]),
                           np.concatenate([junk, st["x0"]]))
    act = np.sort(ics.permutation(n, 32)[:512])
    xi, vi = st["x0"][act], st["v0"][act]
    bulk = sweep(ctx, n, xi, vi, act, eps2, t_blk)
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t_blk)
    oa, *_ = orc.force(xi, vi, act, xp, vp, st["m"], np.arange(n), eps2)
    ea = rel_err_vec(bulk[0], oa)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5
    load_j(ctx, st["x0"] + 0.5, st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    for k in range(n):                         # per-particle staging, same data
        g6.g6_set_j_particle(ctx, k, k, st["tj"][k], 0.0, st["m"][k], np.zeros(3),
                             st["j0"][k] / 6.0, st["a0"][k] / 2.0, st["v0"][k], st["x0"][k])
    single = sweep(ctx, n, xi, vi, act, eps2, t_blk + 2.0 ** -8)
    g6.g6x_set_j_particles(ctx, addr, addr, st["tj"], st["m"], st["j0"] / 6.0,
                           st["a0"] / 2.0, st["v0"], st["x0"])
    again = sweep(ctx, n, xi, vi, act, eps2, t_blk + 2.0 ** -8)
    for u, w in zip(single, again):
        assert np.array_equal(u, w)


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_empty_calls(ctx, orc, prec):
    # ni = 0 is a no-op; nj = 0 leaves every i-particle without partners:
    # zero acceleration, jerk and potential, no nearest neighbour (the slots
    # holding particles beyond nj must not act, not even as a neighbour).
    n = 300
    m, x, v = ics.plummer(n, 3)
    g6.g6x_set_precision(ctx, prec)
    load_j(ctx, x, v, m)
    acc, jerk, pot, nnb = sweep(ctx, n, x[:0], v[:0], np.arange(0), 1e-4, 0.0)
    assert acc.shape == (0, 3) and nnb.shape == (0,)
    acc, jerk, pot, nnb = sweep(ctx, 0, x[:5], v[:5], np.arange(5), 1e-4, 0.0)
    assert np.all(acc == 0) and np.all(jerk == 0) and np.all(pot == 0)
    assert np.all(nnb == -1)
    # and the context still computes normally afterwards
    # one j-particle, which is the i-particle itself: alone again
    acc, jerk, pot, nnb = sweep(ctx, 1, x[:1], v[:1], np.arange(1), 1e-4, 0.0)
    assert np.all(acc == 0) and np.all(pot == 0) and nnb[0] == -1
    acc, *_ = sweep(ctx, n, x, v, np.arange(n), 1e-4, 0.0)
    oa, *_ = orc.force(x, v, np.arange(n), x, v, m, np.arange(n), 1e-4)
    assert np.median(rel_err_vec(acc, oa)) <= _tol(prec)[0]


@pytest.mark.parametrize("prec", [g6.G6X_PREC_DS, g6.G6X_PREC_FP64])
def test_capacity_sized_call_and_massless_particles(orc, prec):
    # nj equal to the context's j capacity and ni equal to its i limit; a
    # tenth of the particles massless (they feel forces, exert none).
    from paper_0902_4463_gb300 import build
    build.build()
    cap, nimax, cid = 8192, 1000, 12
    m, x, v = ics.plummer(cap, 4)
    m = m.copy()
    m[::10] = 0.0
    idx = np.arange(cap)
    g6.g6x_open_ex(cid, cap, nimax)
    try:
        g6.g6x_set_precision(cid, prec)
        load_j(cid, x, v, m)
        act = np.sort(ics.permutation(cap, 8)[:nimax])
        acc, jerk, pot, nnb = sweep(cid, cap, x[act], v[act], act, 1e-5, 0.0)
        with pytest.raises(g6.G6Error):                    # one more i than allowed
            sweep(cid, cap, x[:nimax + 1], v[:nimax + 1], idx[:nimax + 1], 1e-5, 0.0)
        with pytest.raises(g6.G6Error):                    # one more j than capacity
            sweep(cid, cap + 1, x[:5], v[:5], idx[:5], 1e-5, 0.0)
    finally:
        g6.g6_close(cid)
    oa, oj, op, onn, onr = orc.force(x[act], v[act], act, x, v, m, idx, 1e-5)
    med, mx = _tol(prec)
    ea, ep = rel_err_vec(acc, oa), np.abs(pot - op) / np.abs(op)
    assert np.median(ea) <= med and ea.max() <= mx
    assert np.median(ep) <= med and ep.max() <= mx
    check_nn(onn, onr, nnb, x[act], x, idx)


def test_plain_c_client_matches_oracle(orc, tmp_path):
    # The GRAPE calling sequence from a C program (no Python between it and
    # the library): Plummer N = 1024, forces, nearest neighbours and list
    # lengths against the oracle.
    import subprocess
    from tests.test_abi_cpu import _build_c_client
    from paper_0902_4463_gb300 import build
    build.build()
    exe = _build_c_client(tmp_path)
    n, eps2, h2 = 1024, 1e-4, 0.01
    m, x, v = ics.plummer(n, 1)
    lines = ["%d" % n] + ["%.17g %.17g %.17g %.17g %.17g %.17g %.17g" % (m[k], *x[k], *v[k])
                          for k in range(n)]
    (tmp_path / "in.txt").write_text("\n".join(lines) + "\n")
    out = tmp_path / "out.txt"
    r = subprocess.run([exe, str(tmp_path / "in.txt"), str(out), repr(eps2), repr(h2)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    res = np.loadtxt(out)
    acc, jerk, pot = res[:, 0:3], res[:, 3:6], res[:, 6]
    nnb, nblen = res[:, 7].astype(int), res[:, 8].astype(int)
    idx = np.arange(n)
    oa, oj, op, onn, onr = orc.force(x, v, idx, x, v, m, idx, eps2)
    assert np.median(rel_err_vec(acc, oa)) <= 1e-6 and rel_err_vec(acc, oa).max() <= 1e-5
    assert np.median(np.abs(pot - op) / np.abs(op)) <= 1e-6
    check_nn(onn, onr, nnb, x, x, idx)
    olen, _, _ = orc.neighbours(x, idx, x, idx, np.full(n, h2), maxnb=g6.G6_MAXNB)
    assert np.all(np.abs(nblen - olen) <= 1)
