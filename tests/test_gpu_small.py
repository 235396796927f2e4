"""GPU parity of the warp-specialised small-block force kernel (K2s) against
the FP64 oracle.

The kernel holds the whole active block (up to 256 i-particles) as one
i-tile, predicts its j-tiles itself (Eq. 1, Eq. 2 of Sect. 2.2), sums the
forces with the Eq. 3 separations (Sect. 2.3) and reduces the partial sums of
its CTAs inside the launch.  Checked here, for every compiled shape: ragged
block and j-set sizes with the i-particles among the j-particles (self test
by index), j-particles predicted from varied t_j, j-updates staged between
calls (the kernel stores them itself), forced small and odd grids (one
reduction level, ragged groups), two calls in a row (the in-kernel counters
must come back to zero), and the timeout path.  Tolerances: median relative
error <= 1e-6 and max <= 1e-5 for acceleration, jerk and potential."""
import numpy as np
import pytest

from paper_0902_4463_gb300 import g6gb as g6
from paper_0902_4463_gb300 import ics
from tests.gpu_helpers import check_nn, load_j, rel_err_vec, sweep

pytestmark = pytest.mark.gpu

CID = 6


def _ws_variants():
    from paper_0902_4463_gb300 import build
    build.build()
    out = []
    for v in range(g6.g6x_variant_count()):
        info = g6.g6x_variant_info(v)
        if info["ws"]:
            out.append((v, info["ti"] * info["ni_per"]))
    return out


@pytest.fixture()
def ctx():
    from paper_0902_4463_gb300 import build
    build.build()
    g6.g6x_open_ex(CID, 1 << 17, 4096)
    yield CID
    g6.g6x_set_variant(CID, -1, 0)
    g6.g6_close(CID)


def _check(orc, res, st, act, t_blk, eps2, n):
    acc, jerk, pot, nnb = res
    xi, vi = st["x0"][act], st["v0"][act]
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t_blk)
    idx = np.arange(n)
    oa, oj, op, onn, onr = orc.force(xi, vi, act, xp, vp, st["m"], idx, eps2)
    ea, ej = rel_err_vec(acc, oa), rel_err_vec(jerk, oj)
    ep = np.abs(pot - op) / np.abs(op)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5, (np.median(ea), ea.max())
    assert np.median(ej) <= 1e-6 and ej.max() <= 1e-5, (np.median(ej), ej.max())
    assert np.median(ep) <= 1e-6 and ep.max() <= 1e-5, (np.median(ep), ep.max())
    check_nn(onn, onr, nnb, xi, xp, idx)


def test_every_small_block_shape_against_the_oracle(ctx, orc):
    # N = 50001 (196 j-tiles, the last one ragged), j-particles predicted from
    # varied t_j; per shape blocks of 1, a ragged size and the full i-tile
    n, eps2, t_blk = 50001, 1e-5, 0.375
    st = ics.taylor_state(n, 31, t_blk)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    perm = ics.permutation(n, 31)
    shapes = _ws_variants()
    assert len(shapes) >= 5
    for v, itile in shapes:
        g6.g6x_set_variant(ctx, v, 0)
        for m in sorted({1, itile // 2 + 3, itile} & set(range(1, itile + 1))):
            act = perm[:m]
            res = sweep(ctx, n, st["x0"][act], st["v0"][act], act, eps2, t_blk)
            assert g6.g6x_last_config(ctx)["variant"] == v
            _check(orc, res, st, act, t_blk, eps2, n)


@pytest.mark.parametrize("grid", [1, 2, 7, 17, 196])
def test_small_block_grids_and_repeated_calls(ctx, orc, grid):
    # one CTA (one reduction level), a few CTAs in ragged groups, one CTA per
    # j-tile; each twice in a row, with staged j-updates in between that the
    # kernel stores itself before reading its tiles
    n, eps2, t_blk = 50001, 1e-5, 0.25
    st = ics.taylor_state(n, 41, t_blk)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    perm = ics.permutation(n, 41)
    v16 = [v for v, it in _ws_variants() if it == 16][0]
    g6.g6x_set_variant(ctx, v16, grid)
    act = perm[:13]
    res = sweep(ctx, n, st["x0"][act], st["v0"][act], act, eps2, t_blk)
    cfg = g6.g6x_last_config(ctx)
    assert cfg["variant"] == v16 and cfg["grid"] == grid
    _check(orc, res, st, act, t_blk, eps2, n)
    q = ics.permutation(n, 43)[:500]
    st["x0"][q] += 2e-3
    st["tj"][q] = t_blk
    g6.g6x_set_j_particles(ctx, q.astype(np.int32), q.astype(np.int32), st["tj"][q],
                           st["m"][q], st["j0"][q] / 6.0, st["a0"][q] / 2.0, st["v0"][q],
                           st["x0"][q])
    t2 = t_blk + 2.0 ** -7
    res2 = sweep(ctx, n, st["x0"][act], st["v0"][act], act, eps2, t2)
    _check(orc, res2, st, act, t2, eps2, n)


def test_small_block_matches_the_other_kernels(ctx, orc):
    # the same block through the small-block kernel and through the shapes
    # with a separate predictor: the same forces within rounding, the same
    # nearest neighbours
    n, eps2, t_blk = 20000, 1e-5, 0.125
    st = ics.taylor_state(n, 51, t_blk)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    act = ics.permutation(n, 51)[:200]
    xi, vi = st["x0"][act], st["v0"][act]
    v256 = [v for v, it in _ws_variants() if it == 256][0]
    g6.g6x_set_variant(ctx, v256, 0)
    a = sweep(ctx, n, xi, vi, act, eps2, t_blk)
    g6.g6x_set_variant(ctx, 15, 0)                # 32 x 8 x 2 reading predicted tiles
    b = sweep(ctx, n, xi, vi, act, eps2, t_blk)
    assert np.max(rel_err_vec(a[0], b[0])) <= 2e-6
    assert np.max(np.abs(a[2] - b[2]) / np.abs(b[2])) <= 2e-6
    assert np.mean(a[3] == b[3]) >= 0.99
    _check(orc, a, st, act, t_blk, eps2, n)


def test_small_block_timeout_path_leaves_the_context_usable(ctx, orc):
    # with a 1 us limit on every wait the kernel may give up (G6_ETIMEDOUT,
    # no fault, nothing left in flight); the next call with the normal limit
    # is correct, so the reduction counters were cleared
    n, eps2 = 30000, 1e-4
    m, x, v = ics.plummer(n, 61)
    load_j(ctx, x, v, m)
    act = ics.permutation(n, 61)[:64]
    v64 = [vv for vv, it in _ws_variants() if it == 64][0]
    g6.g6x_set_variant(ctx, v64, 0)
    outcome = 0
    g6.g6x_set_wait_limit(1e-6)
    try:
        for _ in range(5):
            try:
                sweep(ctx, n, x[act], v[act], act, eps2, 0.0)
            except g6.G6Error as e:
                outcome = e.code
                break
    finally:
        g6.g6x_set_wait_limit(2.0)
    assert outcome in (0, g6.G6_ETIMEDOUT)
    acc, jerk, pot, nnb = sweep(ctx, n, x[act], v[act], act, eps2, 0.0)
    idx = np.arange(n)
    oa, oj, op, onn, onr = orc.force(x[act], v[act], act, x, v, m, idx, eps2)
    ea = rel_err_vec(acc, oa)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5
    check_nn(onn, onr, nnb, x[act], x, idx)
