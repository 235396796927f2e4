"""Bit-exact pins of the double-single arithmetic on the GPU (Sect. 2.2,
Sect. 2.3), against a CPU restatement written here in numpy float32.

Predictor (Sect. 2.2).  The j-particle's position is held as a DS pair
(hi = the float nearest x, lo = the float nearest x - hi), its velocity,
a/2 and j/6 as floats.  Every product of Eq. 1 is formed in single
precision: the increment dt (v + dt (a/2 + dt j/6)) by two fused
multiply-adds (one rounding each) and a product, dt itself being the float
nearest t_blk - t_j.  The increment is added to the DS position by the DS +
SP addition (ten single-precision operations: TwoSum of hi and the
increment, lo added to its error, a Fast2Sum renormalisation).  Eq. 2 is
v + dt (2 (a/2) + 3 dt (j/6)) with two fused multiply-adds.  Every step
rounds to nearest.  The selectable FP64-add form adds the FP32 increment to
the FP64 position in double precision and splits the sum into its DS pair.
The GPU's predicted words (g6x_get_predicted) must equal this restatement bit
for bit for every particle.

Separation (Eq. 3).  With i and j held as DS pairs, the separation is
(x_j,hi - x_i,hi) + (x_j,lo - x_i,lo) in single precision.  Where the two
high parts are within a factor of two of each other (nearby particles) their
difference is exact (Sterbenz), so the result differs from the exact FP64
separation by the final rounding, 2^-24 |dx|, plus the DS representation
errors of the two positions and the rounding of the small low-part
difference, together at most 2^-47 (|x_i| + |x_j|).  Elsewhere the high
difference rounds too: 2^-23 |dx| + 2^-46 (|x_i| + |x_j|)."""
import numpy as np
import pytest

from paper_0902_4463_gb300 import g6gb as g6
from paper_0902_4463_gb300 import ics
from tests.ds_restate import ds_split, fma32, restated_prediction, rn32
from tests.gpu_helpers import load_j

pytestmark = pytest.mark.gpu

CID = 7


@pytest.fixture()
def ctx():
    from paper_0902_4463_gb300 import build
    build.build()
    g6.g6x_open_ex(CID, 1 << 15, 256)
    yield CID
    g6.g6_close(CID)


@pytest.mark.parametrize("mode", [g6.G6X_PREC_DS, g6.G6X_PREC_DS_X64])
def test_predicted_words_are_bit_exact(ctx, mode):
    # 12000 particles last updated at t_blk - 2^-k, k = 4 .. 12, and some with
    # t_j = t_blk (no increment) and steps up to 1/2
    n, t_blk = 12000, 0.625
    st = ics.taylor_state(n, 71, t_blk)
    st["tj"][:200] = t_blk
    st["tj"][200:400] = t_blk - 0.5
    g6.g6x_set_precision(ctx, mode)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    g6.g6_set_ti(ctx, t_blk)
    hi, lo, vel = g6.g6x_get_predicted(ctx, n)
    rh, rl, rv = restated_prediction(st, t_blk, x64_add=(mode == g6.G6X_PREC_DS_X64))
    for got, want, what in ((hi[:, :3], rh, "hi"), (lo[:, :3], rl, "lo"), (vel[:, :3], rv, "v")):
        bad = np.nonzero(got.view(np.uint32) != want.view(np.uint32))
        assert bad[0].size == 0, (what, bad[0][:5], got[bad][:5], want[bad][:5])
    assert np.array_equal(hi[:, 3], rn32(st["m"]))


def test_eq3_separation_bound_from_predicted_words(ctx, orc):
    # 32 close pairs (separations 1e-7 .. 1e-3 at |x| up to 8) and 32 wide
    # ones, j-particles predicted with t_j = t_blk (their words are the DS
    # pairs of x0); the single-precision Eq. 3 separation from those words
    # and from the i-particle's DS pair meets the bound against FP64
    rng = np.random.default_rng(17)
    npair, t_blk = 64, 0.5
    xc = rng.uniform(-8, 8, size=(npair, 3))
    sep = np.where(np.arange(npair)[:, None] < 32,
                   10.0 ** rng.uniform(-7, -3, size=(npair, 1)),
                   rng.uniform(0.1, 4, size=(npair, 1))) * rng.normal(size=(npair, 3))
    xj = xc + sep
    xi = xc
    n = npair
    st = dict(m=np.full(n, 1.0 / n), x0=xj, v0=rng.normal(size=(n, 3)),
              a0=rng.normal(size=(n, 3)), j0=rng.normal(size=(n, 3)), tj=np.full(n, t_blk))
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    g6.g6_set_ti(ctx, t_blk)
    hi, lo, _ = g6.g6x_get_predicted(ctx, n)
    xp, _ = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], t_blk)
    assert np.array_equal(xp, xj)                       # no increment at t_j = t_blk
    ih, il = ds_split(xi)
    dx_ds = ((hi[:, :3] + (-ih)) + (lo[:, :3] + (-il))).astype(np.float64)
    dx = xp - xi
    xs = np.abs(xi) + np.abs(xp)
    hj = hi[:, :3].astype(np.float64)
    hk = ih.astype(np.float64)
    sterbenz = (hj * hk > 0) & (np.abs(hj) <= 2 * np.abs(hk)) & (np.abs(hk) <= 2 * np.abs(hj))
    bound = np.where(sterbenz, 2.0 ** -24 * np.abs(dx) * (1 + 2.0 ** -20) + 2.0 ** -47 * xs,
                     2.0 ** -23 * np.abs(dx) * (1 + 2.0 ** -20) + 2.0 ** -46 * xs)
    err = np.abs(dx_ds - dx)
    assert np.all(err <= bound), np.max(err / bound)
    assert np.count_nonzero(sterbenz[:32]) >= 90         # the close pairs take the tight bound
    # plain single precision fails the tight bound for the close pairs
    dx_sp = (rn32(xp) - rn32(xi)).astype(np.float64)
    assert np.any(np.abs(dx_sp - dx)[:32] > bound[:32])


def test_list_membership_is_bit_exact(ctx):
    # Sect. 4 lists decided in the kernel's own precision: the key is the
    # single-precision softened r^2, fma(dz, dz, fma(dy, dy, fma(dx, dx,
    # eps2))), of the Eq. 3 separations between the predicted DS words of j
    # and the DS pair of x_i, and the radius is h2 + eps2 rounded to float
    # once.  Every DS list shape must return exactly the j with key < radius
    # (self excluded), in ascending j-slot order, the lowest j-slots where a
    # list is longer than its length, and the full count.  Each radius is
    # the squared FP64 distance of the i-particle's k-th nearest j, so one
    # member sits on the boundary of every list.  The nearest neighbour comes
    # from the same key: the j returned must attain the smallest key with
    # eps2 taken off again in float (partials compare that value, so among j
    # whose values tie any may be returned).
    n, t_blk, eps2, m, maxnb = 8192, 0.625, 1e-8, 256, 256
    st = ics.taylor_state(n, 73, t_blk)
    load_j(ctx, st["x0"], st["v0"], st["m"], st["a0"], st["j0"], st["tj"])
    act = np.sort(ics.permutation(n, 73)[:m])
    rng = np.random.default_rng(73)
    xi = st["x0"][act] + rng.normal(scale=1e-3, size=(m, 3))
    vi = st["v0"][act]
    # the restated words and decision
    jh, jl, _ = restated_prediction(st, t_blk)
    xj = jh.astype(np.float64) + jl.astype(np.float64)
    r64 = [np.sum((xj - xi[q]) ** 2, axis=1) for q in range(m)]
    kth = rng.integers(0, 400, size=m)
    h2 = np.array([np.sort(r64[q])[kth[q]] for q in range(m)])
    ih, il = ds_split(xi)
    e2 = rn32(eps2)
    radius = rn32(h2 + e2.astype(np.float64))
    want, flips, unsoft = [], 0, []
    for q in range(m):
        d = [(jh[:, c] + (-ih[q, c])) + (jl[:, c] + (-il[q, c])) for c in range(3)]
        key = fma32(d[2], d[2], fma32(d[1], d[1], fma32(d[0], d[0], np.full(n, e2))))
        key[act[q]] = np.inf
        r64[q][act[q]] = np.inf
        want.append(np.nonzero(key < radius[q])[0])
        unsoft.append(np.maximum(key - e2, np.float32(0)))
        flips += np.count_nonzero((key < radius[q]) != (r64[q] < h2[q]))
    lens = np.array([w.size for w in want])
    assert lens.min() == 0 and np.count_nonzero(lens > maxnb) > 10 and np.median(lens) > 100
    assert flips > 10          # decisions that FP64 distances would take the other way
    shapes = [k for k in range(g6.g6x_variant_count())
              if g6.g6x_variant_info(k)["list"] == 1
              and g6.g6x_variant_info(k)["prec"] == g6.G6X_PREC_DS]
    try:
        for k in [-1] + shapes:
            g6.g6x_set_variant(ctx, k, 0)
            g6.g6_set_ti(ctx, t_blk)
            g6.g6calc_firsthalf(ctx, n, m, act, xi, vi, eps2, h2)
            nnb = g6.g6calc_lasthalf2(ctx, n, m, eps2)[3]
            for q in range(m):
                assert unsoft[q][nnb[q]] == unsoft[q].min(), (k, q)
            assert g6.g6_read_neighbour_list(ctx) == g6.G6_EOVERFLOW
            for q in range(m):
                rc, ln, ids = g6.g6_get_neighbour_list(ctx, q)
                assert ln == lens[q], (k, q, ln, lens[q])
                assert np.array_equal(ids, want[q][:maxnb]), (k, q)
    finally:
        g6.g6x_set_variant(ctx, -1, 0)
