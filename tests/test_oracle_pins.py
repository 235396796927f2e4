"""Pins for the FP64 oracle against facts fixed outside the oracle itself:
closed forms, finite differences, conservation laws and constructed cases.

Each test names the paper passage whose arithmetic it pins.  A plausible slip
in the oracle (dropped term, wrong sign, swapped operand, wrong coefficient)
makes at least one of these fail; see ``test_oracle_mutations.py``.
"""
import math

import numpy as np
import pytest

from paper_0902_4463_gb300 import ics


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


# ------------------------------------------------------------------ forces --
# Sect. 2.3 (calculation step): softened acceleration, jerk and potential.

@pytest.mark.parametrize("eps2", [0.0, 1e-3])
def test_summed_forces_match_high_precision_brute_force(orc, eps2):
    """Eight particles, every i against every j (self excluded by index),
    evaluated independently in 50-digit decimal arithmetic from the same
    binary64 inputs: the summed softened acceleration, jerk and potential of
    the oracle agree to a few ulps of the largest term, and its nearest
    neighbour is the one the exact squared distances (rational arithmetic)
    give."""
    import decimal
    from fractions import Fraction
    rng = np.random.default_rng(17)
    n = 8
    x = rng.normal(size=(n, 3))
    v = rng.normal(size=(n, 3))
    m = rng.uniform(0.1, 1.0, n)
    idx = np.arange(n)
    acc, jerk, pot, nnb, nnr2 = orc.force(x, v, idx, x, v, m, idx, eps2)
    ctx = decimal.Context(prec=50)
    D = lambda f: ctx.create_decimal(float(f))          # exact binary64 -> decimal
    e2 = D(eps2)
    for i in range(n):
        a = [decimal.Decimal(0)] * 3
        jk = [decimal.Decimal(0)] * 3
        p = decimal.Decimal(0)
        scale_a = scale_j = scale_p = 0.0
        best, best_j = None, -1
        for j in range(n):
            if j == i:
                continue
            r = [ctx.subtract(D(x[j, d]), D(x[i, d])) for d in range(3)]
            u = [ctx.subtract(D(v[j, d]), D(v[i, d])) for d in range(3)]
            r2 = ctx.add(ctx.add(ctx.multiply(r[0], r[0]), ctx.multiply(r[1], r[1])),
                         ctx.multiply(r[2], r[2]))
            s2 = ctx.add(r2, e2)
            s = ctx.sqrt(s2)
            inv3 = ctx.divide(1, ctx.multiply(s2, s))
            rv = sum((ctx.multiply(r[d], u[d]) for d in range(3)), decimal.Decimal(0))
            mj = D(m[j])
            for d in range(3):
                a[d] = ctx.add(a[d], ctx.multiply(ctx.multiply(mj, inv3), r[d]))
                t = ctx.subtract(u[d], ctx.divide(ctx.multiply(3 * rv, r[d]), s2))
                jk[d] = ctx.add(jk[d], ctx.multiply(ctx.multiply(mj, inv3), t))
            p = ctx.subtract(p, ctx.divide(mj, s))
            scale_a = max(scale_a, float(mj * ctx.divide(1, s2)))
            scale_j = max(scale_j, float(mj * inv3 * (abs(rv) * 3 / s + sum(abs(q) for q in u))))
            scale_p = max(scale_p, float(ctx.divide(mj, s)))
            exact = sum((Fraction(float(x[j, d])) - Fraction(float(x[i, d]))) ** 2
                        for d in range(3))
            if best is None or exact < best:
                best, best_j = exact, j
        for d in range(3):
            assert abs(acc[i, d] - float(a[d])) <= 64 * 2.0 ** -52 * scale_a * n, (i, d)
            assert abs(jerk[i, d] - float(jk[d])) <= 64 * 2.0 ** -52 * scale_j * n, (i, d)
        assert abs(pot[i] - float(p)) <= 64 * 2.0 ** -52 * scale_p * n, i
        assert nnb[i] == best_j
        assert nnr2[i] == pytest.approx(float(best), rel=1e-14)


@pytest.mark.parametrize("eps2", [0.0, 0.04])
def test_two_body_closed_form(orc, eps2):
    e = _unit([0.3, -0.7, 0.2])
    d, mj = 1.7, 0.37
    xi = np.zeros((1, 3))
    xj = (d * e)[None, :]
    z = np.zeros((1, 3))
    acc, jerk, pot, nnb, nnr2 = orc.force(xi, z, [0], xj, z, [mj], [1], eps2)
    s2 = d * d + eps2
    assert np.allclose(acc[0], mj * d * e / s2 ** 1.5, rtol=1e-14, atol=0)
    assert np.allclose(jerk[0], 0.0, atol=1e-300)
    assert pot[0] == pytest.approx(-mj / math.sqrt(s2), rel=1e-14)
    assert nnb[0] == 0 and nnr2[0] == pytest.approx(d * d, rel=1e-14)


def test_jerk_radial_and_tangential_closed_forms(orc):
    # With eps = 0: radial relative speed u gives jerk = -2 m u e / d^3
    # (time derivative of m e / d^2 with d' = u); a tangential speed w
    # rotates e at rate w/d, giving jerk = m w / d^3.
    e = _unit([1.0, 2.0, -0.5])
    t = _unit(np.cross(e, [0.0, 0.0, 1.0]))
    d, m, u, w = 0.8, 0.25, 0.6, -1.3
    xi = np.zeros((1, 3))
    xj = (d * e)[None]
    vi = np.zeros((1, 3))
    _, jr, *_ = orc.force(xi, vi, [0], xj, (u * e)[None], [m], [1], 0.0)
    assert np.allclose(jr[0], -2.0 * m * u * e / d ** 3, rtol=1e-13, atol=1e-15)
    _, jt, *_ = orc.force(xi, vi, [0], xj, (w * t)[None], [m], [1], 0.0)
    assert np.allclose(jt[0], m * w * t / d ** 3, rtol=1e-13, atol=1e-15)


def test_equilateral_triangle(orc):
    s, m = 1.3, 0.2
    h = s * math.sqrt(3.0) / 2.0
    x = np.array([[0.0, 0.0, 0.0], [s, 0.0, 0.0], [s / 2.0, h, 0.0]])
    rot = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))[0]
    x = x @ rot.T + np.array([0.3, -0.2, 0.9])
    v = np.zeros_like(x)
    idx = np.arange(3)
    acc, _, pot, _, _ = orc.force(x, v, idx, x, v, np.full(3, m), idx, 0.0)
    cen = x.mean(0)
    for k in range(3):
        expect = math.sqrt(3.0) * m / s ** 2 * _unit(cen - x[k])
        assert np.allclose(acc[k], expect, rtol=1e-13, atol=1e-15)
        assert pot[k] == pytest.approx(-2.0 * m / s, rel=1e-14)


def _cluster(n, seed, eps_scale=1.0):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 3))
    v = rng.normal(size=(n, 3)) * 0.5
    m = rng.random(n) + 0.1
    return m / m.sum(), x, v


def test_jerk_is_time_derivative_of_acceleration(orc):
    # Finite difference of a(t) along straight-line motion x(t) = x + v t,
    # fourth-order central stencil; independent of the jerk formula.
    m, x, v = _cluster(8, 11)
    idx = np.arange(8)
    eps2 = 0.01
    _, jerk, *_ = orc.force(x, v, idx, x, v, m, idx, eps2)
    h = 1e-3

    def acc_at(t):
        xt = x + v * t
        return orc.force(xt, v, idx, xt, v, m, idx, eps2)[0]

    fd = (-acc_at(2 * h) + 8 * acc_at(h) - 8 * acc_at(-h) + acc_at(-2 * h)) / (12 * h)
    scale = np.abs(jerk).max()
    assert np.abs(fd - jerk).max() < 1e-9 * scale


def test_acceleration_is_minus_gradient_of_potential(orc):
    m, x, v = _cluster(8, 5)
    idx = np.arange(8)
    eps2 = 0.02
    acc, *_ = orc.force(x, v, idx, x, v, m, idx, eps2)
    h = 1e-4
    for i in range(8):
        g = np.empty(3)
        for c in range(3):
            def phi(dx):
                xi = x[i:i + 1].copy()
                xi[0, c] += dx
                return orc.force(xi, v[i:i + 1], [i], x, v, m, idx, eps2)[2][0]
            g[c] = (-phi(2 * h) + 8 * phi(h) - 8 * phi(-h) + phi(-2 * h)) / (12 * h)
        assert np.allclose(-g, acc[i], rtol=1e-8, atol=1e-10 * np.abs(acc).max())


def test_momentum_torque_and_pair_energy_balance(orc):
    m, x, v = _cluster(64, 9)
    idx = np.arange(64)
    eps2 = 1e-3
    acc, jerk, pot, _, _ = orc.force(x, v, idx, x, v, m, idx, eps2)
    ma = m[:, None] * acc
    assert np.abs(ma.sum(0)).max() < 1e-14 * np.abs(ma).sum()
    mj = m[:, None] * jerk
    assert np.abs(mj.sum(0)).max() < 1e-14 * np.abs(mj).sum()
    torque = np.cross(x, ma).sum(0)
    assert np.abs(torque).max() < 1e-14 * np.abs(np.cross(x, ma)).sum()
    # half sum m phi equals the explicit pair-loop potential energy
    w = orc.energy(m, x, np.zeros_like(v), eps2)
    assert 0.5 * (m * pot).sum() == pytest.approx(w, rel=1e-13)
    kin = 0.5 * (m * (v * v).sum(1)).sum()
    assert orc.energy(m, x, v, eps2) == pytest.approx(kin + w, rel=1e-13)


def test_self_excluded_by_index_not_by_distance(orc):
    # Two distinct particles at the same point still interact (softened);
    # the particle carrying the i index never acts on itself.
    x = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    v = np.zeros((3, 3))
    m = np.array([0.1, 0.2, 0.3])
    idx = np.array([4, 7, 9])
    eps2 = 0.25
    acc, _, pot, nnb, nnr2 = orc.force(x[:1], v[:1], [4], x, v, m, idx, eps2)
    assert pot[0] == pytest.approx(-(0.2 / 0.5 + 0.3 / math.sqrt(1.25)), rel=1e-14)
    assert acc[0, 0] == pytest.approx(0.3 / 1.25 ** 1.5, rel=1e-14)
    assert nnb[0] == 1 and nnr2[0] == 0.0


# -------------------------------------------------------- nearest neighbour --
# Sect. 2.5: nearest-neighbour search per i-particle.

def test_nearest_neighbour_constructed_line(orc):
    gaps = np.array([0.5, 0.3, 0.9, 0.2, 0.7, 0.4])
    xs = np.concatenate([[0.0], np.cumsum(gaps)])
    n = xs.size
    x = np.zeros((n, 3))
    x[:, 1] = xs
    perm = np.array([3, 0, 6, 2, 5, 1, 4])          # store out of order
    xj = x[perm]
    idx = perm.copy()
    _, _, _, nnb, nnr2 = orc.force(x, np.zeros_like(x), np.arange(n), xj,
                                   np.zeros_like(x), np.ones(n), idx, 1e-4)
    for k in range(n):
        left = gaps[k - 1] if k > 0 else np.inf
        right = gaps[k] if k < n - 1 else np.inf
        near = k - 1 if left < right else k + 1
        assert idx[nnb[k]] == near
        assert nnr2[k] == pytest.approx(min(left, right) ** 2, rel=1e-12)


def test_nearest_neighbour_tie_goes_to_lower_j(orc):
    x = np.array([[-1.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0], [0.0, 1.0, 0]])
    v = np.zeros_like(x)
    idx = np.array([10, 11, 12, 13])
    _, _, _, nnb, _ = orc.force(x[1:2], v[:1], [11], x, v, np.ones(4), idx, 0.0)
    assert nnb[0] == 0
    xr = x[[3, 2, 1, 0]]
    _, _, _, nnb, _ = orc.force(x[1:2], v[:1], [11], xr, v, np.ones(4), idx[[3, 2, 1, 0]], 0.0)
    assert nnb[0] == 0                               # position 0 is now index 13


def test_nearest_neighbour_none_when_alone(orc):
    x = np.array([[0.3, 0.1, 0.2]])
    _, _, pot, nnb, nnr2 = orc.force(x, x, [5], x, x, [1.0], [5], 1e-2)
    assert nnb[0] == -1 and math.isinf(nnr2[0]) and pot[0] == 0.0


# ---------------------------------------------------------- neighbour lists --
# Sect. 4: lists of j within h2 of each i, fixed maximum length (256).

def test_neighbour_list_shells_and_overflow(orc):
    rng = np.random.default_rng(2)
    radii = np.array([0.05, 0.2, 0.099, 0.1001, 0.3, 0.01, 0.0999])
    dirs = rng.normal(size=(radii.size, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    xi = np.array([[0.5, -0.2, 0.1]])
    xj = np.vstack([xi, xi + radii[:, None] * dirs])
    idx = np.arange(xj.shape[0]) + 100
    nblen, nbl, nov = orc.neighbours(xi, [100], xj, idx, [0.1 ** 2], maxnb=256)
    expect = [1 + k for k in range(radii.size) if radii[k] < 0.1]
    assert nblen[0] == len(expect) and nov == 0
    assert list(nbl[0, :nblen[0]]) == expect
    nblen, nbl, nov = orc.neighbours(xi, [100], xj, idx, [0.1 ** 2], maxnb=2)
    assert nblen[0] == len(expect) and nov == 1
    assert list(nbl[0]) == expect[:2]
    nblen, nbl, nov = orc.neighbours(xi, [100], xj, idx, [0.1 ** 2], maxnb=len(expect) - 1)
    assert nov == 1 and list(nbl[0]) == expect[:-1]
    nblen, nbl, nov = orc.neighbours(xi, [100], xj, idx, [0.1 ** 2], maxnb=len(expect))
    assert nov == 0 and list(nbl[0]) == expect


# --------------------------------------------------------------- predictor --
# Sect. 2.2, Eq. 1 and Eq. 2.

def test_predictor_truncation_error_on_circular_motion(orc):
    # Uniform circular motion: the third-order Taylor prediction misses
    # R (w dt)^4 / 24 in x and R (w dt)^5 / 120 in y, and in the velocity
    # R w (w dt)^3 / 6 in vx and R w (w dt)^4 / 24 in vy.
    R, w, t0 = 1.3, 2.1, 0.375
    x0 = np.array([[R, 0.0, 0.0]])
    v0 = np.array([[0.0, R * w, 0.0]])
    a0 = np.array([[-R * w * w, 0.0, 0.0]])
    j0 = np.array([[0.0, -R * w ** 3, 0.0]])
    for dt in (2e-2, 1e-2):
        xp, vp = orc.predict(x0, v0, a0, j0, [t0], t0 + dt)
        th = w * dt
        ex = R * math.cos(th) - xp[0, 0]
        ey = R * math.sin(th) - xp[0, 1]
        evx = -R * w * math.sin(th) - vp[0, 0]
        evy = R * w * math.cos(th) - vp[0, 1]
        assert ex / (R * th ** 4 / 24) == pytest.approx(1.0, abs=2 * th * th)
        assert ey / (R * th ** 5 / 120) == pytest.approx(1.0, abs=2 * th * th)
        assert evx / (R * w * th ** 3 / 6) == pytest.approx(1.0, abs=2 * th * th)
        assert evy / (R * w * th ** 4 / 24) == pytest.approx(1.0, abs=2 * th * th)
        assert xp[0, 2] == 0.0 and vp[0, 2] == 0.0


def test_predictor_exact_for_constant_jerk(orc):
    """Motion with constant jerk is a cubic in time, which Eq. 1 and Eq. 2
    reproduce exactly: the prediction equals the exact rational evaluation
    of x0 + v0 dt + a0 dt^2/2 + j dt^3/6 (and its derivative) to within the
    rounding of the FP64 sums, for many particles, each predicted over its
    own time since t_j (dt = t_blk - t_j)."""
    from fractions import Fraction as F
    rng = np.random.default_rng(29)
    n = 64
    x0, v0 = rng.normal(size=(n, 3)) * 10, rng.normal(size=(n, 3))
    a0, j0 = rng.normal(size=(n, 3)), rng.normal(size=(n, 3)) * 5
    tj = 0.5 - np.ldexp(1.0, -rng.integers(1, 12, n))
    t_blk = 0.5
    xp, vp = orc.predict(x0, v0, a0, j0, tj, t_blk)
    for i in range(n):
        dt = F(t_blk) - F(float(tj[i]))
        for d in range(3):
            ex = (F(float(x0[i, d])) + F(float(v0[i, d])) * dt + F(float(a0[i, d])) * dt ** 2 / 2
                  + F(float(j0[i, d])) * dt ** 3 / 6)
            ev = F(float(v0[i, d])) + F(float(a0[i, d])) * dt + F(float(j0[i, d])) * dt ** 2 / 2
            sx = abs(x0[i, d]) + abs(v0[i, d] * float(dt)) + abs(a0[i, d]) + abs(j0[i, d])
            sv = abs(v0[i, d]) + abs(a0[i, d]) + abs(j0[i, d])
            assert abs(xp[i, d] - float(ex)) <= 8 * 2.0 ** -52 * sx, (i, d)
            assert abs(vp[i, d] - float(ev)) <= 8 * 2.0 ** -52 * sv, (i, d)


# -------------------------------------------------------------- integrator --
# Sect. 2: 4th-order Hermite predictor-corrector with block time steps.

def test_hermite_corrector_exact_for_cubic_acceleration(orc):
    # For a(t) a cubic polynomial the Hermite interpolant is exact: the
    # corrector recovers a'' and a''' and lands on the exact trajectory
    # (integrated here with numpy's polynomial antiderivative).
    rng = np.random.default_rng(4)
    A = rng.normal(size=(4, 3))                      # a, a', a'', a''' at t0
    x0, v0 = rng.normal(size=3), rng.normal(size=3)
    h = 0.3
    polys = [np.polynomial.Polynomial([A[0, c], A[1, c], A[2, c] / 2, A[3, c] / 6])
             for c in range(3)]
    a1 = np.array([p(h) for p in polys])
    j1 = np.array([p.deriv()(h) for p in polys])
    xp, vp = orc.predict(x0[None], v0[None], A[0][None], A[1][None], [0.0], h)
    x1, v1, a2, a3 = orc.hermite_correct(h, xp[0], vp[0], A[0], A[1], a1, j1)
    assert np.allclose(a2, A[2], rtol=1e-11, atol=1e-11)
    assert np.allclose(a3, A[3], rtol=1e-10, atol=1e-10)
    for c in range(3):
        vel = polys[c].integ(k=v0[c])
        pos = vel.integ(k=x0[c])
        assert v1[c] == pytest.approx(vel(h), rel=1e-13, abs=1e-13)
        assert x1[c] == pytest.approx(pos(h), rel=1e-13, abs=1e-13)


def test_aarseth_step_on_circular_orbit(orc):
    # Circular motion with angular rate w: |a^(k)| = |a| w^k, so the
    # criterion gives exactly sqrt(eta) / w.
    A, w, th, eta = 0.8, 3.0, 0.7, 0.02
    c, s = math.cos(th), math.sin(th)
    a = -A * np.array([c, s, 0.0])
    j = A * w * np.array([s, -c, 0.0])
    a2 = A * w * w * np.array([c, s, 0.0])
    a3 = A * w ** 3 * np.array([-s, c, 0.0])
    assert orc.aarseth_dt(a, j, a2, a3, eta) == pytest.approx(math.sqrt(eta) / w, rel=1e-14)


def test_block_step_quantisation(orc):
    dmax = 2.0 ** -4
    assert orc.block_dt(2 ** -6, 0.01, 0.0, dmax) == 2 ** -7      # halve to <= req
    assert orc.block_dt(2 ** -6, 0.001, 0.0, dmax) == 2 ** -10
    assert orc.block_dt(2 ** -6, 1.0, 2 ** -5, dmax) == 2 ** -5   # commensurate: double once
    assert orc.block_dt(2 ** -6, 1.0, 3 * 2 ** -6, dmax) == 2 ** -6  # not commensurate
    assert orc.block_dt(2 ** -4, 1.0, 0.5, dmax) == 2 ** -4       # capped at dt_max
    assert orc.block_dt(2 ** -6, 0.02, 2 ** -5, dmax) == 2 ** -6  # req < 2 dt: keep
    assert orc.block_dt(2 ** -39, 1e-13, 0.0, dmax) == -1.0       # below 2^-40


def _kepler_relative(t, a=1.0, e=0.5, mtot=1.0):
    n = math.sqrt(mtot / a ** 3)
    M = n * t
    E = M
    for _ in range(100):
        E -= (E - e * math.sin(E) - M) / (1.0 - e * math.cos(E))
    r = np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])
    rdot = n * a / (1 - e * math.cos(E))
    vv = np.array([-rdot * math.sin(E), rdot * math.sqrt(1 - e * e) * math.cos(E), 0.0])
    return r, vv


def _kepler_ic(a=1.0, e=0.5):
    rp = a * (1 - e)
    vp = math.sqrt((1 + e) / (a * (1 - e)))
    m = np.array([0.5, 0.5])
    x = np.array([[-rp / 2, 0, 0], [rp / 2, 0, 0]])
    v = np.array([[0, -vp / 2, 0], [0, vp / 2, 0]])
    return m, x, v


def test_kepler_orbit_closed_form_and_fourth_order(orc):
    m, x, v = _kepler_ic()
    t_end = 2.0
    r_exact, v_exact = _kepler_relative(t_end)
    E0 = orc.energy(m, x, v, 0.0)
    assert E0 == pytest.approx(-0.125, rel=1e-14)    # -m1 m2 / (2a)
    errs, dEs = [], []
    for eta in (0.02, 0.005):
        out = orc.hermite_run(m, x, v, 0.0, eta, t_end)
        assert out["err"] == 0 and out["t"] == t_end
        rel = out["x"][1] - out["x"][0]
        errs.append(np.linalg.norm(rel - r_exact))
        dEs.append(abs(orc.energy(m, out["x"], out["v"], 0.0) / E0 - 1))
        # centre of mass stays at rest
        assert np.abs((m[:, None] * out["x"]).sum(0)).max() < 1e-13
    assert errs[1] < 2e-4
    # dt ~ sqrt(eta): a 4x smaller eta halves every step, a 4th-order scheme
    # then cuts both errors about 16x
    assert 8.0 < errs[0] / errs[1] < 32.0
    assert 8.0 < dEs[0] / dEs[1] < 32.0


def test_plummer_energy_conservation_and_block_structure(orc):
    m, x, v = ics.plummer(128, 21)
    eps2 = 1e-2
    E0 = orc.energy(m, x, v, eps2)
    out = orc.hermite_run(m, x, v, eps2, 0.01, 0.25)
    assert out["err"] == 0 and out["t"] == 0.25
    E1 = orc.energy(m, out["x"], out["v"], eps2)
    assert abs(E1 / E0 - 1) < 1e-7
    assert out["nactive"] > 128 and out["hist"].sum() == out["nblocks"]
    # block steps apply the two halves of a pair force at different times,
    # so momentum is conserved only to the integration error
    p = (m[:, None] * out["v"]).sum(0)
    assert np.abs(p).max() < 1e-7


def test_plummer_generator_moments():
    m, x, v = ics.plummer(20000, 1)
    assert m.sum() == pytest.approx(1.0, rel=1e-14)
    assert np.abs((m[:, None] * x).sum(0)).max() < 1e-12
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-12
    # kinetic energy of the model is 1/4 in Henon units (E = -1/4, Q = 1/2)
    T = 0.5 * (m * (v * v).sum(1)).sum()
    assert T == pytest.approx(0.25, rel=0.03)
    # half-mass radius of a Plummer sphere: b / sqrt(2^(2/3) - 1) ~ 0.769
    r = np.sort(np.linalg.norm(x, axis=1))
    assert r[len(r) // 2] == pytest.approx(ics.HENON_B / math.sqrt(2 ** (2 / 3) - 1), rel=0.03)


def test_neighbour_radius_is_strict(orc):
    # r^2 == h2 exactly (0.5^2 = 0.25 in binary) is outside the list.
    xi = np.zeros((1, 3))
    xj = np.array([[0.0, 0, 0], [0.5, 0, 0], [0, 0.25, 0], [0, 0, -0.75]])
    nblen, nbl, nov = orc.neighbours(xi, [0], xj, [0, 1, 2, 3], [0.25])
    assert nblen[0] == 1 and nbl[0, 0] == 2 and nov == 0
