"""Seeded synthetic inputs for the direct-summation Hermite path.

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle's tests.  It holds none of the method's arithmetic (no pair force, no
prediction, no integration step): only initial conditions drawn from seeded
numpy PCG64 streams, so that both sides always see identical inputs.

The paper measures on equal-mass Plummer spheres (Sect. 3, citing Plummer
1915) in N-body (Henon) units; it prints no generator.  The reading used here
is the Aarseth, Henon & Wielen (1974) sampling:
  * cumulative mass fraction X ~ U(0, 0.999) -> r = (X^(-2/3) - 1)^(-1/2);
  * speed fraction q by rejection from g(q) = q^2 (1 - q^2)^(7/2), speed
    q * sqrt(2) (1 + r^2)^(-1/4);
  * isotropic directions;
  * positions scaled by 3 pi / 16 and velocities by (3 pi / 16)^(-1/2), which
    gives E = -1/4 for the continuous model (the sample's own energy differs by
    O(N^-1/2); no re-scaling by a pair sum is done here);
  * shift to the centre-of-mass frame.
"""
import math

import numpy as np

HENON_B = 3.0 * math.pi / 16.0


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(rng, n):
    cth = rng.random(n) * 2.0 - 1.0
    phi = rng.random(n) * 2.0 * math.pi
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def plummer(n, seed, masses=None, xmax=0.999):
    """Plummer sphere of n particles.  Returns (m[n], x[n,3], v[n,3]) float64.

    masses: optional per-particle masses (default equal, total 1)."""
    rng = _rng(seed)
    if masses is None:
        m = np.full(n, 1.0 / n)
    else:
        m = np.asarray(masses, dtype=np.float64).copy()
    X = rng.random(n) * xmax
    X = np.maximum(X, 1e-300)
    r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _isotropic(rng, n)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.random(todo.size)
        yy = rng.random(todo.size) * 0.1
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    speed = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v = speed[:, None] * _isotropic(rng, n)
    x *= HENON_B
    v /= math.sqrt(HENON_B)
    mt = m.sum()
    x -= (m[:, None] * x).sum(0) / mt
    v -= (m[:, None] * v).sum(0) / mt
    return m, x, v


def salpeter_masses(n, seed, alpha=2.35, mlo=0.1, mhi=100.0):
    """n masses from dN/dm ~ m^-alpha on [mlo, mhi] by inverse CDF, sum 1."""
    rng = _rng(seed)
    u = rng.random(n)
    p = 1.0 - alpha
    m = (mlo ** p + u * (mhi ** p - mlo ** p)) ** (1.0 / p)
    return m / m.sum()


def cluster_batch(ncl, seed, nmin=256, nmax=16384):
    """Batch of ncl independent clusters: N_k = round(exp(U(ln nmin, ln nmax))),
    Salpeter masses, Plummer positions and velocities, eps2_k = (4/N_k)^2.
    Returns a list of dicts (n, m, x, v, eps2)."""
    rng = _rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), ncl))).astype(int)
    out = []
    for k, nk in enumerate(ns):
        mk = salpeter_masses(int(nk), seed * 100003 + 2 * k + 1)
        m, x, v = plummer(int(nk), seed * 100003 + 2 * k + 2, masses=mk)
        out.append(dict(n=int(nk), m=m, x=x, v=v, eps2=(4.0 / nk) ** 2))
    return out


def _kepler_E(M, e):
    E = M + e * np.sin(M)
    for _ in range(60):
        E = E - (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
    return E


def plummer_with_binaries(n, seed, fbin=0.1, amin=1e-4, amax=1e-2):
    """Plummer sphere of n stars, a fraction fbin of them in equal-mass
    binaries (each component 1/n).  The binary centres of mass are Plummer
    stars of mass 2/n; semi-major axes log-uniform in [amin, amax], thermal
    eccentricities (e = sqrt(U)), isotropic orientations, uniform mean anomaly.
    Returns (m, x, v, pairs) where pairs[k] = (i1, i2) index the components."""
    nbin = int(round(fbin * n / 2.0))
    nsys = n - nbin
    rng = _rng(seed * 7919 + 17)
    msys = np.full(nsys, 1.0 / n)
    msys[:nbin] = 2.0 / n
    _, X, V = plummer(nsys, seed, masses=msys)
    a = np.exp(rng.uniform(math.log(amin), math.log(amax), nbin))
    e = np.sqrt(rng.random(nbin))
    Mn = rng.random(nbin) * 2.0 * math.pi
    cosi = rng.random(nbin) * 2.0 - 1.0
    inc = np.arccos(cosi)
    Om = rng.random(nbin) * 2.0 * math.pi
    om = rng.random(nbin) * 2.0 * math.pi
    E = _kepler_E(Mn, e)
    mb = 2.0 / n
    fac = np.sqrt(1.0 - e * e)
    rp = np.stack([a * (np.cos(E) - e), a * fac * np.sin(E), np.zeros(nbin)], 1)
    vscale = np.sqrt(mb / a) / (1.0 - e * np.cos(E))
    vp = np.stack([-vscale * np.sin(E), vscale * fac * np.cos(E), np.zeros(nbin)], 1)

    def rot(vec):
        co, so = np.cos(om), np.sin(om)
        x1 = co * vec[:, 0] - so * vec[:, 1]
        y1 = so * vec[:, 0] + co * vec[:, 1]
        z1 = vec[:, 2]
        ci, si = np.cos(inc), np.sin(inc)
        y2 = ci * y1 - si * z1
        z2 = si * y1 + ci * z1
        cO, sO = np.cos(Om), np.sin(Om)
        return np.stack([cO * x1 - sO * y2, sO * x1 + cO * y2, z2], 1)

    rr, vv = rot(rp), rot(vp)
    m = np.full(n, 1.0 / n)
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    x[:nbin] = X[:nbin] - 0.5 * rr
    v[:nbin] = V[:nbin] - 0.5 * vv
    x[nbin:2 * nbin] = X[:nbin] + 0.5 * rr
    v[nbin:2 * nbin] = V[:nbin] + 0.5 * vv
    x[2 * nbin:] = X[nbin:]
    v[2 * nbin:] = V[nbin:]
    pairs = np.stack([np.arange(nbin), np.arange(nbin) + nbin], 1)
    return m, x, v, pairs


def taylor_state(n, seed, t_blk, dt_levels=(4, 12)):
    """Synthetic j-particle Taylor data for prediction tests and sweeps.

    Returns dict with x0, v0 (Plummer), a0, j0 (isotropic with Plummer-like
    magnitudes; they are inputs, not forces of this configuration) and tj, the
    last update time of each particle: t_blk minus a random power-of-two step
    2^-k with k uniform in dt_levels, or 0 for dt_levels=None."""
    m, x, v = plummer(n, seed)
    rng = _rng(seed + 0x9E3779B9)
    a0 = rng.normal(size=(n, 3)) * 0.6
    j0 = rng.normal(size=(n, 3)) * 3.0
    if dt_levels is None:
        tj = np.zeros(n)
    else:
        k = rng.integers(dt_levels[0], dt_levels[1] + 1, size=n)
        tj = t_blk - np.ldexp(1.0, -k)
    return dict(m=m, x0=x, v0=v, a0=a0, j0=j0, tj=tj)


def permutation(n, seed):
    """Seeded permutation of range(n), used to pick active i-particles."""
    return _rng(seed + 12345).permutation(n)
