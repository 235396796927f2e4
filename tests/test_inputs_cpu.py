"""The seeded input generators (paper_0902_4463_gb300/ics.py) against the
distributions they claim to draw from: the Plummer model's mass profile and
virial state (Sect. 3 uses Plummer spheres in Henon units), the Salpeter
mass function of the cluster batch, and the Kepler orbits of the binaries of
the binary-rich Plummer model.  CPU only."""
import math

import numpy as np
import pytest

from paper_0902_4463_gb300 import ics

scipy_stats = pytest.importorskip("scipy.stats")


def test_plummer_mass_profile_and_virial_state():
    n = 65536
    m, x, v = ics.plummer(n, 5)
    assert np.allclose((m[:, None] * x).sum(0), 0, atol=1e-14)
    assert np.allclose((m[:, None] * v).sum(0), 0, atol=1e-14)
    # radii in the model's own length unit (Henon scale 3 pi / 16), sampled
    # up to the mass fraction 0.999: M(<r) = r^3 / (1 + r^2)^(3/2) / 0.999
    r = np.linalg.norm(x, axis=1) / ics.HENON_B
    cdf = lambda q: np.minimum(q ** 3 / (1 + q * q) ** 1.5 / 0.999, 1.0)
    d, p = scipy_stats.kstest(r, cdf)
    assert p > 1e-3, (d, p)
    # kinetic energy 1/4 in Henon units (E = -1/4, virial ratio 1/2)
    t = 0.5 * (m * (v * v).sum(1)).sum()
    assert abs(t - 0.25) < 0.01, t
    # isotropic velocities: no net radial or tangential streaming
    vr = (x * v).sum(1) / np.linalg.norm(x, axis=1)
    assert abs(vr.mean()) < 5 * vr.std() / math.sqrt(n)


def test_plummer_potential_energy_of_a_sample():
    # W = -1/2 in Henon units for the continuous model; a sample of 4096
    # stars differs by O(N^-1/2)
    n = 4096
    m, x, v = ics.plummer(n, 6)
    w = 0.0
    for i in range(0, n, 512):
        d = np.linalg.norm(x[i:i + 512, None, :] - x[None, :, :], axis=2)
        np.fill_diagonal(d[:, i:i + 512], np.inf)
        w -= 0.5 * (m[i:i + 512, None] * m[None, :] / d).sum()
    assert abs(w + 0.5) < 0.03, w


def test_salpeter_masses_follow_the_power_law():
    n, alpha, lo, hi = 200000, 2.35, 0.1, 100.0
    m = ics.salpeter_masses(n, 3)
    assert m.sum() == pytest.approx(1.0, rel=1e-12)
    assert m.max() / m.min() <= hi / lo * (1 + 1e-12)
    # undo the normalisation: the smallest of 2e5 draws sits at the lower
    # bound to within a few parts in 1e6
    raw = m * (lo / m.min())
    p1 = 1.0 - alpha
    cdf = lambda q: (np.clip(q, lo, hi) ** p1 - lo ** p1) / (hi ** p1 - lo ** p1)
    d, p = scipy_stats.kstest(raw, cdf)
    assert p > 1e-3, (d, p)
    # maximum-likelihood slope of the truncated power law
    a_grid = np.linspace(2.2, 2.5, 3001)
    ll = [n * math.log((1 - a) / (hi ** (1 - a) - lo ** (1 - a))) - a * np.log(raw).sum()
          for a in a_grid]
    a_hat = a_grid[int(np.argmax(ll))]
    assert abs(a_hat - alpha) < 0.01, a_hat


def test_binaries_have_the_drawn_kepler_orbits():
    n = 20000
    m, x, v, pairs = ics.plummer_with_binaries(n, 9)
    nbin = pairs.shape[0]
    assert nbin == round(0.1 * n / 2)
    i1, i2 = pairs[:, 0], pairs[:, 1]
    r = x[i2] - x[i1]
    u = v[i2] - v[i1]
    mb = m[i1] + m[i2]
    rn = np.linalg.norm(r, axis=1)
    # two-body orbital energy gives the semi-major axis, angular momentum the
    # eccentricity
    a = 1.0 / (2.0 / rn - (u * u).sum(1) / mb)
    h = np.linalg.norm(np.cross(r, u), axis=1)
    e = np.sqrt(np.maximum(0.0, 1.0 - h * h / (mb * a)))
    assert np.all(a > 1e-4 * (1 - 1e-9)) and np.all(a < 1e-2 * (1 + 1e-9))
    assert np.all(e < 1.0)
    # log-uniform semi-major axes and thermal eccentricities (CDF e^2)
    d, p = scipy_stats.kstest(np.log(a), "uniform", args=(math.log(1e-4), math.log(100.0)))
    assert p > 1e-3, (d, p)
    d, p = scipy_stats.kstest(e * e, "uniform")
    assert p > 1e-3, (d, p)
    # each binary's centre of mass is where its Plummer system star is
    assert np.allclose(0.5 * (x[i1] + x[i2]), ics.plummer(n - nbin, 9,
                       masses=np.r_[np.full(nbin, 2.0 / n), np.full(n - 2 * nbin, 1.0 / n)])[1][:nbin],
                       atol=1e-15)
