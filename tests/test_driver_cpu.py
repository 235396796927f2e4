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
