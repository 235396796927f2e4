"""ctypes marshalling for the C oracle (``oracle.c``).  TEST INFRASTRUCTURE ONLY.

No arithmetic of the method lives here: every function converts numpy arrays to
contiguous float64/int32 buffers, calls the C routine and returns numpy arrays.
``Oracle(path)`` binds any build of ``oracle.c`` (the mutation tests bind
deliberately broken copies); the module-level functions use the default build.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_default = None


def lib_path():
    return _LIB


def compile_source(src, out):
    """gcc-compile one C source (with oracle.h beside it) into a shared library."""
    tmp = out + ".tmp.%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
            "-ffp-contract=off", "-I", _HERE, src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def build(force=False):
    """Compile ``oracle.c`` into ``liboracle.so`` (OpenMP when gcc has it)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_HDR)):
        return _LIB
    return compile_source(_SRC, _LIB)


class RunStats(C.Structure):
    _fields_ = [("nblocks", C.c_long), ("nactive", C.c_long),
                ("t", C.c_double), ("err", C.c_int)]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Oracle:
    """One loaded build of the C oracle."""

    def __init__(self, path):
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.orc_predict.argtypes = [C.c_long, P, P, P, P, P, C.c_double, P, P]
        lib.orc_predict.restype = None
        lib.orc_force.argtypes = [C.c_long, P, P, P, C.c_long, P, P, P, P,
                                  C.c_double, P, P, P, P, P]
        lib.orc_force.restype = None
        lib.orc_neighbours.argtypes = [C.c_long, P, P, C.c_long, P, P, P,
                                       C.c_int, P, P]
        lib.orc_neighbours.restype = C.c_long
        lib.orc_hermite_correct.argtypes = [C.c_double] + [P] * 10
        lib.orc_hermite_correct.restype = None
        lib.orc_aarseth_dt.argtypes = [P, P, P, P, C.c_double]
        lib.orc_aarseth_dt.restype = C.c_double
        lib.orc_block_dt.argtypes = [C.c_double] * 5
        lib.orc_block_dt.restype = C.c_double
        lib.orc_energy.argtypes = [C.c_long, P, P, P, C.c_double]
        lib.orc_energy.restype = C.c_double
        lib.orc_hermite_run.argtypes = [C.c_long, P, P, P, C.c_double,
                                        C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_double, P, P, P,
                                        C.POINTER(RunStats)]
        lib.orc_hermite_run.restype = C.c_int
        self.lib = lib
        self.path = path

    def predict(self, x0, v0, a0, j0, tj, t):
        """Eq. 1 / Eq. 2 prediction of n particles to time t (a0, j0 unscaled)."""
        x0, v0, a0, j0 = (_d(q).reshape(-1, 3) for q in (x0, v0, a0, j0))
        n = x0.shape[0]
        tj = _d(np.broadcast_to(np.asarray(tj, dtype=np.float64), (n,)))
        xp = np.empty((n, 3))
        vp = np.empty((n, 3))
        self.lib.orc_predict(n, _p(x0), _p(v0), _p(a0), _p(j0), _p(tj), float(t),
                             _p(xp), _p(vp))
        return xp, vp

    def force(self, xi, vi, idx_i, xj, vj, mj, idx_j, eps2):
        """Softened acc, jerk, pot and nearest neighbour of each i over all j.

        Returns (acc[ni,3], jerk[ni,3], pot[ni], nnb[ni], nnr2[ni])."""
        xi, vi = _d(xi).reshape(-1, 3), _d(vi).reshape(-1, 3)
        xj, vj = _d(xj).reshape(-1, 3), _d(vj).reshape(-1, 3)
        mj = _d(mj).reshape(-1)
        idx_i, idx_j = _i(idx_i).reshape(-1), _i(idx_j).reshape(-1)
        ni, nj = xi.shape[0], xj.shape[0]
        assert vi.shape[0] == ni and idx_i.shape[0] == ni
        assert vj.shape[0] == nj and mj.shape[0] == nj and idx_j.shape[0] == nj
        acc = np.empty((ni, 3))
        jerk = np.empty((ni, 3))
        pot = np.empty(ni)
        nnb = np.empty(ni, dtype=np.int32)
        nnr2 = np.empty(ni)
        self.lib.orc_force(ni, _p(xi), _p(vi), _p(idx_i), nj, _p(xj), _p(vj), _p(mj),
                           _p(idx_j), float(eps2), _p(acc), _p(jerk), _p(pot),
                           _p(nnb), _p(nnr2))
        return acc, jerk, pot, nnb, nnr2

    def neighbours(self, xi, idx_i, xj, idx_j, h2, maxnb=256):
        """Neighbour lists: returns (nblen[ni], nbl[ni, maxnb], n_overflowed)."""
        xi, xj = _d(xi).reshape(-1, 3), _d(xj).reshape(-1, 3)
        idx_i, idx_j = _i(idx_i).reshape(-1), _i(idx_j).reshape(-1)
        ni, nj = xi.shape[0], xj.shape[0]
        h2 = _d(np.broadcast_to(np.asarray(h2, dtype=np.float64), (ni,)))
        nblen = np.empty(ni, dtype=np.int32)
        nbl = np.full((ni, maxnb), -1, dtype=np.int32)
        nov = self.lib.orc_neighbours(ni, _p(xi), _p(idx_i), nj, _p(xj), _p(idx_j),
                                      _p(h2), int(maxnb), _p(nblen), _p(nbl))
        return nblen, nbl, int(nov)

    def hermite_correct(self, dt, xp, vp, a0, j0, a1, j1):
        """One-particle Hermite corrector: returns (x1, v1, a2, a3)."""
        ins = [_d(q).reshape(3) for q in (xp, vp, a0, j0, a1, j1)]
        outs = [np.empty(3) for _ in range(4)]
        self.lib.orc_hermite_correct(float(dt), *[_p(q) for q in ins],
                                     *[_p(q) for q in outs])
        return tuple(outs)

    def aarseth_dt(self, a, j, a2, a3, eta):
        ins = [_d(q).reshape(3) for q in (a, j, a2, a3)]
        return self.lib.orc_aarseth_dt(*[_p(q) for q in ins], float(eta))

    def block_dt(self, dt_old, dt_req, t, dt_max, dt_min=2.0 ** -40):
        return self.lib.orc_block_dt(float(dt_old), float(dt_req), float(t),
                                     float(dt_max), float(dt_min))

    def energy(self, m, x, v, eps2):
        m = _d(m).reshape(-1)
        x, v = _d(x).reshape(-1, 3), _d(v).reshape(-1, 3)
        return self.lib.orc_energy(m.shape[0], _p(m), _p(x), _p(v), float(eps2))

    def hermite_run(self, m, x, v, eps2, eta, t_end, dt_max=2.0 ** -4,
                    dt_min=2.0 ** -40, eta_s=None):
        """Full block-time-step Hermite integration to t_end.

        Returns dict(x, v, acc, jerk, hist, nblocks, nactive, t, err)."""
        m = _d(m).reshape(-1)
        x = _d(x).reshape(-1, 3).copy()
        v = _d(v).reshape(-1, 3).copy()
        n = m.shape[0]
        if eta_s is None:
            eta_s = eta / 10.0
        acc = np.empty((n, 3))
        jerk = np.empty((n, 3))
        hist = np.zeros(64, dtype=np.int64)
        st = RunStats()
        rc = self.lib.orc_hermite_run(n, _p(m), _p(x), _p(v), float(eps2), float(eta),
                                      float(eta_s), float(dt_max), float(dt_min),
                                      float(t_end), _p(acc), _p(jerk), _p(hist),
                                      C.byref(st))
        return dict(x=x, v=v, acc=acc, jerk=jerk, hist=hist, nblocks=st.nblocks,
                    nactive=st.nactive, t=st.t, err=rc)


def default():
    """The oracle built from ``oracle.c`` (compiled on first use)."""
    global _default
    with _lock:
        if _default is None:
            build()
            _default = Oracle(_LIB)
    return _default


def predict(*a, **k):
    return default().predict(*a, **k)


def force(*a, **k):
    return default().force(*a, **k)


def neighbours(*a, **k):
    return default().neighbours(*a, **k)


def hermite_correct(*a, **k):
    return default().hermite_correct(*a, **k)


def aarseth_dt(*a, **k):
    return default().aarseth_dt(*a, **k)


def block_dt(*a, **k):
    return default().block_dt(*a, **k)


def energy(*a, **k):
    return default().energy(*a, **k)


def hermite_run(*a, **k):
    return default().hermite_run(*a, **k)
