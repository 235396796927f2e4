"""Thin ctypes binding of ``libg6gb.so`` (declared in ``include/g6gb.h``).

Argument marshalling only: every function converts numpy arrays (or device
pointers) to the C types and calls the C entry point of the same name; all
work of the hot path happens in the CUDA library.  There is no fallback: if
the library is missing or cannot load, ``lib()`` raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libg6gb.so")

G6_OK = 0
G6_EINVAL = -22
G6_ENOTOPEN = -19
G6_EBUSY = -16
G6_ENOMEM = -12
G6_EIO = -5
G6_ETIMEDOUT = -110
G6_ENODEV = -6
G6_EOVERFLOW = 1
G6_MAXNB = 256
G6X_MAXNB_LIMIT = 4096
G6_MAX_CLUSTERS = 16
G6X_PREC_DS = 0
G6X_PREC_FP64 = 1
G6X_PREC_DS_X64 = 2
G6X_PREC_DS_DSSUB = 3
G6X_NOALLOC_NI_MAX = 16384
G6X_NOALLOC_SCRATCH_BYTES = 147456 * 72

# Record layouts of the device-resident entry points (g6x_jrec, g6x_irec,
# g6x_out in g6gb.h).
JREC = np.dtype([("x", "<f8", 3), ("v", "<f8", 3), ("a2", "<f8", 3), ("j6", "<f8", 3),
                 ("mass", "<f8"), ("tj", "<f8"), ("address", "<i4"), ("index", "<i4")])
IREC = np.dtype([("x", "<f8", 3), ("v", "<f8", 3), ("h2", "<f8"), ("index", "<i4"),
                 ("pad", "<i4")])
OUT = np.dtype([("acc", "<f8", 3), ("jerk", "<f8", 3), ("pot", "<f8"), ("nnb", "<i4"),
                ("nnr2", "<f4")])
assert JREC.itemsize == 120 and IREC.itemsize == 64 and OUT.itemsize == 64

# Every symbol include/g6gb.h declares.
EXPORTS = [
    "g6_open", "g6_close", "g6_npipes", "g6_set_tunit", "g6_set_xunit", "g6_set_ti",
    "g6_set_j_particle", "g6calc_firsthalf", "g6calc_lasthalf", "g6calc_lasthalf2",
    "g6_read_neighbour_list", "g6_get_neighbour_list", "g6x_open_ex",
    "g6x_set_precision", "g6x_set_ni_max", "g6x_set_stream", "g6x_set_allocator",
    "g6x_set_j_particles", "g6x_strerror", "g6x_set_j_dev", "g6x_calc_dev",
    "g6x_calc_dev_noalloc", "g6x_sync", "g6x_set_variant",
    "g6x_autotune", "g6x_load_tuning", "g6x_clear_tuning", "g6x_get_predicted", "g6x_last_config",
    "g6x_launch_count", "g6x_set_wait_limit", "g6x_probe_wait_timeout", "g6x_set_timing", "g6x_get_timing", "g6h_correct_block", "g6h_create", "g6h_run", "g6h_get_state", "g6h_energy",
    "g6h_stats", "g6h_profile", "g6h_destroy", "g6h_checkpoint", "g6h_restore",
    "g6h_set_neighbour_radius", "g6h_neighbour_stats", "g6h_run_blocks",
    "g6h_correct_block_ex", "g6h_set_force_noise", "g6hb_set_force_noise",
    "g6x_fp32_probe", "g6x_fp64_probe", "g6x_plan_launch", "g6x_variant_info",
    "g6x_set_max_neighbours", "g6x_max_neighbours", "g6x_list_reruns",
    "g6x_batch_create", "g6x_batch_destroy", "g6x_batch_irecs", "g6x_batch_results",
    "g6x_batch_set_j", "g6x_batch_set_j_many", "g6x_batch_calc", "g6x_batch_launch_count",
    "g6x_batch_set_schedule", "g6x_batch_get_schedule", "g6x_batch_autotune", "g6hb_autotune",
    "g6hb_set_schedule", "g6x_batch_set_timing", "g6x_batch_get_timing", "g6hb_batch",
    "g6hb_create", "g6hb_step", "g6hb_run", "g6hb_set_mode", "g6hb_stats", "g6hb_get_state",
    "g6hb_destroy", "g6hb_get_state_ex",
]

_lib = None
P = C.c_void_p
I = C.c_int
D = C.c_double
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class G6Error(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, strerror(code) if _lib else "", code))


def lib():
    """Load libg6gb.so (raises if it was not built: no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libg6gb.so is not built; run paper_0902_4463_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        sig = {
            "g6_open": (I, [I]), "g6_close": (I, [I]), "g6_npipes": (I, []),
            "g6_set_tunit": (I, [I]), "g6_set_xunit": (I, [I]), "g6_set_ti": (I, [I, D]),
            "g6_set_j_particle": (I, [I, I, I, D, D, D, P, P, P, P, P]),
            "g6calc_firsthalf": (None, [I, I, I, P, P, P, P, P, P, D, P]),
            "g6calc_lasthalf": (I, [I, I, I, P, P, P, D, P, P, P, P]),
            "g6calc_lasthalf2": (I, [I, I, I, P, P, P, D, P, P, P, P, P]),
            "g6_read_neighbour_list": (I, [I]),
            "g6_get_neighbour_list": (I, [I, I, I, P, P]),
            "g6x_open_ex": (I, [I, I, I]), "g6x_set_precision": (I, [I, I]),
            "g6x_set_ni_max": (I, [I, I]), "g6x_set_stream": (I, [I, P]),
            "g6x_set_allocator": (I, [ALLOC_FN, FREE_FN, P]),
            "g6x_set_j_particles": (I, [I, I, P, P, P, P, P, P, P, P]),
            "g6x_strerror": (C.c_char_p, [I]),
            "g6x_set_j_dev": (I, [I, I, P]),
            "g6x_calc_dev": (I, [I, D, I, I, P, D, I, P]),
            "g6x_calc_dev_noalloc": (I, [I, D, I, I, P, D, P]),
            "g6x_sync": (I, [I]),
            "g6x_autotune": (I, [I, I, I, C.c_char_p]),
            "g6x_load_tuning": (I, [C.c_char_p]),
            "g6x_clear_tuning": (I, []), "g6x_set_variant": (I, [I, I, I]),
            "g6x_get_predicted": (I, [I, I, P, P, P, P, P]),
            "g6x_last_config": (I, [I, P, P, P, P, P, P]),
            "g6x_launch_count": (C.c_longlong, [I]),
            "g6x_set_wait_limit": (I, [D]),
            "g6x_probe_wait_timeout": (I, [I]),
            "g6x_set_timing": (I, [I, I]),
            "g6x_get_timing": (I, [I, P, P]),
            "g6h_correct_block": (I, [I, D, P, P, D, D, D, P, P, P, P, P, P, P]),
            "g6h_correct_block_ex": (I, [I, D, P, P, D, D, D, P, P, P, P, P, P, P, D]),
            "g6h_set_force_noise": (I, [P, D]),
            "g6hb_set_force_noise": (I, [P, D]),
            "g6x_fp32_probe": (I, [I, P, P]),
            "g6x_fp64_probe": (I, [I, P, P]),
            "g6x_variant_info": (I, [I, P]),
            "g6x_set_max_neighbours": (I, [I, I]),
            "g6x_max_neighbours": (I, [I]),
            "g6x_list_reruns": (C.c_longlong, [I]),
            "g6x_plan_launch": (I, [I, I, I, I, I, P]),
            "g6h_create": (P, [I, I, P, P, P, D, D, D, D, D, P]),
            "g6h_run": (I, [P, D]),
            "g6h_run_blocks": (C.c_longlong, [P, D, C.c_longlong]),
            "g6h_get_state": (I, [P, P, P, P, P, P, P]),
            "g6h_energy": (I, [P, P, P]),
            "g6h_stats": (I, [P, P, P, P]),
            "g6h_profile": (I, [P, P, P, P]),
            "g6h_destroy": (None, [P]),
            "g6h_checkpoint": (I, [P, C.c_char_p]),
            "g6h_set_neighbour_radius": (I, [P, D]),
            "g6h_neighbour_stats": (I, [P, P, P, P]),
            "g6h_restore": (P, [I, C.c_char_p, P]),
            "g6x_batch_create": (P, [I, P, I, I, I, P]),
            "g6x_batch_destroy": (I, [P]),
            "g6x_batch_irecs": (P, [P, I]),
            "g6x_batch_results": (P, [P, I]),
            "g6x_batch_set_j": (I, [P, I, I, I, D, D, P, P, P, P]),
            "g6x_batch_set_j_many": (I, [P, I, I, P, P, P, P, P, P, P, P]),
            "g6x_batch_calc": (I, [P, P, P, P, I]),
            "g6x_batch_launch_count": (C.c_longlong, [P]),
            "g6x_batch_set_schedule": (I, [P, I, I, I, I, I]),
            "g6x_batch_get_schedule": (I, [P, P]),
            "g6x_batch_autotune": (I, [P, I, P, P, P, I, P, P]),
            "g6hb_autotune": (I, [P, I, P, P]),
            "g6hb_set_schedule": (I, [P, I, I, I, I, I]),
            "g6x_batch_set_timing": (I, [P, I]),
            "g6x_batch_get_timing": (I, [P, P, P]),
            "g6hb_batch": (P, [P]),
            "g6hb_create": (P, [I, P, P, P, P, P, D, D, D, D, I, I, I, P]),
            "g6hb_step": (I, [P, D]),
            "g6hb_run": (I, [P, D]),
            "g6hb_set_mode": (I, [P, I]),
            "g6hb_stats": (I, [P, P, P, P, P, P]),
            "g6hb_get_state": (I, [P, P, P, P]),
            "g6hb_get_state_ex": (I, [P, P, P, P, P, P, P]),
            "g6hb_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc < 0:
        raise G6Error(rc, what)
    return rc


def strerror(code):
    return lib().g6x_strerror(int(code)).decode()


# ------------------------------------------------------------ GRAPE-6 API --

def g6_open(cid):
    return _check(lib().g6_open(cid), "g6_open")


def g6x_open_ex(cid, nj_max, ni_max):
    return _check(lib().g6x_open_ex(cid, int(nj_max), int(ni_max)), "g6x_open_ex")


def g6_close(cid):
    return _check(lib().g6_close(cid), "g6_close")


def g6_npipes():
    return lib().g6_npipes()


def g6_set_tunit(v):
    return lib().g6_set_tunit(int(v))


def g6_set_xunit(v):
    return lib().g6_set_xunit(int(v))


def g6_set_ti(cid, ti):
    return _check(lib().g6_set_ti(cid, float(ti)), "g6_set_ti")


def g6_set_j_particle(cid, address, index, tj, dtj, mass, k18, j6, a2, v, x):
    args = [_d(q, 3) for q in (k18, j6, a2, v, x)]
    return _check(lib().g6_set_j_particle(cid, int(address), int(index), float(tj),
                                          float(dtj), float(mass), *[_p(q) for q in args]),
                  "g6_set_j_particle")


def g6x_set_j_particles(cid, address, index, tj, mass, j6, a2, v, x):
    address, index = _i(address), _i(index)
    n = address.shape[0]
    tj = _d(np.broadcast_to(np.asarray(tj, dtype=np.float64), (n,)))
    mass = _d(np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,)))
    j6, a2, v, x = (_d(q, (n, 3)) for q in (j6, a2, v, x))
    return _check(lib().g6x_set_j_particles(cid, n, _p(address), _p(index), _p(tj), _p(mass),
                                            _p(j6), _p(a2), _p(v), _p(x)),
                  "g6x_set_j_particles")


def g6calc_firsthalf(cid, nj, ni, index, xi, vi, eps2, h2=None):
    index = _i(index)
    xi, vi = _d(xi, (ni, 3)), _d(vi, (ni, 3))
    h2 = None if h2 is None else _d(np.broadcast_to(np.asarray(h2, dtype=np.float64), (ni,)))
    # keep the marshalled arrays alive until the call returned (it copies them)
    lib().g6calc_firsthalf(cid, int(nj), int(ni), _p(index), _p(xi), _p(vi), None, None,
                           None, float(eps2), _p(h2))


def g6calc_lasthalf2(cid, nj, ni, eps2=0.0):
    """Returns (acc[ni,3], jerk[ni,3], pot[ni], nnbindex[ni])."""
    acc = np.empty((ni, 3))
    jerk = np.empty((ni, 3))
    pot = np.empty(ni)
    nnb = np.empty(ni, dtype=np.int32)
    _check(lib().g6calc_lasthalf2(cid, int(nj), int(ni), None, None, None, float(eps2), None,
                                  _p(acc), _p(jerk), _p(pot), _p(nnb)), "g6calc_lasthalf2")
    return acc, jerk, pot, nnb


def g6calc_lasthalf(cid, nj, ni, eps2=0.0):
    """Returns (acc[ni,3], jerk[ni,3], pot[ni])."""
    acc = np.empty((ni, 3))
    jerk = np.empty((ni, 3))
    pot = np.empty(ni)
    _check(lib().g6calc_lasthalf(cid, int(nj), int(ni), None, None, None, float(eps2), None,
                                 _p(acc), _p(jerk), _p(pot)), "g6calc_lasthalf")
    return acc, jerk, pot


def g6_read_neighbour_list(cid):
    return _check(lib().g6_read_neighbour_list(cid), "g6_read_neighbour_list")


def g6_get_neighbour_list(cid, ipipe, maxlength=None):
    """Returns (rc, nblen, list) where list holds min(nblen, maxlength, the
    context's list length) ids; maxlength defaults to that list length."""
    maxnb = g6x_max_neighbours(cid)
    maxlength = maxnb if maxlength is None else int(maxlength)
    nbl = np.empty(max(1, maxlength), dtype=np.int32)
    nblen = C.c_int(0)
    rc = _check(lib().g6_get_neighbour_list(cid, int(ipipe), int(maxlength), C.byref(nblen),
                                            _p(nbl)), "g6_get_neighbour_list")
    n = min(nblen.value, maxlength, maxnb)
    return rc, nblen.value, nbl[:n].copy()


# ------------------------------------------------------------- extensions --

def g6x_set_max_neighbours(cid, maxnb):
    return _check(lib().g6x_set_max_neighbours(cid, int(maxnb)), "g6x_set_max_neighbours")


def g6x_max_neighbours(cid):
    return _check(lib().g6x_max_neighbours(cid), "g6x_max_neighbours")


def g6x_list_reruns(cid):
    return lib().g6x_list_reruns(cid)

def g6x_set_precision(cid, mode):
    return _check(lib().g6x_set_precision(cid, int(mode)), "g6x_set_precision")


def g6x_set_ni_max(cid, ni_max):
    return _check(lib().g6x_set_ni_max(cid, int(ni_max)), "g6x_set_ni_max")


def g6x_set_stream(cid, stream_ptr):
    return _check(lib().g6x_set_stream(cid, C.c_void_p(int(stream_ptr) if stream_ptr else 0)),
                  "g6x_set_stream")


def g6x_set_variant(cid, variant=-1, grid=0):
    return _check(lib().g6x_set_variant(cid, int(variant), int(grid)), "g6x_set_variant")


def g6x_set_j_dev(cid, n, d_rec_ptr):
    return _check(lib().g6x_set_j_dev(cid, int(n), C.c_void_p(int(d_rec_ptr))),
                  "g6x_set_j_dev")


def g6x_calc_dev(cid, ti, nj, ni, d_irec_ptr, eps2, nl, d_out_ptr):
    return _check(lib().g6x_calc_dev(cid, float(ti), int(nj), int(ni),
                                     C.c_void_p(int(d_irec_ptr)), float(eps2), int(nl),
                                     C.c_void_p(int(d_out_ptr))), "g6x_calc_dev")


def g6x_calc_dev_noalloc(cid, ti, nj, ni, d_irec_ptr, eps2, d_out_ptr):
    """Allocation-free form of g6x_calc_dev (partial sums in a fixed static
    device array; ni <= G6X_NOALLOC_NI_MAX; no neighbour lists)."""
    return _check(lib().g6x_calc_dev_noalloc(cid, float(ti), int(nj), int(ni),
                                             C.c_void_p(int(d_irec_ptr)), float(eps2),
                                             C.c_void_p(int(d_out_ptr))),
                  "g6x_calc_dev_noalloc")


def g6x_autotune(cid, nj, m_max, path=None):
    return _check(lib().g6x_autotune(cid, int(nj), int(m_max),
                                     None if path is None else str(path).encode()),
                  "g6x_autotune")


def g6x_load_tuning(path):
    return _check(lib().g6x_load_tuning(str(path).encode()), "g6x_load_tuning")


def g6x_clear_tuning():
    return lib().g6x_clear_tuning()


def g6x_sync(cid):
    return _check(lib().g6x_sync(cid), "g6x_sync")


def g6x_get_predicted(cid, nj, fp64=False):
    """DS mode: (hi[nj,4], lo[nj,4], vel[nj,4]) float32; FP64 mode: (x[nj,4], v[nj,4])."""
    if fp64:
        x = np.empty((nj, 4))
        v = np.empty((nj, 4))
        _check(lib().g6x_get_predicted(cid, int(nj), None, None, None, _p(x), _p(v)),
               "g6x_get_predicted")
        return x, v
    hi = np.empty((nj, 4), dtype=np.float32)
    lo = np.empty((nj, 4), dtype=np.float32)
    vel = np.empty((nj, 4), dtype=np.float32)
    _check(lib().g6x_get_predicted(cid, int(nj), _p(hi), _p(lo), _p(vel), None, None),
           "g6x_get_predicted")
    return hi, lo, vel


def g6x_last_config(cid):
    vals = [C.c_int(0) for _ in range(6)]
    _check(lib().g6x_last_config(cid, *[C.byref(v) for v in vals]), "g6x_last_config")
    return dict(zip(("variant", "ti", "tj", "ni_per", "grid", "jtiles"),
                    [v.value for v in vals]))


def g6x_launch_count(cid):
    return lib().g6x_launch_count(cid)


def g6x_set_wait_limit(seconds):
    return _check(lib().g6x_set_wait_limit(float(seconds)), "g6x_set_wait_limit")


def g6x_probe_wait_timeout(cid):
    """Code reported by one bounded wait that nothing completes (G6_ETIMEDOUT
    when the timeout path works)."""
    return lib().g6x_probe_wait_timeout(cid)


def g6x_plan_launch(mode, nj, ni, list_=False, sm_count=152):
    """The launch a calculation would get (no GPU needed): dict with variant,
    ti, tj, ni_per, grid, jtiles."""
    out = np.zeros(6, dtype=np.int32)
    _check(lib().g6x_plan_launch(int(mode), int(nj), int(ni), int(bool(list_)), int(sm_count),
                                 out.ctypes.data_as(C.c_void_p)), "g6x_plan_launch")
    return dict(zip(("variant", "ti", "tj", "ni_per", "grid", "jtiles"), (int(v) for v in out)))


def g6x_variant_info(variant):
    """Shape of a compiled force-kernel variant: dict with ti, tj, ni_per,
    list, prec, fpred, twin, ws."""
    out = np.zeros(8, dtype=np.int32)
    _check(lib().g6x_variant_info(int(variant), out.ctypes.data_as(C.c_void_p)),
           "g6x_variant_info")
    return dict(zip(("ti", "tj", "ni_per", "list", "prec", "fpred", "twin", "ws"),
                    (int(v) for v in out)))


def g6x_variant_count():
    return _check(lib().g6x_variant_info(-1, None), "g6x_variant_info")


def g6x_fp32_probe(iters=10000):
    """Measured packed-FP32 FMA rate of the current device: (TFLOP/s, ms of
    the timed launch)."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib().g6x_fp32_probe(int(iters), C.byref(tf), C.byref(ms)), "g6x_fp32_probe")
    return tf.value, ms.value


def g6x_fp64_probe(iters=200):
    """Measured FP64 FMA rate of the current device: (TFLOP/s, ms of the
    timed launch)."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib().g6x_fp64_probe(int(iters), C.byref(tf), C.byref(ms)), "g6x_fp64_probe")
    return tf.value, ms.value


def g6x_set_timing(cid, enable=True):
    return _check(lib().g6x_set_timing(cid, int(bool(enable))), "g6x_set_timing")


def g6x_get_timing(cid):
    """Returns (ms[4], count[4]) for scatter, predictor, force, reduction."""
    ms = np.zeros(4)
    cnt = np.zeros(4, dtype=np.int64)
    _check(lib().g6x_get_timing(cid, _p(ms), _p(cnt)), "g6x_get_timing")
    return ms, cnt


_torch_hooks = None


def g6x_use_torch_allocator():
    """Route every later g6_open's device allocations through PyTorch's
    caching allocator (torch.cuda.caching_allocator_alloc/delete)."""
    global _torch_hooks
    import torch

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib().g6x_set_allocator(hooks[0], hooks[1], None), "g6x_set_allocator")
    _torch_hooks = hooks


def g6x_use_cuda_allocator():
    global _torch_hooks
    _check(lib().g6x_set_allocator(ALLOC_FN(), FREE_FN(), None), "g6x_set_allocator")
    _torch_hooks = None


# --------------------------------------------------------- Hermite driver --

def g6h_correct_block(t_blk, t0, dt, eta, dt_max, dt_min, xp, vp, a0, j0, a1, j1,
                      force_noise=0.0):
    """Host Hermite corrector + next step for a block (C++).  Returns
    (x1, v1, dt_new, n_too_small); xp and vp are not modified.  force_noise:
    the relative force error the time-step choice allows for (0: none)."""
    xp = _d(xp).reshape(-1, 3).copy()
    vp = _d(vp).reshape(-1, 3).copy()
    n = xp.shape[0]
    t0 = _d(np.broadcast_to(np.asarray(t0, dtype=np.float64), (n,)))
    dt = _d(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
    a0, j0, a1, j1 = (_d(q, (n, 3)) for q in (a0, j0, a1, j1))
    dt_new = np.empty(n)
    rc = _check(lib().g6h_correct_block_ex(n, float(t_blk), _p(t0), _p(dt), float(eta),
                                           float(dt_max), float(dt_min), _p(xp), _p(vp),
                                           _p(a0), _p(j0), _p(a1), _p(j1), _p(dt_new),
                                           float(force_noise)),
                "g6h_correct_block_ex")
    return xp, vp, dt_new, rc


class G6HSim:
    """Owner of a g6h_sim handle (the C++ Hermite block-time-step driver)."""

    def __init__(self, cid, m, x, v, eps2, eta, eta_s=0.0, dt_max=2.0 ** -4,
                 dt_min=2.0 ** -40):
        m = _d(m).reshape(-1)
        n = m.shape[0]
        x, v = _d(x, (n, 3)), _d(v, (n, 3))
        err = C.c_int(0)
        h = lib().g6h_create(cid, n, _p(m), _p(x), _p(v), float(eps2), float(eta),
                             float(eta_s), float(dt_max), float(dt_min), C.byref(err))
        if not h:
            raise G6Error(err.value or G6_EINVAL, "g6h_create")
        self.h = h
        self.n = n

    def run(self, t_end):
        return _check(lib().g6h_run(self.h, float(t_end)), "g6h_run")

    def set_force_noise(self, rel):
        return _check(lib().g6h_set_force_noise(self.h, float(rel)), "g6h_set_force_noise")

    def set_neighbour_radius(self, h2):
        return _check(lib().g6h_set_neighbour_radius(self.h, float(h2)),
                      "g6h_set_neighbour_radius")

    def neighbour_stats(self):
        v = [C.c_longlong(0) for _ in range(3)]
        _check(lib().g6h_neighbour_stats(self.h, *[C.byref(a) for a in v]),
               "g6h_neighbour_stats")
        return dict(lists=v[0].value, entries=v[1].value, overflowed=v[2].value)

    def run_blocks(self, t_end, max_blocks):
        """Advance at most max_blocks block steps toward t_end; returns the
        number taken."""
        r = lib().g6h_run_blocks(self.h, float(t_end), int(max_blocks))
        if r < 0:
            raise G6Error(int(r), "g6h_run_blocks")
        return int(r)

    def checkpoint(self, path):
        return _check(lib().g6h_checkpoint(self.h, os.fsencode(path)), "g6h_checkpoint")

    @classmethod
    def restore(cls, cid, path):
        """A driver rebuilt from a checkpoint on the opened cluster id cid."""
        err = C.c_int(0)
        h = lib().g6h_restore(cid, os.fsencode(path), C.byref(err))
        if not h:
            raise G6Error(err.value or G6_EINVAL, "g6h_restore")
        obj = cls.__new__(cls)
        obj.h = h
        obj.n = int(np.fromfile(path, dtype="<i8", count=2, offset=8)[0])
        return obj

    def state(self):
        n = self.n
        x, v, a, j = (np.empty((n, 3)) for _ in range(4))
        t, dt = np.empty(n), np.empty(n)
        _check(lib().g6h_get_state(self.h, _p(x), _p(v), _p(a), _p(j), _p(t), _p(dt)),
               "g6h_get_state")
        return dict(x=x, v=v, acc=a, jerk=j, t=t, dt=dt)

    def energy(self):
        ek, ep = C.c_double(0), C.c_double(0)
        _check(lib().g6h_energy(self.h, C.byref(ek), C.byref(ep)), "g6h_energy")
        return ek.value, ep.value

    def stats(self):
        nb, na = C.c_longlong(0), C.c_longlong(0)
        hist = np.zeros(64, dtype=np.int64)
        _check(lib().g6h_stats(self.h, C.byref(nb), C.byref(na), _p(hist)), "g6h_stats")
        return dict(nblocks=nb.value, nactive=na.value, hist=hist)

    def profile(self):
        """Seconds in (scheduler, force calls, correction) during run()."""
        a, b, c = C.c_double(0), C.c_double(0), C.c_double(0)
        _check(lib().g6h_profile(self.h, C.byref(a), C.byref(b), C.byref(c)), "g6h_profile")
        return dict(sched_s=a.value, force_s=b.value, correct_s=c.value)

    def close(self):
        if self.h:
            lib().g6h_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _mapped(ptr, dtype, n):
    """numpy view of n records of dtype at a host address (mapped memory)."""
    buf = (C.c_char * (n * dtype.itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=dtype, count=n)


class G6Batch:
    """Owner of a g6x_batch: ncl independent clusters computed together."""

    def __init__(self, nj, precision=G6X_PREC_DS, variant=-1, grid_mul=0):
        nj = _i(nj).reshape(-1)
        err = C.c_int(0)
        h = lib().g6x_batch_create(len(nj), _p(nj), precision, variant, grid_mul, C.byref(err))
        if not h:
            raise G6Error(err.value or G6_EINVAL, "g6x_batch_create")
        self.h = h
        self.nj = nj
        self.ncl = len(nj)

    def irecs(self, cl):
        """Writable IREC view of cluster cl's i-records (mapped memory)."""
        return _mapped(lib().g6x_batch_irecs(self.h, cl), IREC, int(self.nj[cl]))

    def results(self, cl, ni):
        """Copy of cluster cl's first ni results."""
        return _mapped(lib().g6x_batch_results(self.h, cl), OUT, int(self.nj[cl]))[:ni].copy()

    def set_j(self, cl, m, x, v, a2=None, j6=None, tj=0.0, addr=None):
        """Stage particles of cluster cl: addresses addr (default all nj[cl]),
        index = address; a2 = a/2 and j6 = j/6 pre-scaled; tj scalar or per
        particle."""
        addr = np.arange(int(self.nj[cl])) if addr is None else np.asarray(addr).reshape(-1)
        n = len(addr)
        m = _d(m).reshape(-1)
        x, v = _d(x, (n, 3)), _d(v, (n, 3))
        a2 = np.zeros((n, 3)) if a2 is None else _d(a2, (n, 3))
        j6 = np.zeros((n, 3)) if j6 is None else _d(j6, (n, 3))
        tj = _d(np.broadcast_to(np.asarray(tj, dtype=np.float64), (n,)))
        addr = _i(addr)
        _check(lib().g6x_batch_set_j_many(self.h, cl, n, _p(addr), _p(addr), _p(tj), _p(m),
                                          _p(j6), _p(a2), _p(v), _p(x)),
               "g6x_batch_set_j_many")

    def set_i(self, cl, x, v, index=None):
        n = len(x)
        r = self.irecs(cl)
        r["x"][:n] = x
        r["v"][:n] = v
        r["h2"][:n] = 0.0
        r["index"][:n] = np.arange(n) if index is None else index
        r["pad"][:n] = 0

    def calc(self, t_blk, eps2, ni, mode=0):
        t_blk, eps2, ni = _d(t_blk), _d(eps2), _i(ni)
        return _check(lib().g6x_batch_calc(self.h, _p(t_blk), _p(eps2), _p(ni), int(mode)),
                      "g6x_batch_calc")

    def launch_count(self):
        return lib().g6x_batch_launch_count(self.h)

    def set_timing(self, on=True):
        return _check(lib().g6x_batch_set_timing(self.h, int(on)), "g6x_batch_set_timing")

    def timing(self):
        ms, n = C.c_double(0), C.c_longlong(0)
        _check(lib().g6x_batch_get_timing(self.h, C.byref(ms), C.byref(n)),
               "g6x_batch_get_timing")
        return ms.value, n.value

    def set_schedule(self, small_variant, small_grid_mul=1, threshold=0, large_variant=-1,
                     large_grid_mul=1):
        return _check(lib().g6x_batch_set_schedule(self.h, small_variant, small_grid_mul,
                                                   threshold, large_variant, large_grid_mul),
                      "g6x_batch_set_schedule")

    def schedule(self):
        s = np.zeros(5, dtype=np.int32)
        _check(lib().g6x_batch_get_schedule(self.h, _p(s)), "g6x_batch_get_schedule")
        return tuple(int(v) for v in s)

    def autotune(self, patterns, eps2, t_blk, reps=2):
        """Tune the schedule on active-set patterns [npat][ncl]; returns
        (schedule, mean ms per call)."""
        pat = _i(patterns).reshape(-1, self.ncl)
        s = np.zeros(5, dtype=np.int32)
        ms = C.c_double(0)
        _check(lib().g6x_batch_autotune(self.h, pat.shape[0], _p(pat), _p(_d(eps2)),
                                        _p(_d(t_blk)), int(reps), _p(s), C.byref(ms)),
               "g6x_batch_autotune")
        return tuple(int(v) for v in s), ms.value

    def close(self):
        if self.h:
            lib().g6x_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class G6HBatchSim:
    """Owner of a g6hb_sim: the Hermite driver over a batch of clusters."""

    def __init__(self, clusters, eps2, eta, eta_s=0.0, dt_max=2.0 ** -4, dt_min=2.0 ** -40,
                 variant=-1, grid_mul=0, mode=0):
        n = _i([len(c[0]) for c in clusters])
        m = _d(np.concatenate([c[0] for c in clusters]))
        x = _d(np.concatenate([c[1] for c in clusters]))
        v = _d(np.concatenate([c[2] for c in clusters]))
        eps2 = _d(np.broadcast_to(np.asarray(eps2, dtype=np.float64), (len(n),)))
        err = C.c_int(0)
        h = lib().g6hb_create(len(n), _p(n), _p(m), _p(x), _p(v), _p(eps2), float(eta),
                              float(eta_s), float(dt_max), float(dt_min), int(variant),
                              int(grid_mul), int(mode), C.byref(err))
        if not h:
            raise G6Error(err.value or G6_EINVAL, "g6hb_create")
        self.h = h
        self.n = n
        self.off = np.concatenate([[0], np.cumsum(n)])

    def step(self, t_end):
        return _check(lib().g6hb_step(self.h, float(t_end)), "g6hb_step")

    def run(self, t_end):
        return _check(lib().g6hb_run(self.h, float(t_end)), "g6hb_run")

    def set_mode(self, mode):
        return _check(lib().g6hb_set_mode(self.h, int(mode)), "g6hb_set_mode")

    def set_force_noise(self, rel):
        return _check(lib().g6hb_set_force_noise(self.h, float(rel)), "g6hb_set_force_noise")

    def autotune(self, reps=2):
        s = np.zeros(5, dtype=np.int32)
        ms = C.c_double(0)
        _check(lib().g6hb_autotune(self.h, int(reps), _p(s), C.byref(ms)), "g6hb_autotune")
        return tuple(int(v) for v in s), ms.value

    def set_schedule(self, sched):
        return _check(lib().g6hb_set_schedule(self.h, *[int(v) for v in sched]),
                      "g6hb_set_schedule")

    def set_timing(self, on=True):
        return _check(lib().g6x_batch_set_timing(lib().g6hb_batch(self.h), int(on)),
                      "g6x_batch_set_timing")

    def timing(self):
        """(GPU milliseconds summed over batch calls, calls) since set_timing."""
        ms, n = C.c_double(0), C.c_longlong(0)
        _check(lib().g6x_batch_get_timing(lib().g6hb_batch(self.h), C.byref(ms), C.byref(n)),
               "g6x_batch_get_timing")
        return ms.value, n.value

    def stats(self):
        v = [C.c_longlong(0) for _ in range(3)] + [C.c_double(0), C.c_double(0)]
        _check(lib().g6hb_stats(self.h, *[C.byref(a) for a in v]), "g6hb_stats")
        return dict(nsteps=v[0].value, nactive=v[1].value, interactions=v[2].value,
                    sec_gpu=v[3].value, sec_host=v[4].value)

    def state(self):
        tot = int(self.off[-1])
        x, v, t = np.empty((tot, 3)), np.empty((tot, 3)), np.empty(tot)
        _check(lib().g6hb_get_state(self.h, _p(x), _p(v), _p(t)), "g6hb_get_state")
        return dict(x=x, v=v, t=t)

    def full_state(self):
        """x, v, acc, jerk [sum n, 3]; t, dt [sum n]: each particle at its own
        last block time, next due at t + dt."""
        tot = int(self.off[-1])
        x, v, a, j = (np.empty((tot, 3)) for _ in range(4))
        t, dt = np.empty(tot), np.empty(tot)
        _check(lib().g6hb_get_state_ex(self.h, _p(x), _p(v), _p(a), _p(j), _p(t), _p(dt)),
               "g6hb_get_state_ex")
        return dict(x=x, v=v, acc=a, jerk=j, t=t, dt=dt)

    def close(self):
        if self.h:
            lib().g6hb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
