"""CPU restatement, in numpy float32, of the library's single-precision and
double-single arithmetic (Sect. 2.2 predictor, Sect. 2.3 separations), used by
the bit-exact GPU pins.  Every operation rounds to nearest, as the GPU's do;
nothing here calls the library or the oracle."""
import numpy as np

f32 = np.float32


def rn32(x):
    """The float nearest a double (ties to even)."""
    return np.asarray(x, dtype=np.float64).astype(f32)


def fma32(a, b, c):
    """Single-precision fused multiply-add a * b + c with one rounding.  The
    product of two floats is exact in double; the double sum of it and c is
    exact unless its TwoSum error is non-zero, and then rounding the double
    sum to float is still the single rounding of the exact value unless the
    double sum sits exactly halfway between two floats -- in that case the
    sign of the error decides."""
    a64, b64, c64 = (np.asarray(v, dtype=f32).astype(np.float64) for v in (a, b, c))
    p = a64 * b64
    s = p + c64
    bb = s - p
    err = (p - (s - bb)) + (c64 - bb)
    r = s.astype(f32)
    rf = r.astype(np.float64)
    d = s - rf
    toward = np.where(d > 0, np.inf, -np.inf).astype(f32)
    rn = np.nextafter(r, toward)
    mid = (d != 0) & (2.0 * s == rf + rn.astype(np.float64)) & (err != 0)
    beyond = np.sign(err) == np.sign(d)
    return np.where(mid & beyond, rn, r)


def two_sum32(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def ds_plus_sp(hi, lo, d):
    """DS + SP addition: (hi, lo) + d in ten single-precision operations."""
    s, e = two_sum32(hi, d)
    e = e + lo
    rh = s + e
    rl = e - (rh - s)
    return rh, rl


def ds_split(x):
    hi = rn32(x)
    lo = rn32(np.asarray(x, dtype=np.float64) - hi.astype(np.float64))
    return hi, lo


def restated_prediction(st, t_blk, x64_add=False):
    """Eq. 1 and Eq. 2 in the library's single-precision form, from the data
    the library stores (doubles rounded to float once on the device)."""
    xh, xl = ds_split(st["x0"])
    v = rn32(st["v0"])
    a2 = rn32(st["a0"] / 2.0)
    j6 = rn32(st["j0"] / 6.0)
    h = rn32(t_blk - st["tj"])[:, None] * np.ones((1, 3), dtype=f32)
    inc = h * fma32(h, fma32(h, j6, a2), v)
    if x64_add:
        px = st["x0"] + inc.astype(np.float64)
        hi, lo = ds_split(px)
    else:
        hi, lo = ds_plus_sp(xh, xl, inc)
    vel = fma32(h, fma32(f32(3.0) * h, j6, f32(2.0) * a2), v)
    return hi, lo, vel
