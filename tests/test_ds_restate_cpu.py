"""The float32 restatement used by the bit-exact GPU pins, checked on the
CPU: its fused multiply-add against exact rational arithmetic (one rounding,
ties to even), and its DS + SP addition against the exact sum (the pair
holds hi + lo + d to within the DS rounding, and hi is the float nearest the
pair's value)."""
from fractions import Fraction

import numpy as np

from tests.ds_restate import ds_plus_sp, ds_split, f32, fma32


def test_fma32_restatement_against_exact_rationals():
    # the fused multiply-add emulation against exact rational arithmetic,
    # including operands built to land the double sum halfway between floats
    from fractions import Fraction
    rng = np.random.default_rng(5)
    a = rng.normal(size=4000).astype(f32)
    b = rng.normal(size=4000).astype(f32)
    c = rng.normal(size=4000).astype(f32)
    # halfway cases: c = -(a b) rounded, plus a tiny remainder
    c[:500] = (-(a[:500].astype(np.float64) * b[:500])).astype(f32)
    got = fma32(a, b, c)
    for k in range(a.size):
        exact = Fraction(float(a[k])) * Fraction(float(b[k])) + Fraction(float(c[k]))
        cand = [np.nextafter(got[k], f32(-np.inf)), got[k], np.nextafter(got[k], f32(np.inf))]
        errs = [abs(Fraction(float(x)) - exact) for x in cand]
        assert errs[1] <= min(errs), k
        if errs[1] == min(errs[0], errs[2]):           # a tie: even mantissa
            assert int(got[k].view(np.int32)) % 2 == 0, k


def test_ds_plus_sp_against_exact_sums():
    rng = np.random.default_rng(9)
    x = rng.uniform(-10, 10, size=3000)
    d = (rng.normal(size=3000) * 10.0 ** rng.uniform(-8, 0, size=3000)).astype(f32)
    hi, lo = ds_split(x)
    rh, rl = ds_plus_sp(hi, lo, d)
    for k in range(x.size):
        exact = Fraction(float(hi[k])) + Fraction(float(lo[k])) + Fraction(float(d[k]))
        got = Fraction(float(rh[k])) + Fraction(float(rl[k]))
        # DS keeps about 48 bits: error within 2^-44 of the magnitude
        assert abs(got - exact) <= Fraction(2) ** -44 * abs(exact) + Fraction(2) ** -140
        assert abs(float(rl[k])) <= 0.5 * float(np.spacing(abs(rh[k]))) + 1e-300
