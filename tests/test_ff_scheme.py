"""Host model of the double-FP32 product's arithmetic (gemm_ff.cu,
ff_arith.cuh), checked against exact rational arithmetic.

The model takes the kernels' steps in FP32 (numpy float32 scalars round to
nearest, like the CUDA intrinsics): each FP64 operand cut by its bit pattern
into hi (leading 24 significand bits) and lo (the next 29, rounded to 24);
per term the exact product of the leading parts as p + e (TwoProduct), p
added to the running sum s by TwoSum, its error, e and the cross terms
ah*bl + al*bh added to c (Dot2 of Ogita, Rump and Oishi); the row kernel
renormalises (s, c) every 32 terms, the long-k kernel restarts (s, c) every
32 terms and adds each run into (S, C) by float-float addition.  It pins
the stated error bound (3e-11 of sum |a b|) and the split's properties; the
CUDA kernels themselves are checked on the device by tests/test_gpu_ffgemm.py.
"""
import struct
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32
BOUND = 3e-11


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def split(x):
    """hi + lo from the bit pattern of x, as the device's ff_split."""
    b = _bits(x)
    sgn = -1.0 if b >> 63 else 1.0
    e = ((b >> 52) & 0x7FF) - 1023
    f = b & ((1 << 52) - 1)
    if e < -126:
        return f32(0.0), f32(0.0)
    if e > 127:
        return f32(sgn * np.inf), f32(0.0)
    hi = f32(sgn * (1 + (f >> 29) / 2.0**23) * 2.0**e)
    r = f & ((1 << 29) - 1)
    if r == 0 or e < -74:
        return hi, f32(0.0)
    lo = f32(sgn * float(f32(r)) * 2.0 ** (e - 52))
    return hi, lo


def two_prod(a, b):
    p = f32(a * b)
    e = f32(float(a) * float(b) - float(p))  # exact in FP64, and exactly an FP32 number
    return p, e


def two_sum(s, p):
    t = f32(s + p)
    z = f32(t - s)
    q = f32(f32(s - f32(t - z)) + f32(p - z))
    return t, q


def term(ah, al, bh, bl, s, c):
    p, e = two_prod(ah, bh)
    t, q = two_sum(s, p)
    # fma(ah, bl, fma(al, bh, e)): each product exact in FP64, one rounding to FP32
    inner = f32(float(al) * float(bh) + float(e))
    cross = f32(float(ah) * float(bl) + float(inner))
    return t, f32(c + f32(q + cross))


def ff_add(S, C, s, c):
    t, q = two_sum(S, s)
    return t, f32(C + f32(q + c))


def dot_rows(a, b):
    """Row kernel: one (s, c), renormalised every 32 terms."""
    s = c = f32(0.0)
    for k, (x, y) in enumerate(zip(a, b)):
        ah, al = split(x)
        bh, bl = split(y)
        s, c = term(ah, al, bh, bl, s, c)
        if k % 32 == 31:
            s, c = two_sum(s, c)  # the new c is the exact remainder
    return float(s) + float(c)


def dot_long(a, b):
    """Long-k kernel: runs of 32 from zero, added into (S, C)."""
    S = C = f32(0.0)
    for k0 in range(0, len(a), 32):
        s = c = f32(0.0)
        for x, y in zip(a[k0:k0 + 32], b[k0:k0 + 32]):
            ah, al = split(x)
            bh, bl = split(y)
            s, c = term(ah, al, bh, bl, s, c)
        S, C = ff_add(S, C, s, c)
    return float(S) + float(C)


def exact(a, b):
    return sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))


def test_split_properties():
    rng = np.random.default_rng(0)
    xs = rng.standard_normal(4000) * 10.0 ** rng.uniform(-30, 30, 4000)
    for x in xs:
        hi, lo = split(x)
        err = abs(Fraction(float(x)) - Fraction(float(hi)) - Fraction(float(lo)))
        if abs(x) >= 2.0**-74:
            assert err <= Fraction(2) ** -47 * abs(Fraction(float(x)))
        else:  # lo below the FP32 normal range is dropped
            assert lo == 0.0 and err < Fraction(2) ** -97
        assert abs(float(x) - float(hi)) < 2.0**-23 * abs(x)  # leading 24 bits
    # flush below the FP32 normal range, infinities above it
    assert split(1e-39) == (0.0, 0.0)
    assert np.isinf(split(1e39)[0])
    assert split(-0.0) == (0.0, 0.0)


def test_two_prod_is_exact():
    rng = np.random.default_rng(1)
    for a, b in rng.standard_normal((500, 2)).astype(np.float32):
        p, e = two_prod(a, b)
        assert Fraction(float(p)) + Fraction(float(e)) == Fraction(float(a)) * Fraction(float(b))


@pytest.mark.parametrize("kind", ["rows", "long"])
@pytest.mark.parametrize("k,scale,seed", [(256, 0, 0), (200, 8, 1), (97, 0, 2)])
def test_dot_within_bound(kind, k, scale, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(k) * 10.0 ** rng.uniform(-scale, scale, k)
    b = rng.standard_normal(k) * 10.0 ** rng.uniform(-scale, scale, k)
    got = (dot_rows if kind == "rows" else dot_long)(a, b)
    ref = exact(a, b)
    s = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(a, b))
    err = abs(Fraction(got) - ref)
    assert err <= Fraction(BOUND) * s
    assert float(err / s) <= 1e-13  # random operands: near FP64 level


def test_compensation_carries_cancellation():
    """Large terms that cancel leave the small ones: a plain FP32 sum loses
    them, the compensated pair keeps them to about 2^-46 of sum |a b|."""
    rng = np.random.default_rng(3)
    big = rng.standard_normal(64) * 1e4
    small = rng.standard_normal(64) * 1e-4
    a = np.concatenate([big, -big, small])
    b = np.ones_like(a)
    ref = float(exact(a, b))
    naive = float(np.sum(a.astype(np.float32), dtype=np.float32))
    for got in (dot_long(a, b), dot_rows(a, b)):
        assert abs(got - ref) <= 3e-11 * np.sum(np.abs(a))
        assert abs(got - ref) <= 1e-8
    assert abs(naive - ref) > 1e-5
