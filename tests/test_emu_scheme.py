"""Host model of the FP64-accurate tensor-core product's arithmetic (exact
operand splitting into digit slices; Ozaki, Ogita, Oishi and Rump, Numer.
Algorithms 59, 2012), checked against exact rational arithmetic.

The model follows the kernels' integer steps: a row frame 2^E with E = 1 +
the largest floor(log2|x|) of the row (subnormals included), X =
floor(|x| 2^(60-E)) split into ten signed 6-bit digits; per order d = p + q
an FP32 accumulator of the digit products over K (exact while below 2^24);
the ten accumulators combined as hi = V_0 2^12 + V_1 2^6 + V_2 and
lo = sum_{g>=3} V_g 2^(6(9-g)) in 64-bit integers.  It pins the design
constants (slices, bits, the 512-long exact pass, the integer ranges) and
the error bound the GPU tests use; the CUDA kernel itself is checked on the
device by tests/test_gpu_emu_gemm.py.
"""
import math
import struct
from fractions import Fraction

import numpy as np

BETA, SLICES, KCHUNK = 6, 10, 512
F = BETA * SLICES


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _lead(x):
    b = _bits(x)
    ef = (b >> 52) & 0x7FF
    if ef:
        return ef - 1023
    m = b & ((1 << 52) - 1)
    return -1074 + m.bit_length() - 1 if m else None


def _frame(row):
    leads = [l for l in (_lead(x) for x in row) if l is not None]
    return max(leads) + 1 if leads else 0


def _digits(x, E):
    b = _bits(x)
    ef = (b >> 52) & 0x7FF
    m = b & ((1 << 52) - 1)
    q = -1074
    if ef:
        m |= 1 << 52
        q = ef - 1075
    sh = q + F - E
    X = m << sh if sh >= 0 else (0 if sh <= -64 else m >> -sh)
    assert X < (1 << F)
    s = -1 if b >> 63 else 1
    return [s * ((X >> (F - BETA * p)) & 63) for p in range(1, SLICES + 1)]


def _f32_sum(terms):
    acc = np.float32(0.0)
    for t in terms:
        acc = np.float32(acc + np.float32(t))
    return acc


def _emulated_product(A, B):
    M, K = A.shape
    N = B.shape[0]
    EA = [_frame(r) for r in A]
    EB = [_frame(r) for r in B]
    DA = [[_digits(x, EA[i]) for x in A[i]] for i in range(M)]
    DB = [[_digits(x, EB[j]) for x in B[j]] for j in range(N)]
    C = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            V = []
            for g in range(SLICES):          # order d = g + 2
                terms = []
                for k0 in range(0, K, 16):   # one MMA of 16 products per slice pair
                    for p in range(g + 1):
                        qq = g - p
                        terms.append(sum(DA[i][k][p] * DB[j][k][qq]
                                         for k in range(k0, min(K, k0 + 16))))
                V.append(int(_f32_sum(terms)))
            hi = V[0] * 4096 + V[1] * 64 + V[2]
            lo = sum(V[g] * (1 << (BETA * (SLICES - 1 - g))) for g in range(3, SLICES))
            assert abs(hi) < 2 ** 40 and abs(lo) < 2 ** 62
            lo_unit = 2.0 ** (-BETA * (SLICES - 1))
            # one rounding, like the kernel's fma(hi, 2^-12, (double)lo * 2^-54)
            s = float(Fraction(hi) * Fraction(2) ** -12 + Fraction(float(lo) * lo_unit))
            C[i, j] = math.ldexp(s, EA[i] + EB[j] - 2 * BETA)
    return C


def test_digit_frames_reconstruct_to_60_bits():
    rng = np.random.default_rng(0)
    rows = [rng.standard_normal(9) * 10.0 ** rng.uniform(-300, 300, size=9),
            np.array([5e-324, -1e-320, 3e-310, 0.0, 2e-315]),
            np.zeros(4),
            rng.standard_normal(7)]
    for row in rows:
        E = _frame(row)
        for x in row:
            if x != 0:
                assert abs(x) < 2.0 ** E
            d = _digits(x, E)
            assert all(abs(v) <= 63 for v in d)
            val = sum(Fraction(v) * Fraction(2) ** (-BETA * (p + 1)) for p, v in enumerate(d))
            assert abs(Fraction(float(x)) - val * Fraction(2) ** E) < Fraction(2) ** (E - F)


def test_accumulators_exact_up_to_order_nine():
    # order d = g + 2 sums g + 1 slice pairs; up to eight terms of K products
    # of 6-bit digits stay below 2^24 for K <= 512 (exact in FP32)
    for g in range(SLICES):
        terms = g + 1                      # slice pairs p + q = g
        bound = terms * KCHUNK * 63 * 63
        if g + 2 <= 9:
            assert bound < 2 ** 24
        else:                              # orders 10 and 11: below 2^25
            assert bound < 2 ** 25
    # the epilogue's integer combination stays inside 64 bits
    lo_max = sum((2 ** 25) * (1 << (BETA * (SLICES - 1 - g))) for g in range(3, SLICES))
    assert lo_max < 2 ** 62


def test_emulated_product_within_bound_of_exact():
    rng = np.random.default_rng(4)
    M, N, K = 5, 4, 40
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-50, 50, size=(M, 1))
    B = rng.standard_normal((N, K)) * 10.0 ** rng.uniform(-50, 50, size=(N, 1))
    A[1, : K // 2] = A[1, K // 2:]                 # exact cancellation against B[2]
    B[2, K // 2:] = -B[2, : K // 2]
    C = _emulated_product(A, B)
    for i in range(M):
        for j in range(N):
            exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i], B[j]))
            err = abs(Fraction(float(C[i, j])) - exact)
            bound = Fraction(K) * Fraction(2) ** -52 * Fraction(float(np.abs(A[i]).max())) \
                * Fraction(float(np.abs(B[j]).max())) + Fraction(2) ** -51 * abs(exact)
            assert err <= bound
    assert C[1, 2] == 0.0


def test_truncation_is_what_limits_accuracy():
    """On a product with cancellation ten slices are at least as accurate as
    nine and within the FP64-level bound; the truncation after the last slice
    is the scheme's only approximation besides the final FP64 rounding."""
    global SLICES, F
    rng = np.random.default_rng(9)
    A = rng.standard_normal((3, 64))
    B = rng.standard_normal((3, 64))
    B -= np.outer((B @ A[0]) / (A[0] @ A[0]), A[0])   # rows of B orthogonal to A[0]
    exact = [sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[0], B[j])) for j in range(3)]
    errs = {}
    saved = SLICES, F
    try:
        for s in (9, 10):
            SLICES, F = s, BETA * s
            C = _emulated_product(A[:1], B)
            errs[s] = max(float(abs(Fraction(float(C[0, j])) - exact[j])) for j in range(3))
    finally:
        SLICES, F = saved
    assert errs[10] <= errs[9]
    assert errs[10] <= 64 * 2.0 ** -52 * np.abs(A[0]).max() * np.abs(B).max()
