"""Host model of the subspace eigensolver's FP64 Sturm count (la.cu,
sturm_count_minors): the number of eigenvalues of a symmetric tridiagonal T
below x from the signs of its leading principal minors
p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}, a zero minor counted as a sign
change, the pair (p_{i-1}, p_i) rescaled by a power of two when the larger
leaves [2^-500, 2^500].  Checked against LAPACK's eigenvalues on random
tridiagonals, including ranges that force the rescaling; the device code is
checked by tests/test_gpu_la.py and every Davidson test.
"""
import struct

import numpy as np


def _bits(v):
    return struct.unpack("<q", struct.pack("<d", float(v)))[0]


def _dexp(v):
    return (_bits(v) >> 52) & 0x7FF


def _from_bits(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def count_minors(d, e2, x):
    p0, p1 = 1.0, d[0] - x
    if _dexp(p1) == 0:
        p1 = -1e-300
    c = 1 if _bits(p1) < 0 else 0
    for i in range(1, len(d)):
        p2 = (d[i] - x) * p1 - e2[i - 1] * p0
        b1 = _bits(p1)
        if _dexp(p2) == 0:
            p2 = 1e-300 if b1 < 0 else -1e-300
        c += (_bits(p2) < 0) != (b1 < 0)
        ex = max(_dexp(p1), _dexp(p2))
        if ex > 1023 + 500 or ex < 1023 - 500:
            sc = _from_bits((2046 - ex) << 52)
            p2 *= sc
            p1 *= sc
        p0, p1 = p1, p2
    return c


def _check(rng, m, dscale, escale, npts):
    d = rng.standard_normal(m) * dscale
    e = rng.standard_normal(max(m - 1, 0)) * escale
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    w = np.linalg.eigvalsh(T)
    off = 1e-9 * max(1.0, float(np.max(np.abs(w))))
    xs = list(rng.uniform(w.min() - 1, w.max() + 1, npts))
    if m > 1:
        xs += list((w[:-1] + w[1:]) / 2)  # between neighbours
    xs += list(w - off) + list(w + off)
    for x in xs:
        assert count_minors(d, e * e, x) == int(np.sum(w < x)), (m, x)


def test_counts_match_eigenvalues():
    rng = np.random.default_rng(0)
    for _ in range(60):
        _check(rng, int(rng.integers(1, 90)), 3.0, 10 ** rng.uniform(-6, 1), 10)


def test_counts_with_rescaling():
    """Wide diagonals and long chains: the minors run far outside
    [2^-500, 2^500] and are rescaled."""
    rng = np.random.default_rng(1)
    for _ in range(12):
        m = int(rng.integers(150, 256))
        _check(rng, m, 10 ** rng.uniform(2, 4), 10 ** rng.uniform(-8, 3), 6)


def test_zero_minor_counts_as_change():
    # T = [[0, 1], [1, 0]], x = 0: p_1 = 0 (counted), eigenvalues -1, 1 -> one below 0
    assert count_minors(np.array([0.0, 0.0]), np.array([1.0]), 0.0) == 1
