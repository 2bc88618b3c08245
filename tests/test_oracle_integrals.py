"""Pins of the oracle's integrals against facts that do not come from the
oracle itself: library special functions, closed forms, an independent
numerical quadrature, finite differences and exact invariances."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_2511_18233_gb300 import synth

PI = math.pi


def _nrm(l, a):
    return synth._norm(l, a)


# ------------------------------------------------------------------ Boys
@pytest.mark.parametrize("m", range(0, 9))
def test_boys_against_confluent_hypergeometric(oracle, m):
    # F_m(T) = 1F1(m+1/2; m+3/2; -T)/(2m+1), evaluated in 40-digit arithmetic
    # by mpmath (an independent arbitrary-precision library)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for T in [0.0, 1e-9, 1e-3, 0.37, 1.0, 4.2, 11.0, 29.9, 34.99, 35.01, 48.0, 120.0, 900.0]:
        ref = float(mpmath.hyp1f1(m + 0.5, m + 1.5, -T) / (2 * m + 1))
        assert oracle.boys(m, T) == pytest.approx(ref, rel=4e-15, abs=1e-300)


def test_boys_special_values(oracle):
    for m in range(10):
        assert oracle.boys(m, 0.0) == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)
    for T in [0.5, 3.0, 20.0, 40.0, 77.0]:
        assert oracle.boys(0, T) == pytest.approx(0.5 * math.sqrt(PI / T) * math.erf(math.sqrt(T)),
                                                  rel=1e-14)
        # downward identity F_m = (2T F_{m+1} + e^-T)/(2m+1)
        for m in range(7):
            lhs = oracle.boys(m, T)
            rhs = (2 * T * oracle.boys(m + 1, T) + math.exp(-T)) / (2 * m + 1)
            assert lhs == pytest.approx(rhs, rel=1e-13)


# ------------------------------------------------------------------ overlap
@pytest.mark.parametrize("idx", [0, 1])
def test_overlap_matches_quadrature_and_unit_diagonal(oracle, idx):
    mol = synth.workload(idx, with_mo=False)
    S = oracle.overlap(mol.coords, mol.shells)
    np.testing.assert_allclose(np.diag(S), 1.0, atol=1e-14)
    np.testing.assert_allclose(S, synth.overlap_matrix(mol.coords, mol.shells), atol=1e-13)


# ------------------------------------------------------------------ closed forms
def _sss(a, A, b, B, c, Cc):
    """(s_a s_b|s_c) for normalised s primitives, closed form."""
    A, B, Cc = map(np.asarray, (A, B, Cc))
    p = a + b
    P = (a * A + b * B) / p
    rho = p * c / (p + c)
    T = rho * np.sum((P - Cc) ** 2)
    F0 = 1.0 if T == 0 else 0.5 * math.sqrt(PI / T) * math.erf(math.sqrt(T))
    val = 2 * PI ** 2.5 / (p * c * math.sqrt(p + c)) * math.exp(-a * b / p * np.sum((A - B) ** 2)) * F0
    return val * _nrm((0, 0, 0), a) * _nrm((0, 0, 0), b) * _nrm((0, 0, 0), c)


def test_sss_closed_form(oracle):
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b, c = rng.uniform(0.05, 5.0, 3)
        A, B, Cc = rng.normal(0, 1.5, (3, 3))
        v = oracle.int3c_triple(0, a, A, 0, b, B, 0, c, Cc)[0, 0, 0]
        assert v == pytest.approx(_sss(a, A, b, B, c, Cc), rel=1e-13)


def test_two_centre_closed_form(oracle):
    coords = np.array([[0.0, 0.0, 0.0], [0.3, -1.1, 2.0]])
    aux = np.array([(0, 0, 0.7), (1, 0, 0.25)], dtype=synth.SHELL_DTYPE)
    M = oracle.int2c(coords, aux)
    for (i, j) in [(0, 0), (0, 1), (1, 1)]:
        a, b = aux["exp"][i], aux["exp"][j]
        R2 = np.sum((coords[i] - coords[j]) ** 2)
        rho = a * b / (a + b)
        T = rho * R2
        F0 = 1.0 if T == 0 else 0.5 * math.sqrt(PI / T) * math.erf(math.sqrt(T))
        ref = 2 * PI ** 2.5 / (a * b * math.sqrt(a + b)) * F0 * _nrm((0, 0, 0), a) * _nrm((0, 0, 0), b)
        assert M[i, j] == pytest.approx(ref, rel=1e-13)
        assert M[j, i] == pytest.approx(ref, rel=1e-13)


def test_p_aux_is_centre_derivative_of_s_aux(oracle):
    # (x - C_x) e^{-g r_C^2} = (1/2g) d/dC_x e^{-g r_C^2}: the normalised p
    # integral divided by N_p equals the C_x derivative (5-point FD of the
    # closed-form s integral) divided by 2g N_s.
    rng = np.random.default_rng(7)
    h = 1e-3
    for _ in range(6):
        a, b, g = rng.uniform(0.1, 3.0, 3)
        A, B, Cc = rng.normal(0, 1.2, (3, 3))
        p = oracle.int3c_triple(0, a, A, 0, b, B, 1, g, Cc)[0, 0, :]
        for d in range(3):
            vals = []
            for s in (-2, -1, 1, 2):
                C2 = Cc.copy()
                C2[d] += s * h
                vals.append(_sss(a, A, b, B, g, C2))
            fd = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
            e = [0, 0, 0]
            e[d] = 1
            lhs = p[d] / _nrm(tuple(e), g)
            rhs = fd / (2 * g * _nrm((0, 0, 0), g))
            assert lhs == pytest.approx(rhs, rel=1e-7, abs=1e-12)


@pytest.mark.parametrize("la,lb,lc", [(1, 0, 0), (2, 1, 0), (2, 2, 1), (0, 2, 1), (1, 1, 1)])
def test_bra_swap_symmetry(oracle, la, lb, lc):
    rng = np.random.default_rng(la * 9 + lb * 3 + lc)
    a, b, c = rng.uniform(0.1, 2.5, 3)
    A, B, Cc = rng.normal(0, 1.0, (3, 3))
    ab = oracle.int3c_triple(la, a, A, lb, b, B, lc, c, Cc)
    ba = oracle.int3c_triple(lb, b, B, la, a, A, lc, c, Cc)
    np.testing.assert_allclose(ab, ba.transpose(1, 0, 2), rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ quadrature
_GHX, _GHW = np.polynomial.hermite.hermgauss(24)


def _pair2d(i, j, k, a, A, b, B, g, Cc, t):
    """int int (x1-A)^i (x1-B)^j (x2-C)^k exp(-a(x1-A)^2 - b(x1-B)^2
    - t^2 (x1-x2)^2 - g(x2-C)^2) dx1 dx2 by 2-D Gauss-Hermite after
    completing the square (exact for these polynomial degrees)."""
    Q = np.array([[a + b + t * t, -t * t], [-t * t, g + t * t]])
    lin = np.array([a * A + b * B, g * Cc])
    m = np.linalg.solve(Q, lin)
    c0 = -(a * A * A + b * B * B + g * Cc * Cc) + lin @ m
    L = np.linalg.cholesky(Q)
    Linv_T = np.linalg.inv(L).T
    y1, y2 = np.meshgrid(_GHX, _GHX, indexing="ij")
    w = np.outer(_GHW, _GHW)
    x1 = m[0] + Linv_T[0, 0] * y1 + Linv_T[0, 1] * y2
    x2 = m[1] + Linv_T[1, 0] * y1 + Linv_T[1, 1] * y2
    f = (x1 - A) ** i * (x1 - B) ** j * (x2 - Cc) ** k
    return math.exp(c0) * np.sum(w * f) / np.prod(np.diag(L))


def _coulomb_quad(ca, a, A, cb, b, B, cc, g, Cc):
    """(a b|c) from 1/r = 2/sqrt(pi) int_0^inf exp(-t^2 r^2) dt, the t
    integral by adaptive quadrature and each t slice by exact separable
    Gauss-Hermite products."""
    def integrand(t):
        v = 1.0
        for d in range(3):
            v *= _pair2d(ca[d], cb[d], cc[d], a, A[d], b, B[d], g, Cc[d], t)
        return v
    val1, _ = integrate.quad(integrand, 0.0, 1.0, epsabs=0, epsrel=1e-13, limit=200)
    # tail with t = 1/u
    val2, _ = integrate.quad(lambda u: integrand(1.0 / u) / (u * u), 1e-12, 1.0, epsabs=0,
                             epsrel=1e-13, limit=200)
    nr = _nrm(ca, a) * _nrm(cb, b) * _nrm(cc, g)
    return 2.0 / math.sqrt(PI) * (val1 + val2) * nr


@pytest.mark.parametrize("la,lb,lc", [(0, 0, 0), (1, 0, 1), (2, 1, 0), (2, 2, 1), (1, 2, 1),
                                      (0, 0, 2), (1, 1, 2), (2, 2, 2)])
def test_three_centre_against_quadrature(oracle, la, lb, lc):
    rng = np.random.default_rng(100 + 9 * la + 3 * lb + lc)
    a, b, g = rng.uniform(0.15, 2.0, 3)
    A, B, Cc = rng.normal(0, 1.0, (3, 3))
    ints = oracle.int3c_triple(la, a, A, lb, b, B, lc, g, Cc)
    comps = [synth.cart_components(l) for l in (la, lb, lc)]
    # check a handful of components per triple
    picks = [(0, 0, 0), (len(comps[0]) - 1, len(comps[1]) - 1, len(comps[2]) - 1),
             (len(comps[0]) // 2, 0, len(comps[2]) - 1)]
    for (i, j, k) in picks:
        ref = _coulomb_quad(comps[0][i], a, A, comps[1][j], b, B, comps[2][k], g, Cc)
        assert ints[i, j, k] == pytest.approx(ref, rel=1e-9, abs=1e-12)


# ------------------------------------------------------------------ derivatives
@pytest.mark.parametrize("la,lb,lc", [(0, 0, 0), (1, 1, 0), (2, 1, 1), (2, 2, 1), (2, 0, 0),
                                      (1, 0, 2), (2, 2, 2)])
def test_centre_derivatives_fd_and_translation(oracle, la, lb, lc):
    rng = np.random.default_rng(200 + 9 * la + 3 * lb + lc)
    a, b, g = rng.uniform(0.15, 2.5, 3)
    cen = [np.array(v) for v in rng.normal(0, 1.0, (3, 3))]
    d = oracle.int3c_triple(la, a, cen[0], lb, b, cen[1], lc, g, cen[2], deriv=True)
    # translational invariance: the three centre derivatives sum to zero
    s = d.sum(axis=0)
    assert np.max(np.abs(s)) < 1e-12 * max(1.0, np.max(np.abs(d)))
    # 5-point finite differences of the integrals themselves
    h = 1e-3
    for c in range(3):
        for x in range(3):
            vals = []
            for st in (-2, -1, 1, 2):
                cc = [v.copy() for v in cen]
                cc[c][x] += st * h
                vals.append(oracle.int3c_triple(la, a, cc[0], lb, b, cc[1], lc, g, cc[2]))
            fd = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
            np.testing.assert_allclose(d[c, x], fd, rtol=1e-7, atol=1e-9)


def test_atom_derivative_tensors_sum_to_zero(oracle):
    mol = synth.workload(0, with_mo=False)
    tot3 = 0.0
    tot2 = 0.0
    for A in range(mol.natm):
        tot3 = tot3 + oracle.int3c_deriv_atom(A, mol.coords, mol.shells, mol.aux_j)
        tot2 = tot2 + oracle.int2c_deriv_atom(A, mol.coords, mol.aux_j)
    assert np.max(np.abs(tot3)) < 1e-12
    assert np.max(np.abs(tot2)) < 1e-12


def test_atom_derivative_tensor_fd(oracle):
    mol = synth.workload(0, with_mo=False)
    A, x, h = 1, 1, 1e-3
    d3 = oracle.int3c_deriv_atom(A, mol.coords, mol.shells, mol.aux_j)[x]
    d2 = oracle.int2c_deriv_atom(A, mol.coords, mol.aux_j)[x]
    v3, v2 = [], []
    for st in (-2, -1, 1, 2):
        c = mol.coords.copy()
        c[A, x] += st * h
        v3.append(oracle.int3c(c, mol.shells, mol.aux_j))
        v2.append(oracle.int2c(c, mol.aux_j))
    fd3 = (v3[0] - 8 * v3[1] + 8 * v3[2] - v3[3]) / (12 * h)
    fd2 = (v2[0] - 8 * v2[1] + 8 * v2[2] - v2[3]) / (12 * h)
    np.testing.assert_allclose(d3, fd3, atol=2e-9)
    np.testing.assert_allclose(d2, fd2, atol=2e-9)
