"""Pins of the oracle's ris energies, gradients and couplings against facts
that do not come from the oracle's own formulas: dense diagonalisation, a
secular equation solved by bisection, exact invariances of the RI model,
Hellmann-Feynman finite differences of re-solved eigenvalues and
finite-difference eigenvector overlaps."""
import itertools

import numpy as np
import pytest

from paper_2511_18233_gb300 import synth


@pytest.fixture(scope="module")
def mol0():
    return synth.workload(0)


@pytest.fixture(scope="module")
def orc0(oracle, mol0):
    m = mol0
    return oracle.RisOracle(m.coords, m.shells, m.aux_j, m.aux_k, m.C, m.mo_energy, m.nocc)


def _make(oracle, m, coords=None, C=None, cls=None, cx=0.25):
    cls = cls or oracle.RisOracle
    return cls(m.coords if coords is None else coords, m.shells, m.aux_j, m.aux_k,
               m.C if C is None else C, m.mo_energy, m.nocc, cx=cx)


def test_davidson_matches_dense(orc0):
    w, X = orc0.tda_dense(6)
    w2, X2, _ = orc0.tda_davidson(6, tol=1e-11)
    np.testing.assert_allclose(w2, w, rtol=1e-13)
    np.testing.assert_allclose(X2, X, atol=1e-9)


def test_apply_A_matches_dense(orc0, mol0):
    A, _ = orc0.dense_AB()
    X = synth.random_amplitudes(3, mol0.nocc, mol0.nvir, seed=3)
    AX = orc0.apply_A(X)
    ref = (A @ X.reshape(3, -1).T).T.reshape(X.shape)
    np.testing.assert_allclose(AX, ref, atol=1e-13)
    np.testing.assert_allclose(A, A.T, atol=1e-14)


def test_secular_equation_one_aux_function(oracle):
    # one carbon, one s auxiliary function, c_x = 0, one occupied orbital:
    # A = diag(de) + 2 b b^T, so each eigenvalue is a root of
    # 1 + 2 sum_a b_a^2/(de_a - w) = 0 in (de_k, de_k+1), found by bisection.
    el = ["C"]
    xyz = np.zeros((1, 3))
    shells = synth.build_shells(el)
    aux = synth.build_aux(el, False)
    nao = int(sum(synth.ncart(int(l)) for l in shells["l"]))
    rng = np.random.default_rng(11)
    S = synth.overlap_matrix(xyz, shells)
    C = synth.lowdin_mo(S, synth.haar_orthogonal(nao, rng))
    eps = synth.orbital_energies(1, nao - 1, rng)
    orc = oracle.RisOracle(xyz, shells, aux, aux, C, eps, 1, cx=0.0)
    w, _ = orc.tda_dense(4)
    b = orc.ovJ[0, :, 0] / np.sqrt(orc.MJ[0, 0])
    d = orc.de[0]
    assert np.all(np.diff(d) > 0)

    def f(x):
        return 1.0 + 2.0 * np.sum(b * b / (d - x))
    roots = []
    for k in range(4):
        lo, hi = d[k] + 1e-15, d[k + 1] - 1e-15
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(mid) < 0:
                lo = mid
            else:
                hi = mid
        roots.append(0.5 * (lo + hi))
    np.testing.assert_allclose(w, roots, rtol=1e-12)


def test_ri_invariant_under_aux_mixing(oracle, mol0):
    # (pq|rs)_ris = T M^-1 T^T is unchanged by any invertible transform of the
    # auxiliary functions: T -> T G, M -> G^T M G.
    base = _make(oracle, mol0)
    w0, _ = base.tda_dense(5)
    rng = np.random.default_rng(3)

    class Mixed(oracle.RisOracle):
        def _setup(self):
            super()._setup()
            for T, M, name in ((self.TJ, self.MJ, "J"), (self.TK, self.MK, "K")):
                n = M.shape[0]
                G = np.eye(n) + 0.3 * rng.standard_normal((n, n))
                setattr(self, "T" + name, T @ G)
                setattr(self, "M" + name, G.T @ M @ G)
            self.MJinv = np.linalg.solve(self.MJ, np.eye(self.MJ.shape[0]))
            self.MKinv = np.linalg.solve(self.MK, np.eye(self.MK.shape[0]))
            Co, Cv = self.Co, self.Cv
            self.ovJ = self._mo3(self.TJ, Co, Cv)
            self.ooK = self._mo3(self.TK, Co, Co)
            self.vvK = self._mo3(self.TK, Cv, Cv)
            self.ovK = self._mo3(self.TK, Co, Cv)

    w1, _ = _make(oracle, mol0, cls=Mixed).tda_dense(5)
    np.testing.assert_allclose(w1, w0, rtol=1e-11)


def _rotation_rep(R, shells):
    """Matrix D with chi'_c(R r) = sum_c' D[c, c'] chi_c'(r) for normalised
    cartesian primitives rotated with the molecule."""
    blocks = []
    for s in shells:
        l, a = int(s["l"]), float(s["exp"])
        comps = synth.cart_components(l)
        idx = {c: k for k, c in enumerate(comps)}
        D = np.zeros((len(comps), len(comps)))
        for k, c in enumerate(comps):
            poly = {(0, 0, 0): 1.0}
            for d in range(3):
                for _ in range(c[d]):
                    new = {}
                    for mono, coef in poly.items():
                        for e in range(3):
                            m2 = list(mono)
                            m2[e] += 1
                            m2 = tuple(m2)
                            new[m2] = new.get(m2, 0.0) + coef * R[d, e]
                    poly = new
            for mono, coef in poly.items():
                D[k, idx[mono]] += coef * synth._norm(c, a) / synth._norm(mono, a)
        blocks.append(D)
    n = sum(b.shape[0] for b in blocks)
    out = np.zeros((n, n))
    o = 0
    for b in blocks:
        out[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    return out


def test_rotation_invariance_of_energies(oracle):
    m = synth.workload(1, with_mo=False)
    # a small piece of the C20H22 chain keeps this fast while carrying p aux
    keep = [0, 1, 2, 20, 21, 22]
    el = [m.elements[k] for k in keep]
    xyz = m.coords[keep]
    small = synth.make_molecule("frag", el, xyz, seed=77, p_aux=True)
    base = _make(oracle, small)
    w0, _ = base.tda_dense(4)
    R = synth.haar_rotation(np.random.default_rng(9))
    D = _rotation_rep(R, small.shells)
    C_rot = np.linalg.solve(D.T, small.C)
    rot = _make(oracle, small, coords=xyz @ R.T, C=C_rot)
    w1, _ = rot.tda_dense(4)
    np.testing.assert_allclose(w1, w0, rtol=1e-11)
    # rigid translation
    tr = _make(oracle, small, coords=xyz + np.array([1.7, -0.4, 3.1]))
    np.testing.assert_allclose(tr.tda_dense(4)[0], w0, rtol=1e-12)


def _fd5(fun, h=1e-3):
    # 5-point central difference, truncation O(h^4): at h = 1e-3 bohr about
    # 1e-10 of the derivative here (it grows 16x at h = 2e-3, so truncation,
    # not rounding, dominates), well inside the 1e-8 relative pins below
    return (fun(-2 * h) - 8 * fun(-h) + 8 * fun(h) - fun(2 * h)) / (12 * h)


def _relerr(a, ref):
    # relative error of a result array: max|diff| / max|ref|
    a, ref = np.asarray(a), np.asarray(ref)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def test_gradient_is_hellmann_feynman_of_resolved_eigenvalues(oracle, mol0, orc0):
    nst = 4
    w, X = orc0.tda_dense(nst)
    g = orc0.gradients(range(nst), X, atoms=[0, 7])
    for (A, x) in [(0, 0), (0, 2), (7, 1)]:
        def om(d):
            c = mol0.coords.copy()
            c[A, x] += d
            return _make(oracle, mol0, coords=c).tda_dense(nst)[0]
        fd = _fd5(om)
        assert _relerr(g[:, A, x], fd) <= 1e-8


def test_pair_energy_derivative_fd(oracle, mol0, orc0):
    X = synth.random_amplitudes(3, mol0.nocc, mol0.nvir, seed=21)
    pairs = [(0, 0), (0, 1), (2, 1)]
    d = orc0.pair_energy_derivs(pairs, X, atoms=[2, 9])
    for (A, x) in [(2, 0), (9, 1), (9, 2)]:
        for p, (I, J) in enumerate(pairs):
            def e(dd):
                c = mol0.coords.copy()
                c[A, x] += dd
                return _make(oracle, mol0, coords=c).pair_energy(X[I], X[J])
            assert d[p, A, x] == pytest.approx(_fd5(e), rel=1e-8, abs=1e-12)


def test_gradient_sum_rule_and_nac_antisymmetry(orc0):
    w, X = orc0.tda_dense(4)
    g = orc0.gradients(range(4), X)
    # translation: the per-atom derivatives of every pair energy sum to zero
    assert np.max(np.abs(g.sum(axis=1))) < 1e-11
    n12 = orc0.nacs([(0, 1), (1, 0)], w, X)
    np.testing.assert_allclose(n12[0], -n12[1], atol=1e-13)
    num = orc0.pair_energy_derivs([(0, 2), (2, 0)], X)
    np.testing.assert_allclose(num[0], num[1], atol=1e-13)


def test_nac_matches_fd_eigenvector_overlap(oracle, mol0, orc0):
    nst = 4
    w, X = orc0.tda_dense(nst)
    I, J = 0, 1
    nac = orc0.nacs([(I, J)], w, X, atoms=[1])[0]
    for x in range(3):
        def ov(d):
            c = mol0.coords.copy()
            c[1, x] += d
            _, Xd = _make(oracle, mol0, coords=c).tda_dense(nst)
            xj = Xd[J] * np.sign(np.sum(Xd[J] * X[J]))
            return np.sum(X[I] * xj)
        assert abs(nac[1, x] - _fd5(ov)) <= 1e-8 * np.max(np.abs(nac[1]))


def test_rpa_dense_solution_and_tda_limit(oracle, mol0, orc0):
    om, X, Y = orc0.rpa_dense(4)
    A, B = orc0.dense_AB()
    for k in range(4):
        x, y = X[k].ravel(), Y[k].ravel()
        np.testing.assert_allclose(A @ x + B @ y, om[k] * x, atol=1e-11)
        np.testing.assert_allclose(B @ x + A @ y, -om[k] * y, atol=1e-11)
        assert x @ x - y @ y == pytest.approx(1.0, rel=1e-12)
        assert orc0.pair_energy(X[k], X[k], Y[k], Y[k]) == pytest.approx(om[k], rel=1e-12)

    class NoB(oracle.RisOracle):
        def dense_AB(self):
            A, B = super().dense_AB()
            return A, np.zeros_like(B)
    om0, X0, Y0 = _make(oracle, mol0, cls=NoB).rpa_dense(4)
    np.testing.assert_allclose(om0, orc0.tda_dense(4)[0], rtol=1e-12)
    assert np.max(np.abs(Y0)) < 1e-12


def test_rpa_gradient_and_nac_fd(oracle, mol0, orc0):
    nst = 3
    om, X, Y = orc0.rpa_dense(nst)
    g = orc0.gradients(range(nst), X, Y, atoms=[3])
    nac = orc0.nacs([(0, 1)], om, X, Y, atoms=[3])[0]
    for x in (0, 2):
        def w_of(d):
            c = mol0.coords.copy()
            c[3, x] += d
            return _make(oracle, mol0, coords=c).rpa_dense(nst)[0]
        assert _relerr(g[:, 3, x], _fd5(w_of)) <= 1e-8

        def ov(d):
            c = mol0.coords.copy()
            c[3, x] += d
            _, Xd, Yd = _make(oracle, mol0, coords=c).rpa_dense(nst)
            s = np.sign(np.sum(Xd[1] * X[1]) - np.sum(Yd[1] * Y[1]))
            return np.sum(X[0] * Xd[1] * s) - np.sum(Y[0] * Yd[1] * s)
        assert abs(nac[3, x] - _fd5(ov)) <= 1e-8 * np.max(np.abs(nac[3]))


def test_zvector_solution_against_integral_level_forms(orc0, mol0):
    """The oracle's Z-vector (dense solve of (A+B) Z = rhs) checked through the
    integral-level kernels instead of the dense matrices: for random V,
    V.(A+B).Z must equal V.rhs; A+B must be positive definite (CG applies)."""
    rhs = synth.random_amplitudes(3, mol0.nocc, mol0.nvir, seed=11)
    Z = orc0.zvector(rhs)
    A, B = orc0.dense_AB()
    assert np.linalg.eigvalsh(A + B)[0] > 0
    V = synth.random_amplitudes(2, mol0.nocc, mol0.nvir, seed=12)
    for k in range(3):
        for v in V:
            lhs = orc0.apb_form(v, Z[k])
            assert abs(lhs - float(np.sum(v * rhs[k]))) <= 1e-11 * max(1.0, abs(lhs))
    # the dense A+B agrees with the integral-level bilinear form
    u, w = V
    assert abs(u.reshape(-1) @ (A + B) @ w.reshape(-1) - orc0.apb_form(u, w)) <= 1e-12


def test_d_aux_gradient_is_hellmann_feynman(oracle, mol0):
    """With d auxiliary shells on carbon and K-fit exponents distinct from the
    J-fit ones, the oracle's analytic gradient equals the 5-point finite
    difference of re-solved eigenvalues (pins its l = 2 auxiliary integrals,
    metric and derivative paths end to end)."""
    aj = synth.build_aux(mol0.elements, True)
    carb = [k for k, e in enumerate(mol0.elements) if e == "C"]
    d = np.array([(a, 2, 0.3 / 1.32 ** 2) for a in carb], dtype=synth.SHELL_DTYPE)
    aux_j = np.concatenate([aj, d])
    aux_k = synth.build_aux(mol0.elements, False).copy()
    aux_k["exp"] *= 1.3

    def make(coords):
        return oracle.RisOracle(coords, mol0.shells, aux_j, aux_k, mol0.C, mol0.mo_energy,
                                mol0.nocc)

    nst = 3
    w, X = make(mol0.coords).tda_dense(nst)
    g = make(mol0.coords).gradients(range(nst), X, atoms=[1])
    for x in (0, 2):
        def om(dd):
            c = mol0.coords.copy()
            c[1, x] += dd
            return make(c).tda_dense(nst)[0]
        assert _relerr(g[:, 1, x], _fd5(om)) <= 1e-8


def test_apply_ApB_AmB_matches_dense(orc0, mol0):
    A, B = orc0.dense_AB()
    Z = synth.random_amplitudes(2, mol0.nocc, mol0.nvir, seed=31)
    P, M = orc0.apply_ApB_AmB(Z)
    z = Z.reshape(2, -1)
    np.testing.assert_allclose(P.reshape(2, -1), z @ (A + B).T, atol=1e-13)
    np.testing.assert_allclose(M.reshape(2, -1), z @ (A - B).T, atol=1e-13)


def test_rpa_davidson_matches_dense(orc0):
    om, X, Y = orc0.rpa_dense(6)
    om2, X2, Y2, _ = orc0.rpa_davidson(6, tol=1e-10)
    np.testing.assert_allclose(om2, om, rtol=1e-13)
    # eigenvector error <= residual / gap (gaps here >= 1e-3 Ha)
    assert np.max(np.abs(X2 - X)) <= 1e-6 and np.max(np.abs(Y2 - Y)) <= 1e-6
    np.testing.assert_allclose(np.sum(X2 ** 2 - Y2 ** 2, axis=(1, 2)), 1.0, rtol=1e-12)


def test_phase_rule(oracle):
    rng = np.random.default_rng(17)
    X = rng.standard_normal((4, 3, 5))
    flips = np.array([1, -1, -1, 1])
    s, Xa = oracle.phase_align(X * flips[:, None, None], X)
    np.testing.assert_array_equal(s, flips)
    np.testing.assert_array_equal(Xa, X)
    # five dominant determinants of the previous state, equal magnitudes
    # taken in index order: elements 0, 1 (|3|) and 2, 3, 4 (|1|), not 5
    prev = np.array([[[3.0, -3.0, 1.0, 1.0, 1.0, 1.0, 0.5]]])
    new = np.array([[[1.0, 1.0, 1.0, 1.0, 1.0, -100.0, -100.0]]])
    assert oracle.phase_align(new, prev)[0][0] == 1      # 3 - 3 + 1 + 1 + 1 > 0
    new2 = new.copy()
    new2[0, 0, 2] = -3.0                                  # overlap 3 - 3 - 3 + 1 + 1 < 0
    assert oracle.phase_align(new2, prev)[0][0] == -1
    zero = np.array([[[1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0]]])
    assert oracle.phase_align(zero, prev)[0][0] == 1      # zero overlap keeps the sign


def test_metric_inverse_routes_agree_when_well_conditioned(oracle, mol0):
    X = synth.random_amplitudes(1, mol0.nocc, mol0.nvir, seed=41)
    out = []
    for route in ("solve", "cholesky", "eigh"):
        o = oracle.RisOracle(mol0.coords, mol0.shells, mol0.aux_j, mol0.aux_k, mol0.C,
                             mol0.mo_energy, mol0.nocc, metric_inverse=route)
        out.append((o.pair_energy(X[0], X[0]), o.pair_energy_derivs([(0, 0)], X, atoms=[0])[0, 0]))
    for e, g in out[1:]:
        assert abs(e - out[0][0]) <= 1e-13 * abs(out[0][0])
        assert np.max(np.abs(g - out[0][1])) <= 1e-11 * np.max(np.abs(out[0][1]))


@pytest.mark.slow
def test_flake_gradient_fp64_floor(oracle):
    """The flake's s+p Coulomb metric has cond(M_J) ~ 6e8.  Three FP64 routes
    to M_J^-1 that are equal in exact arithmetic (LU solve, Cholesky, eigh)
    give the same pair energies to ~1e-13 but gradients that differ by
    1e-6 .. 1e-4 of max|g|: the gradient's terms c^T dM c and c^T dv, with
    fitting coefficients c = M^-1 v large along the metric's smallest
    eigenvectors, cancel to a much smaller sum.  No FP64 evaluation of the
    RI derivative formula reaches 1e-9 there; the spread between the routes
    is the FP64 floor that the flake's GPU parity is held to."""
    mol = synth.workload(2)
    M = oracle.int2c(mol.coords, mol.aux_j)
    lam = np.linalg.eigvalsh(M)
    assert lam[-1] / lam[0] > 1e8
    X = synth.random_amplitudes(1, mol.nocc, mol.nvir, seed=43)
    Y = 0.1 * synth.random_amplitudes(1, mol.nocc, mol.nvir, seed=44)
    res = []
    for route in ("solve", "cholesky", "eigh"):
        o = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                             mol.nocc, metric_inverse=route)
        res.append((o.pair_energy(X[0], X[0], Y[0], Y[0]),
                    o.pair_energy_derivs([(0, 0)], X, Y, atoms=[0])[0, 0]))
    e0, g0 = res[0]
    spread = max(np.max(np.abs(g - g0)) for _, g in res[1:]) / np.max(np.abs(g0))
    print(f"flake FP64 route spread: energy "
          f"{max(abs(e - e0) for e, _ in res[1:]) / abs(e0):.1e}, gradient {spread:.1e}")
    for e, _ in res[1:]:
        assert abs(e - e0) <= 1e-12 * abs(e0)
    assert 1e-7 <= spread <= 5e-4
