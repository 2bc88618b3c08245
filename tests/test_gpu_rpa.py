"""Full RPA-ris (X, Y) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from paper_2511_18233_gb300 import synth

gpu = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def ris_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris


@pytest.fixture(scope="module")
def small(oracle):
    mol = synth.workload(0)
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc)
    om, X, Y = orc.rpa_dense(6)
    return mol, orc, om, X, Y


def _ctx(ris_mod, mol, **opt):
    c = ris_mod.Context(rpa=1, **opt)
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    return c


@gpu
def test_rpa_products(ris_mod, small):
    mol, orc, om, X, Y = small
    c = _ctx(ris_mod, mol)
    Z = synth.random_amplitudes(3, mol.nocc, mol.nvir, seed=4)
    P, M = c.apply(Z)
    A, B = orc.dense_AB()
    z = Z.reshape(3, -1).T
    assert _rel(P, ((A + B) @ z).T.reshape(Z.shape)) <= 1e-12
    assert _rel(M, ((A - B) @ z).T.reshape(Z.shape)) <= 1e-12


@gpu
def test_rpa_excitations(ris_mod, small):
    mol, orc, om, X, Y = small
    c = _ctx(ris_mod, mol)
    w, Xg, Yg = c.excite(5)
    np.testing.assert_allclose(w, om[:5], rtol=1e-9)
    gaps = np.array([min(abs(om[k] - om[j]) for j in range(6) if j != k) for k in range(5)])
    for k in range(5):
        tol = max(4 * 1e-10 / gaps[k], 1e-9)
        assert np.max(np.abs(Xg[k] - X[k])) <= tol
        assert np.max(np.abs(Yg[k] - Y[k])) <= tol
        assert np.sum(Xg[k] ** 2 - Yg[k] ** 2) == pytest.approx(1.0, abs=1e-9)


@gpu
def test_rpa_gradients_and_nacs(ris_mod, small):
    mol, orc, om, X, Y = small
    c = _ctx(ris_mod, mol)
    Xi, Yi = np.ascontiguousarray(X[:5]), np.ascontiguousarray(Y[:5])
    g = c.gradient(range(5), X=Xi, Y=Yi)
    ref = orc.gradients(range(5), X[:5], Y[:5])
    assert _rel(g, ref) <= 1e-9
    assert np.max(np.abs(g.sum(axis=1))) <= 1e-10 * np.max(np.abs(g))
    pairs = [(0, 1), (3, 2)]
    nac = c.nac(pairs, X=Xi, Y=Yi, omega=np.ascontiguousarray(om[:5]))
    assert _rel(nac, orc.nacs(pairs, om[:5], X[:5], Y[:5])) <= 1e-9
    # with the library's own amplitudes
    w, Xg, Yg = c.excite(5)
    g2 = c.gradient([0, 1])
    assert _rel(g2, orc.gradients([0, 1], Xg, Yg)) <= 1e-9


@gpu
def test_rpa_mixed_stated_error(ris_mod, small):
    mol, orc, om, X, Y = small
    c = _ctx(ris_mod, mol, precision=ris_mod.MIXED)
    w, Xg, Yg = c.excite(5)
    assert np.max(np.abs(w - om[:5])) <= 1e-6
    g = c.gradient(range(3))
    assert np.max(np.abs(g - orc.gradients(range(3), X[:3], Y[:3]))) <= 1e-5
