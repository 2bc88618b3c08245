"""Generality of the minimal auxiliary basis: J- and K-fitting sets with
different exponents (their union then holds both), and d auxiliary shells
(l = 2, cartesian components normalised one by one).  FP64 energies,
gradients and couplings against the oracle at the parity tolerance."""
import numpy as np
import pytest

from paper_2511_18233_gb300 import synth

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def ris_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris


def _sets(mol):
    aj = synth.build_aux(mol.elements, True)
    carb = [k for k, e in enumerate(mol.elements) if e == "C"]
    d = np.array([(a, 2, 0.3 / 1.32 ** 2) for a in carb], dtype=synth.SHELL_DTYPE)
    aux_j = np.concatenate([aj, d])
    aux_k = synth.build_aux(mol.elements, False).copy()
    aux_k["exp"] *= 1.3  # exponents distinct from the J set
    return aux_j, aux_k


@pytest.fixture(scope="module")
def case(oracle):
    mol = synth.workload(0)
    aux_j, aux_k = _sets(mol)
    orc = oracle.RisOracle(mol.coords, mol.shells, aux_j, aux_k, mol.C, mol.mo_energy, mol.nocc)
    w, X = orc.tda_dense(5)
    return mol, aux_j, aux_k, orc, w, X


@gpu
def test_d_aux_and_distinct_exponents(ris_mod, case):
    mol, aux_j, aux_k, orc, w, X = case
    c = ris_mod.Context()
    c.build_aux(mol.coords, mol.shells, aux_j, aux_k)
    d = c.dims()
    nJ = sum(synth.ncart(int(l)) for l in aux_j["l"])
    assert d["nauxJ"] == nJ and d["nauxK"] == len(aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    om, Xg = c.excite(4)
    np.testing.assert_allclose(om, w[:4], rtol=1e-9)
    Xin = np.ascontiguousarray(X[:4])
    g = c.gradient([0, 2], X=Xin)
    gr = orc.gradients([0, 2], X[:4])
    assert np.max(np.abs(g - gr)) <= 1e-9 * np.max(np.abs(gr))
    num = np.zeros((1, mol.natm, 3))
    c.nac([(1, 3)], X=Xin, omega=np.ascontiguousarray(w[:4]), numerator=num)
    nr = orc.pair_energy_derivs([(1, 3)], X[:4])
    assert np.max(np.abs(num - nr)) <= 1e-9 * np.max(np.abs(nr))
    assert np.max(np.abs(g.sum(axis=1))) <= 1e-10 * np.max(np.abs(g))


@gpu
def test_d_aux_mixed_stated_error(ris_mod, case):
    mol, aux_j, aux_k, orc, w, X = case
    c = ris_mod.Context(precision=ris_mod.MIXED)
    c.build_aux(mol.coords, mol.shells, aux_j, aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    om, Xg = c.excite(4)
    assert np.max(np.abs(om - w[:4])) <= 1e-6
    g = c.gradient([0, 2])
    assert np.max(np.abs(g - orc.gradients([0, 2], X[:4]))) <= 1e-5


@gpu
@pytest.mark.parametrize("rpa", [0, 1])
def test_k_set_inside_j_set_in_another_order(ris_mod, oracle, rpa):
    """K functions that are J functions listed in another order: the K half
    transforms are then gathered from the J ones (TDA: A X, energies and
    gradients; RPA: (A + B) X and (A - B) X, whose B part reads the gathered
    ov block)."""
    mol = synth.workload(0)
    aux_j = synth.build_aux(mol.elements, True)
    aux_k = synth.build_aux(mol.elements, False)[::-1].copy()
    orc = oracle.RisOracle(mol.coords, mol.shells, aux_j, aux_k, mol.C, mol.mo_energy, mol.nocc)
    c = ris_mod.Context(rpa=rpa)
    c.build_aux(mol.coords, mol.shells, aux_j, aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    Xr = synth.random_amplitudes(3, mol.nocc, mol.nvir, seed=21)
    A, B = orc.dense_AB()
    x = Xr.reshape(3, -1)
    if rpa:
        p, m = c.apply(Xr)
        for got, M in ((p, A + B), (m, A - B)):
            ref = (x @ M.T).reshape(Xr.shape)
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
        return
    got = c.apply(Xr)
    ref = (x @ A.T).reshape(Xr.shape)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    w, X = orc.tda_dense(4)
    om, Xg = c.excite(3)
    np.testing.assert_allclose(om, w[:3], rtol=1e-9)
    g = c.gradient([0, 2], X=np.ascontiguousarray(X[:3]))
    gr = orc.gradients([0, 2], X[:3])
    assert np.max(np.abs(g - gr)) <= 1e-9 * np.max(np.abs(gr))
