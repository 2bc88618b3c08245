"""Orbital energy window (MO-space truncation): the library keeps occupied
MOs within mo_window below the HOMO and virtual MOs within mo_window above
the LUMO; every result must equal the oracle run on the same truncated MO
set (FP64 parity tolerance), and a window wider than the spectrum changes
nothing."""
import numpy as np
import pytest

from paper_2511_18233_gb300 import synth

gpu = pytest.mark.gpu
W = 0.35


@pytest.fixture(scope="module")
def ris_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris


def _ctx(ris_mod, mol, C=None, eps=None, nocc=None, **opt):
    c = ris_mod.Context(**opt)
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C if C is None else C, mol.mo_energy if eps is None else eps,
              mol.nocc if nocc is None else nocc)
    return c


def _window(mol):
    e, o = mol.mo_energy, mol.nocc
    i0 = int(np.argmax(e[:o] >= e[o - 1] - W))
    a1 = o + int(np.sum(e[o:] <= e[o] + W))
    return i0, a1


@gpu
def test_window_matches_oracle_on_truncated_mos(ris_mod, oracle):
    mol = synth.workload(0)
    i0, a1 = _window(mol)
    assert i0 > 0 and a1 < mol.C.shape[1]
    c = _ctx(ris_mod, mol, mo_window=W)
    assert c.mo_window() == (i0, mol.nocc - i0, a1 - mol.nocc)
    om, X = c.excite(4)
    assert X.shape == (4, mol.nocc - i0, a1 - mol.nocc)
    Cs = np.ascontiguousarray(mol.C[:, i0:a1])
    es = np.ascontiguousarray(mol.mo_energy[i0:a1])
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, Cs, es, mol.nocc - i0)
    w, Xr = orc.tda_dense(5)
    np.testing.assert_allclose(om, w[:4], rtol=1e-9)
    g = c.gradient([0, 3], X=np.ascontiguousarray(Xr[:4]))
    gr = orc.gradients([0, 3], Xr[:4])
    assert np.max(np.abs(g - gr)) <= 1e-9 * np.max(np.abs(gr))
    # the same as handing the library the truncated MOs directly
    c2 = _ctx(ris_mod, mol, C=Cs, eps=es, nocc=mol.nocc - i0)
    om2, X2 = c2.excite(4)
    np.testing.assert_allclose(om2, om, rtol=1e-13)


@gpu
def test_wide_window_changes_nothing(ris_mod):
    mol = synth.workload(0)
    c0 = _ctx(ris_mod, mol)
    c1 = _ctx(ris_mod, mol, mo_window=100.0)
    assert c1.mo_window() == (0, mol.nocc, mol.C.shape[1] - mol.nocc)
    np.testing.assert_array_equal(c0.excite(3)[0], c1.excite(3)[0])
