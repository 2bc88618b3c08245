"""Parity on the 2-copy cut-down of the packed 12 x C20H22 workload (84 atoms,
1024 AOs, 8 states as for the full packed workload): the first two chains of
that packing.  Energies against the oracle's Davidson, gradients and one
coupling against the oracle's per-atom derivative route on two atoms (one per
chain), the translation sum rule on every gradient; FP64 at the parity
tolerance, mixed precision at the stated error."""
import numpy as np
import pytest

from paper_2511_18233_gb300 import synth

gpu = pytest.mark.gpu
NS = 8
ATOMS = [3, 45]          # a carbon of each chain
PAIR = (2, 3)


@pytest.fixture(scope="module")
def ris_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris


@pytest.fixture(scope="module")
def ref(oracle):
    mol = synth.packed_cutdown(2)
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc)
    w, X, _ = orc.tda_davidson(NS + 1, tol=1e-10)
    g = orc.gradients([0, NS - 1], X[:NS], atoms=ATOMS)
    num = orc.pair_energy_derivs([PAIR], X[:NS], atoms=ATOMS)
    return mol, w[:NS], X[:NS], g, num


def _run(ris_mod, mol, **opt):
    c = ris_mod.Context(**opt)
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    om, X = c.excite(NS)
    g = c.gradient(range(NS))
    num = np.zeros((NS - 1, mol.natm, 3))
    c.nac([(s, s + 1) for s in range(NS - 1)], numerator=num)
    return om, X, g, num


@gpu
@pytest.mark.slow
def test_cutdown_fp64_parity(ris_mod, ref):
    mol, w, X, g_ref, num_ref = ref
    om, Xg, g, num = _run(ris_mod, mol)
    np.testing.assert_allclose(om, w, rtol=1e-9)
    sel = g[[0, NS - 1]][:, ATOMS]
    gr = g_ref[:, ATOMS]
    assert np.max(np.abs(sel - gr)) <= 1e-9 * np.max(np.abs(gr))
    nr = num_ref[0, ATOMS]
    assert np.max(np.abs(num[PAIR[0], ATOMS] - nr)) <= 1e-9 * np.max(np.abs(nr))
    # translation sum rule on every gradient and coupling numerator
    assert np.max(np.abs(g.sum(axis=1))) <= 1e-10 * np.max(np.abs(g))
    assert np.max(np.abs(num.sum(axis=1))) <= 1e-10 * np.max(np.abs(num))


@gpu
@pytest.mark.slow
def test_cutdown_streamed_fp64_parity(ris_mod, ref):
    """The streamed form (screened-pair integrals, auxiliary blocks,
    regenerated derivative integrals) on the same cut-down, at the FP64
    parity tolerance against the oracle."""
    mol, w, X, g_ref, num_ref = ref
    om, Xg, g, num = _run(ris_mod, mol, stream=1, stream_block=48)
    np.testing.assert_allclose(om, w, rtol=1e-9)
    # relative error of a result array (G14): max|diff| over the sampled
    # atoms against the array's largest element (the library's full array;
    # the oracle sampled two atoms only)
    sel = g[[0, NS - 1]][:, ATOMS]
    gr = g_ref[:, ATOMS]
    assert np.max(np.abs(sel - gr)) <= 1e-9 * max(np.max(np.abs(gr)), np.max(np.abs(g[[0, NS - 1]])))
    nr = num_ref[0, ATOMS]
    assert np.max(np.abs(num[PAIR[0], ATOMS] - nr)) <= 1e-9 * max(np.max(np.abs(nr)),
                                                                  np.max(np.abs(num[PAIR[0]])))
    assert np.max(np.abs(g.sum(axis=1))) <= 1e-10 * np.max(np.abs(g))


@gpu
@pytest.mark.slow
def test_cutdown_mixed_stated_error(ris_mod, ref):
    mol, w, X, g_ref, num_ref = ref
    om, Xg, g, num = _run(ris_mod, mol, precision=ris_mod.MIXED)
    assert np.max(np.abs(om - w)) <= 1e-6
    assert np.max(np.abs(g[[0, NS - 1]][:, ATOMS] - g_ref[:, ATOMS])) <= 1e-5
    assert np.max(np.abs(num[PAIR[0], ATOMS] - num_ref[0, ATOMS])) <= 1e-5
