"""The ris-approximated Z-vector solve (A+B) Z = rhs on the GPU against the
oracle: a dense solve on the small chain, and at the C20H22 size the
integral-level bilinear form V.(A+B).Z = V.rhs for random V (the dense
matrix is too large there).  FP64: the CG residual tolerance is 1e-12
relative, so the solution error is bounded by cond(A+B) * 1e-12; mixed
precision: residual 1e-6 relative on the 3xTF32 operator."""
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


@pytest.fixture(scope="module")
def small(oracle):
    mol = synth.workload(0)
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc)
    rhs = synth.random_amplitudes(4, mol.nocc, mol.nvir, seed=21)
    rhs[2] = 0.0  # a zero right-hand side stays zero
    A, B = orc.dense_AB()
    ev = np.linalg.eigvalsh(A + B)
    return mol, orc, rhs, orc.zvector(rhs), ev[-1] / ev[0]


def _ctx(ris_mod, mol, **opt):
    c = ris_mod.Context(**opt)
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    return c


@gpu
@pytest.mark.parametrize("rpa", [0, 1])
def test_zvector_fp64_matches_dense_solve(ris_mod, small, rpa):
    mol, orc, rhs, Zref, kappa = small
    c = _ctx(ris_mod, mol, rpa=rpa, conv_tol=1e-12)
    Z = c.zvector(np.ascontiguousarray(rhs))
    err = np.max(np.abs(Z - Zref)) / np.max(np.abs(Zref))
    assert err <= max(1e-9, 2 * kappa * 1e-12)
    assert np.all(Z[2] == 0.0)
    st = c.stats()
    assert st["n_products"] > 0 and st["residual_max"] <= 1e-12


@gpu
def test_zvector_mixed(ris_mod, small):
    mol, orc, rhs, Zref, kappa = small
    c = _ctx(ris_mod, mol, precision=ris_mod.MIXED)
    Z = c.zvector(np.ascontiguousarray(rhs))
    err = np.max(np.abs(Z - Zref)) / np.max(np.abs(Zref))
    assert err <= max(1e-5, 4 * kappa * 1e-6)


@gpu
def test_zvector_device_pointers(ris_mod, small):
    import torch
    mol, orc, rhs, Zref, kappa = small
    c = _ctx(ris_mod, mol, conv_tol=1e-12)
    r = torch.as_tensor(rhs, device="cuda")
    Z = torch.zeros_like(r)
    c.zvector(r, out=Z)
    assert np.max(np.abs(Z.cpu().numpy() - Zref)) <= max(1e-9, 2 * kappa * 1e-12) * np.max(np.abs(Zref))


@gpu
@pytest.mark.slow
def test_zvector_chain_bilinear_form(ris_mod, oracle):
    mol = synth.workload(1)
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc)
    rhs = synth.random_amplitudes(2, mol.nocc, mol.nvir, seed=31)
    c = _ctx(ris_mod, mol, conv_tol=1e-12)
    Z = c.zvector(rhs)
    V = synth.random_amplitudes(2, mol.nocc, mol.nvir, seed=32)
    for k in range(2):
        for v in V:
            lhs = orc.apb_form(v, Z[k])
            assert abs(lhs - float(np.sum(v * rhs[k]))) <= 1e-9 * max(1.0, np.linalg.norm(Z[k]))
