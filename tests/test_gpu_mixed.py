"""The 3xTF32 tensor-core path against FP64.

Stated error of the mixed form (against the FP64 oracle): excitation
energies <= 1e-6 Ha; gradients and coupling numerators dE_IJ/dR <= 1e-5
Ha/bohr (absolute, per component), so a coupling itself is within
1e-5/|omega_J - omega_I| 1/bohr.  The GEMM itself: 3xTF32 with FP32
accumulation in tensor memory keeps |C - A B^T| <= 2e-6 (|A| |B|^T)
elementwise up to K ~ 2000 and <= 1e-5 (|A| |B|^T) at K ~ 2e4, where the
FP32 accumulator's rounding grows with the number of terms; beyond K = 16384
the library runs the product in chunks whose results it sums in FP64.
"""
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


@gpu
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (200, 130, 71), (7, 300, 1000), (1278, 441, 18648),
                                   (2982, 441, 71), (64, 64, 4), (96, 160, 131072)])
def test_tc_gemm_against_fp64(ris_mod, M, N, K):
    rng = np.random.default_rng(M + 7 * N + 13 * K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = ris_mod.debug_gemm_tf32x3(A, B)
    ref = A @ B.T
    bound = np.abs(A) @ np.abs(B).T
    tol = 2e-6 if K <= 2048 else 1e-5
    print(f"\ntc_gemm {M}x{N}x{K}: max err / sum|a||b| {np.max(np.abs(C - ref) / bound):.1e}, "
          f"/ max|ref| {np.max(np.abs(C - ref)) / np.max(np.abs(ref)):.1e}")
    assert np.max(np.abs(C - ref) / bound) <= tol
    # and far below a single TF32 product's error (2^-11 relative per operand)


def _ctx(ris_mod, mol, **opt):
    c = ris_mod.Context(**opt)
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    return c


@pytest.fixture(scope="module")
def small(oracle):
    mol = synth.workload(0)
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc)
    w, X = orc.tda_dense(6)
    return mol, orc, w, X


@gpu
def test_mixed_apply(ris_mod, small):
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol, precision=ris_mod.MIXED)
    Xr = synth.random_amplitudes(5, mol.nocc, mol.nvir, seed=2)
    got = c.apply(Xr)
    ref = orc.apply_A(Xr)
    assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref))


@gpu
@pytest.mark.parametrize("eig32", [0, 1])
def test_mixed_small_stated_error(ris_mod, small, eig32):
    """Stated error, with the FP64 subspace eigensolver (default) and with
    its FP32 form (option eig_fp32)."""
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol, precision=ris_mod.MIXED, eig_fp32=eig32)
    om, Xg = c.excite(5)
    assert np.max(np.abs(om - w[:5])) <= 1e-6
    g = c.gradient(range(5))
    gref = orc.gradients(range(5), X[:5])
    assert np.max(np.abs(g - gref)) <= 1e-5
    pairs = [(0, 1), (2, 3)]
    num = np.zeros((2, mol.natm, 3))
    nac = c.nac(pairs, numerator=num)
    numref = orc.pair_energy_derivs(pairs, X[:5])
    assert np.max(np.abs(num - numref)) <= 1e-5
    gaps = np.array([abs(w[J] - w[I]) for I, J in pairs])
    nref = numref / np.array([w[J] - w[I] for I, J in pairs])[:, None, None]
    assert np.all(np.max(np.abs(nac - nref), axis=(1, 2)) <= 1e-5 / gaps)


@gpu
def test_mixed_refined_to_fp64(ris_mod, small):
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol, precision=ris_mod.MIXED, refine=1)
    om, Xg = c.excite(5)
    np.testing.assert_allclose(om, w[:5], rtol=1e-9)
    st = c.stats()
    assert st["n_products"] > 0


@pytest.fixture(scope="module")
def chain(oracle):
    mol = synth.workload(1)
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc)
    w, X, _ = orc.tda_davidson(11, tol=1e-10)
    return mol, orc, w, X


@gpu
@pytest.mark.slow
@pytest.mark.parametrize("eig32", [0, 1])
def test_mixed_chain_stated_error(ris_mod, chain, eig32):
    mol, orc, w, X = chain
    c = _ctx(ris_mod, mol, precision=ris_mod.MIXED, eig_fp32=eig32)
    om, Xg = c.excite(10)
    assert np.max(np.abs(om - w[:10])) <= 1e-6
    g = c.gradient(range(10))
    atoms = [3, 21]
    gref = orc.gradients([0, 7], X[:10], atoms=atoms)
    assert np.max(np.abs(g[[0, 7]][:, atoms] - gref[:, atoms])) <= 1e-5
    num = np.zeros((9, mol.natm, 3))
    c.nac([(s, s + 1) for s in range(9)], numerator=num)
    nref = orc.pair_energy_derivs([(2, 3)], X[:10], atoms=atoms)
    assert np.max(np.abs(num[2, atoms] - nref[0, atoms])) <= 1e-5


@gpu
def test_subspace_ff_same_states(ris_mod):
    """The double-FP32 subspace products (option subspace_ff, default on)
    against FP64 ones on the C20H22 chain: the same excitation energies to
    well below the stated error, and the double-FP32 kernels actually ran."""
    mol = synth.workload(1)
    out = {}
    for ff in (0, 1):
        c = _ctx(ris_mod, mol, precision=ris_mod.MIXED, subspace_ff=ff, profile=1)
        c.stats()  # reset the per-class timers
        om, X = c.excite(10)
        out[ff] = (om, c.stats())
        c.close()
    assert out[1][1]["ff_gemm_ms"] > 0 and out[0][1]["ff_gemm_ms"] == 0
    print(f"\nsubspace products: FP64 {out[0][1]['gemm_ms']:.2f} ms; double-FP32 "
          f"{out[1][1]['ff_gemm_ms']:.2f} ms + FP64 {out[1][1]['gemm_ms']:.2f} ms")
    assert np.max(np.abs(out[1][0] - out[0][0])) <= 1e-8
    assert out[1][1]["residual_max"] <= 1e-6
