"""The streamed form for large systems (option stream): three-centre integrals
only on the screened function pairs, mixed there with the metric factors;
MO transforms over blocks of auxiliary functions; the exchange part of the
Davidson products over blocks of occupied orbitals; derivative integrals
regenerated block by block in the gradient.

Forced on the C20H22 chain with small blocks (several of them, ragged last
ones, blocks inside the K part and the J-only part), the streamed form must
reproduce the dense form: in FP64 to rounding (the two differ only in
summation order), in mixed precision within the stated error of the FP64
results.  The full packed 12 x C20H22 workload (6144 AOs, where the dense
form would need about a terabyte) runs in mixed precision and is checked by
properties that hold at any size."""
import numpy as np
import pytest

from paper_2511_18233_gb300 import synth

gpu = pytest.mark.gpu
NS = 6


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


def _run(ris_mod, mol, ns, X=None, **opt):
    c = ris_mod.Context(**opt)
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    om, Xg = c.excite(ns)
    Xin = np.ascontiguousarray(Xg if X is None else X)
    g = c.gradient(range(ns), X=Xin)
    num = np.zeros((ns - 1, mol.natm, 3))
    c.nac([(s, s + 1) for s in range(ns - 1)], X=Xin, omega=np.ascontiguousarray(om), numerator=num)
    st = c.stats()
    c.close()
    return om, Xg, g, num, st


@pytest.fixture(scope="module")
def chain_dense(ris_mod):
    mol = synth.workload(1)
    return mol, _run(ris_mod, mol, NS)


@gpu
@pytest.mark.parametrize("block", [7, 40])
def test_streamed_fp64_equals_dense(ris_mod, chain_dense, block):
    mol, (om, X, g, num, _) = chain_dense
    # 102 J functions (42 s, then 60 p) in blocks of at most `block`
    om2, X2, g2, num2, st = _run(ris_mod, mol, NS, X=X, stream=1, stream_block=block)
    assert _rel(om2, om) <= 1e-12
    # the same amplitudes on both sides: the derivative kernels alone
    assert _rel(g2, g) <= 1e-11
    assert _rel(num2, num) <= 1e-11
    assert np.max(np.abs(g2.sum(axis=1))) <= 1e-10 * np.max(np.abs(g2))


@gpu
def test_streamed_mixed_within_stated_error(ris_mod, chain_dense):
    mol, (om, X, g, num, _) = chain_dense
    # occupied blocks of 20 (71 = 3 x 20 + 11) in the exchange products
    om2, X2, g2, num2, st = _run(ris_mod, mol, NS, X=X, precision=ris_mod.MIXED, stream=1,
                                 stream_block=16, occ_block=20)
    assert np.max(np.abs(om2 - om)) <= 1e-6
    assert np.max(np.abs(g2 - g)) <= 1e-5
    assert np.max(np.abs(num2 - num)) <= 1e-5
    assert st["residual_max"] <= 1e-6
    # and against the dense mixed form (same arithmetic, other order)
    om3, _, g3, _, _ = _run(ris_mod, mol, NS, X=X, precision=ris_mod.MIXED)
    assert np.max(np.abs(om2 - om3)) <= 5e-7
    assert np.max(np.abs(g2 - g3)) <= 5e-6


@gpu
@pytest.mark.slow
def test_packed_12x_c20h22_streamed_mixed(ris_mod):
    """12 x C20H22 (504 atoms, 6144 AOs, 852 occupied, 1224 J / 504 K
    auxiliary functions): 8 states, 8 gradients, 7 adjacent couplings in the
    streamed mixed form.  The oracle is out of reach at this size (its dense
    three-centre tensor alone is 370 GB), so the checks are properties: the
    Davidson residuals within the mixed tolerance, the translation sum rule
    on every gradient and coupling numerator, the numerators symmetric in the
    pair, and ascending positive energies.  (Parity of the same streamed
    code against the dense form and the oracle: the tests above and
    test_gpu_cutdown.py.)"""
    mol = synth.workload(3)
    assert mol.nao == 6144 and mol.nocc == 852
    ns = 8
    c = ris_mod.Context(precision=ris_mod.MIXED)
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    om, X = c.excite(ns)
    st = c.stats()
    g = c.gradient(range(ns))
    pairs = [(s, s + 1) for s in range(ns - 1)]
    num = np.zeros((ns - 1, mol.natm, 3))
    nac = c.nac(pairs, numerator=num)
    back = np.zeros((1, mol.natm, 3))
    c.nac([(1, 0)], numerator=back)
    print(f"\npacked 12 x C20H22: omega {np.round(om, 6).tolist()}; residual {st['residual_max']:.1e}; "
          f"products {int(st['n_products'])}; peak {st['bytes_peak'] / 2**30:.1f} GiB")
    assert np.all(np.diff(om) >= 0) and om[0] > 0
    assert st["residual_max"] <= 1e-6
    for a in (*g, *num):
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a.sum(axis=0))) <= 1e-8 * np.max(np.abs(a))
    # the (1,0) and (0,1) numerators come from differently ordered
    # tensor-core products; their values are ~1e-5 Ha/bohr, so the check is
    # absolute, two orders below the stated 1e-5 Ha/bohr error
    sym = float(np.max(np.abs(back[0] - num[0])))
    print(f"numerator symmetry {sym:.1e} Ha/bohr (max |num| {np.max(np.abs(num[0])):.1e})")
    assert sym <= 1e-7
    c.close()
