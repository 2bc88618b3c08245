"""Parity of the sm_103a library (through its C ABI) against the FP64 oracle.

Tolerances (FP64 path):
  * integrals / metric-derived quantities and gradients/couplings computed
    from the same amplitudes: max|diff| / max|ref| <= 1e-9 per result array;
  * excitation energies: relative 1e-9 (the Davidson eigenvalue error is
    quadratic in the residual, <= 1e-10 here, so rounding dominates);
  * amplitudes: |diff| <= 2 r/gap with r the residual tolerance (1e-10) and
    gap the distance to the nearest other eigenvalue (first-order
    perturbation bound), floored at 1e-9.
"""
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
def test_boys_function(ris_mod, oracle):
    rng = np.random.default_rng(0)
    T = np.concatenate([np.linspace(0, 45, 700), rng.uniform(0, 60, 300), [0.0, 1e-12, 39.999, 40.0, 40.001, 300.0]])
    m = rng.integers(0, 10, size=T.size).astype(np.int32)
    got = ris_mod.debug_boys(m, T)
    ref = np.array([oracle.boys(int(a), float(b)) for a, b in zip(m, T)])
    np.testing.assert_allclose(got, ref, rtol=2e-14, atol=0)


@gpu
def test_apply_A_small(ris_mod, small):
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol)
    Xr = synth.random_amplitudes(4, mol.nocc, mol.nvir, seed=9)
    got = c.apply(Xr)
    ref = orc.apply_A(Xr)
    assert _rel(got, ref) <= 1e-12


@gpu
def test_excitation_energies_small(ris_mod, small):
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol)
    om, Xg = c.excite(5)
    np.testing.assert_allclose(om, w[:5], rtol=1e-9)
    gaps = np.array([min(abs(w[k] - w[j]) for j in range(6) if j != k) for k in range(5)])
    for k in range(5):
        tol = max(2 * 1e-10 / gaps[k], 1e-9)
        assert np.max(np.abs(Xg[k] - X[k])) <= tol
    st = c.stats()
    assert st["n_products"] > 0 and st["excite_ms"] > 0


@gpu
@pytest.mark.parametrize("precond", [0, 1])
def test_preconditioners_same_states(ris_mod, small, precond):
    """Both Davidson preconditioners (Coulomb-exact fixed shift, diagonal per
    state) reach the oracle's eigenpairs; the preconditioner changes only how
    many products it takes.  A seeded search from the converged vectors
    needs no new products."""
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol, precond=precond)
    om, Xg = c.excite(5)
    np.testing.assert_allclose(om, w[:5], rtol=1e-9)
    om2, Xg2 = c.excite_guess(5, np.ascontiguousarray(Xg))
    np.testing.assert_allclose(om2, om, rtol=1e-12)
    assert c.stats()["n_iter"] == 0


@gpu
def test_coulomb_preconditioner_cuts_products(ris_mod):
    mol = synth.chain_molecule(12, 12, p_aux=True)
    n = {}
    om = {}
    for p in (0, 1):
        c = _ctx(ris_mod, mol, precond=p)
        om[p], _ = c.excite(6)
        n[p] = c.stats()["n_products"]
    np.testing.assert_allclose(om[0], om[1], rtol=1e-9)
    assert n[0] < 0.75 * n[1]


@gpu
def test_fewer_mos_than_aos(ris_mod, oracle):
    """MOs from canonical orthogonalisation with near-dependent AO
    combinations dropped (nmo < nao): energies, gradients and couplings
    against the oracle at the FP64 tolerance."""
    el, xyz = synth.chain_geometry(4)
    mol = synth.make_molecule("C4H6", el, xyz, 31, True, lindep=1e-2)
    assert mol.C.shape[1] < mol.nao
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc)
    w, X = orc.tda_dense(5)
    c = _ctx(ris_mod, mol)
    om, Xg = c.excite(4)
    np.testing.assert_allclose(om, w[:4], rtol=1e-9)
    Xin = np.ascontiguousarray(X[:4])
    assert _rel(c.gradient([0, 3], X=Xin), orc.gradients([0, 3], X[:4])) <= 1e-9
    assert _rel(c.nac([(1, 2)], X=Xin, omega=np.ascontiguousarray(w[:4])),
                orc.nacs([(1, 2)], w[:4], X[:4])) <= 1e-9


@gpu
def test_gradients_and_nac_small(ris_mod, small):
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol)
    Xin = np.ascontiguousarray(X[:5])
    g = c.gradient(range(5), X=Xin)
    ref = orc.gradients(range(5), X[:5])
    assert _rel(g, ref) <= 1e-9
    # translation sum rule
    assert np.max(np.abs(g.sum(axis=1))) <= 1e-10 * np.max(np.abs(g))
    nac = c.nac([(0, 1), (1, 0), (2, 4)], X=Xin, omega=np.ascontiguousarray(w[:5]))
    nref = orc.nacs([(0, 1), (1, 0), (2, 4)], w[:5], X[:5])
    assert _rel(nac, nref) <= 1e-9


@gpu
def test_full_pipeline_small(ris_mod, small):
    """excite -> gradient -> nac with the library's own amplitudes."""
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol)
    om, Xg = c.excite(5)
    g = c.gradient(range(5))
    ref = orc.gradients(range(5), Xg)
    assert _rel(g, ref) <= 1e-9
    nac = c.nac([(0, 1)])
    nref = orc.nacs([(0, 1)], om, Xg)
    assert _rel(nac, nref) <= 1e-9


def _grad_nac(c, ns):
    om, Xg = c.excite(ns)
    return om, c.gradient(range(ns)), c.nac([(0, 1), (1, 2)])


@gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_derivative_prefetch_same_results(ris_mod, small, precision):
    """Derivative integrals started on the side stream at ris_build_aux give
    the results of computing them in the first gradient call (same kernels,
    same order: equal up to a 1e-10 relative margin), and a context reused
    over a second geometry matches a fresh one."""
    mol = small[0]
    prec = ris_mod.MIXED if precision == "mixed" else ris_mod.FP64
    a = _grad_nac(_ctx(ris_mod, mol, precision=prec, deriv_prefetch=0), 4)
    c = _ctx(ris_mod, mol, precision=prec, deriv_prefetch=1)
    b = _grad_nac(c, 4)
    for x, y in zip(a, b):
        assert _rel(x, y) <= 1e-10
    xyz = mol.coords + 0.02 * np.random.default_rng(4).standard_normal(mol.coords.shape)
    c.build_aux(xyz, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    again = _grad_nac(c, 4)
    f = ris_mod.Context(precision=prec, deriv_prefetch=0)
    f.build_aux(xyz, mol.shells, mol.aux_j, mol.aux_k)
    f.build_B(mol.C, mol.mo_energy, mol.nocc)
    for x, y in zip(again, _grad_nac(f, 4)):
        assert _rel(x, y) <= 1e-10


@gpu
def test_random_amplitudes_and_device_pointers(ris_mod, small):
    import torch
    mol, orc, w, X = small
    c = _ctx(ris_mod, mol)
    Xr = synth.random_amplitudes(3, mol.nocc, mol.nvir, seed=5)
    pairs = [(0, 1), (2, 0), (1, 2)]
    om = np.array([0.1, 0.2, 0.35])
    ref = orc.pair_energy_derivs(pairs, Xr)
    num = np.zeros((3, mol.natm, 3))
    nac = c.nac(pairs, X=Xr, omega=om, numerator=num)
    assert _rel(num, ref) <= 1e-9
    den = np.array([om[J] - om[I] for I, J in pairs])
    assert _rel(nac, ref / den[:, None, None]) <= 1e-9
    g = c.gradient([2, 0], X=Xr)
    assert _rel(g, orc.pair_energy_derivs([(2, 2), (0, 0)], Xr)) <= 1e-9
    # a coupling of a state with itself is degenerate: error, numerator still written
    num2 = np.zeros((1, mol.natm, 3))
    with pytest.raises(ris_mod.RisError) as e:
        c.nac([(2, 2)], X=Xr, omega=om, numerator=num2)
    assert e.value.code == -8
    np.testing.assert_array_equal(num2[0], g[0])
    # the same calls with device buffers give identical bits
    Xd = torch.as_tensor(Xr, device="cuda")
    od = torch.as_tensor(om, device="cuda")
    nd = torch.zeros((3, mol.natm, 3), dtype=torch.float64, device="cuda")
    numd = torch.zeros_like(nd)
    c.nac(pairs, X=Xd, omega=od, out=nd, numerator=numd)
    np.testing.assert_array_equal(numd.cpu().numpy(), num)
    np.testing.assert_array_equal(nd.cpu().numpy(), nac)


@pytest.fixture(scope="module")
def chain(oracle):
    mol = synth.workload(1)
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc)
    w, X, _ = orc.tda_davidson(11, tol=1e-11)
    return mol, orc, w, X


@gpu
@pytest.mark.slow
def test_chain_c20h22_parity(ris_mod, chain):
    """The 42-atom chain with s+p Coulomb auxiliaries: 10 states, spot-checked
    gradients and adjacent couplings on sampled atoms."""
    mol, orc, w, X = chain
    c = _ctx(ris_mod, mol)
    om, Xg = c.excite(10)
    np.testing.assert_allclose(om, w[:10], rtol=1e-9)
    Xin = np.ascontiguousarray(X[:10])
    g = c.gradient(range(10), X=Xin)
    atoms = [0, 19, 33]
    ref = orc.gradients([0, 4, 9], X[:10], atoms=atoms)
    for k, s in enumerate([0, 4, 9]):
        assert _rel(g[s, atoms], ref[k, atoms]) <= 1e-9
    pairs = [(s, s + 1) for s in range(9)]
    nac = c.nac(pairs, X=Xin, omega=np.ascontiguousarray(w[:10]))
    nref = orc.nacs([(0, 1), (5, 6)], w[:10], X[:10], atoms=atoms)
    assert _rel(nac[0, atoms], nref[0, atoms]) <= 1e-9
    assert _rel(nac[5, atoms], nref[1, atoms]) <= 1e-9
    assert np.max(np.abs(g.sum(axis=1))) <= 1e-10 * np.max(np.abs(g))


@gpu
@pytest.mark.slow
def test_chain_c20h22_full_arrays(ris_mod, chain):
    """One complete gradient array (all 42 atoms) and all nine adjacent
    coupling numerators of the chain against the oracle's per-atom route,
    element by element, at the oracle's amplitudes; plus the translation sum
    rule on every array."""
    mol, orc, w, X = chain
    Xin = np.ascontiguousarray(X[:10])
    c = _ctx(ris_mod, mol)
    g = c.gradient([0], X=Xin)
    pairs = [(s, s + 1) for s in range(9)]
    num = np.zeros((9, mol.natm, 3))
    c.nac(pairs, X=Xin, omega=np.ascontiguousarray(w[:10]), numerator=num)
    ref = orc.pair_energy_derivs([(0, 0)] + pairs, Xin)
    assert _rel(g[0], ref[0]) <= 1e-9
    for p in range(9):
        assert _rel(num[p], ref[1 + p]) <= 1e-9, p
    for a in (g[0], *num):
        assert np.max(np.abs(a.sum(axis=0))) <= 1e-10 * np.max(np.abs(a))


@gpu
def test_error_paths(ris_mod, small):
    mol = small[0]
    c = ris_mod.Context()
    with pytest.raises(ris_mod.RisError) as e:
        c.build_B(mol.C, mol.mo_energy, mol.nocc)
    assert e.value.code == -7
    bad = mol.shells.copy()
    bad["l"][0] = 3
    with pytest.raises(ris_mod.RisError) as e:
        c.build_aux(mol.coords, bad, mol.aux_j, mol.aux_k)
    assert e.value.code == -1
    # two auxiliary functions on top of each other: singular metric
    dup = np.concatenate([mol.aux_j, mol.aux_j[:1]])
    with pytest.raises(ris_mod.RisError) as e:
        c.build_aux(mol.coords, mol.shells, dup, mol.aux_k)
    assert e.value.code == -3
    c2 = _ctx(ris_mod, mol)
    with pytest.raises(ris_mod.RisError) as e:
        c2.gradient([0])
    assert e.value.code == -7
    om, X = c2.excite(3)
    with pytest.raises(ris_mod.RisError) as e:
        c2.nac([(0, 0)])
    assert e.value.code == -8
