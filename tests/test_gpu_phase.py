"""Phase tracking along a trajectory: each state's sign follows the previous
step through the overlap over its five most dominant determinants.  The
decision (an integer per state) is compared bit-exactly with the oracle's
phase rule; planted sign flips are undone; couplings computed from
the aligned amplitudes change sign exactly with the flipped states."""
import numpy as np
import pytest

from paper_2511_18233_gb300 import serve, synth

gpu = pytest.mark.gpu
NS = 5


@pytest.fixture(scope="module")
def ris_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris


def rule(X, Xp):
    """The oracle's phase decision per state (five most dominant
    determinants of the previous step)."""
    from oracle import ris_oracle
    return ris_oracle.phase_align(X, Xp)[0]


def _ctx(ris_mod, mol, coords):
    c = ris_mod.Context()
    c.build_aux(coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    return c


@gpu
def test_planted_flips_are_undone(ris_mod):
    mol = synth.serving_molecule("chain", 8, 5)
    c = _ctx(ris_mod, mol, mol.coords)
    om, X0 = c.excite(NS)
    num0 = np.zeros((2, mol.natm, 3))
    c.nac([(0, 1), (1, 3)], numerator=num0)
    flip = np.array([1, -1, 1, -1, 1])
    Xp = X0 * flip[:, None, None]
    Xa = np.zeros_like(X0)
    sg = c.phase_align(Xp, X_out=Xa)
    np.testing.assert_array_equal(sg, flip)
    np.testing.assert_array_equal(Xa, Xp)
    num1 = np.zeros((2, mol.natm, 3))
    c.nac([(0, 1), (1, 3)], numerator=num1)
    np.testing.assert_allclose(num1[0], -num0[0], rtol=0, atol=1e-12 * np.max(np.abs(num0)))
    np.testing.assert_allclose(num1[1], num0[1], rtol=0, atol=1e-12 * np.max(np.abs(num0)))
    assert np.all(c.phase_align(Xp) == 1)  # already aligned


@gpu
def test_decisions_match_rule_along_steps(ris_mod):
    mol = synth.serving_molecule("flake", 4.5, 6)
    spec = serve.TrajectorySpec(0, "flake", 4.5, NS, 1, 6)
    prev = None
    for step in range(3):
        xyz = serve.step_coords(mol.coords, spec, step)
        c = _ctx(ris_mod, mol, xyz)
        om, X = c.excite(NS)
        if prev is not None:
            expect = rule(X, prev)
            Xa = np.zeros_like(X)
            sg = c.phase_align(prev, X_out=Xa)
            np.testing.assert_array_equal(sg, expect)
            np.testing.assert_array_equal(Xa, X * sg[:, None, None])
            X = Xa
        prev = X
        c.close()


@gpu
def test_serving_keeps_phases_and_returns_time_couplings(ris_mod):
    specs = [serve.TrajectorySpec(0, "chain", 12, 6, 2, 12)]
    trajs = serve.build_trajectories(specs)
    ex = serve.RisExecutor(1, "mixed", 0, False)
    seen = []
    for tr in trajs:
        ex.make_resident(tr)
    try:
        for step in range(3):
            req = serve.Request(trajs[0], step, serve.step_coords(trajs[0].ref, specs[0], step))
            res, _ = ex(0, req)
            s = trajs[0].state
            seen.append(s["X"][s["cur"]].cpu().numpy().copy())
            v = serve.step_velocities(trajs[0].mol.elements, specs[0], step)
            np.testing.assert_allclose(res["T"], np.einsum("pax,ax->p", res["nac"], v))
    finally:
        ex.close()
    for a, b in zip(seen, seen[1:]):
        assert np.all(rule(b, a) == 1)  # every state's phase follows the previous step
