"""The ris excitation energy as a torch.autograd.Function: backward against
central finite differences of the re-solved energy and against the oracle."""
import numpy as np
import pytest

from paper_2511_18233_gb300 import synth

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build
    build.build()
    return torch


def _fd(model, coords, state, A, x, h, points=2):
    def e(d):
        c = coords.copy()
        c[A, x] += d
        return float(model.solve(__import__("torch").as_tensor(c))[0][state])
    if points == 2:
        return (e(h) - e(-h)) / (2 * h)
    return (e(-2 * h) - 8 * e(-h) + 8 * e(h) - e(2 * h)) / (12 * h)


@gpu
@pytest.mark.parametrize("rpa", [False, True])
def test_autograd_small_against_fd_and_oracle(torch_mod, oracle, rpa):
    torch = torch_mod
    from paper_2511_18233_gb300.autograd import RisModel
    mol = synth.workload(0)
    model = RisModel(mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy, mol.nocc, 4, rpa=rpa)
    R = torch.tensor(mol.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    w = model.energy(R, 1)
    w.backward()
    g = R.grad.cpu().numpy()
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy, mol.nocc)
    if rpa:
        om, X, Y = orc.rpa_dense(4)
        ref = orc.gradients([1], X, Y)[0]
    else:
        om, X = orc.tda_dense(4)
        ref = orc.gradients([1], X)[0]
    assert float(w.detach()) == pytest.approx(om[1], rel=1e-9)
    assert np.max(np.abs(g - ref)) <= 1e-9 * np.max(np.abs(ref))
    for (A, x) in [(0, 0), (5, 1)]:
        fd2 = _fd(model, mol.coords, 1, A, x, 1e-3, 2)
        fd5 = _fd(model, mol.coords, 1, A, x, 1e-3, 5)
        # 2-point stencil at h = 1e-3 bohr: O(h^2) truncation, ~1e-7 Ha/bohr here
        assert abs(g[A, x] - fd2) <= 1e-6
        assert abs(g[A, x] - fd5) <= 1e-9


@gpu
@pytest.mark.slow
def test_autograd_flake_rpa(torch_mod, oracle):
    """C54H18 flake, RPA, 20 states: the state-1 energy's backward against
    2-point central differences (step 1e-3 bohr) and the oracle (one atom)."""
    torch = torch_mod
    from paper_2511_18233_gb300 import ris
    from paper_2511_18233_gb300.autograd import RisModel
    mol = synth.workload(2)
    assert mol.nao == 1134 and mol.nocc == 171
    model = RisModel(mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy, mol.nocc, 20, rpa=True,
                     precision=ris.FP64)
    R = torch.tensor(mol.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    w = model.energy(R, 0)
    w.backward()
    g = R.grad.cpu().numpy()
    assert np.max(np.abs(g.sum(axis=0))) <= 1e-8
    # the oracle's gradient of the same state (library amplitudes), one atom
    out = model.solve(torch.as_tensor(mol.coords))
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy, mol.nocc)
    ref = orc.gradients([0], out[1][:1], out[2][:1], atoms=[60])[0]
    # cond(M_J) ~ 6e8 limits the agreement of two FP64 RI evaluations to ~1e-7
    assert np.max(np.abs(g[60] - ref[60])) <= 1e-6 * np.max(np.abs(ref[60]))
    # central differences, step 1e-3 bohr.  The flake's J metric has a
    # condition number ~6e8, so each FP64 energy carries ~1e-8 Ha of rounding
    # noise, i.e. ~1e-5 Ha/bohr in a 2-point difference at this step.
    for (A, x) in [(0, 0), (60, 1)]:
        fd = _fd(model, mol.coords, 0, A, x, 1e-3, 2)
        assert abs(g[A, x] - fd) <= 5e-5
