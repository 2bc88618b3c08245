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
    assert float(w) == pytest.approx(om[1], rel=1e-9)
    assert np.max(np.abs(g - ref)) <= 1e-9 * np.max(np.abs(ref))
    for (A, x) in [(0, 0), (5, 1)]:
        fd2 = _fd(model, mol.coords, 1, A, x, 1e-3, 2)
        fd5 = _fd(model, mol.coords, 1, A, x, 1e-3, 5)
        assert g[A, x] == pytest.approx(fd2, rel=1e-5, abs=1e-8)
        assert g[A, x] == pytest.approx(fd5, rel=1e-7, abs=1e-10)


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
    for (A, x) in [(0, 0), (60, 1)]:
        fd = _fd(model, mol.coords, 0, A, x, 1e-3, 2)
        assert g[A, x] == pytest.approx(fd, rel=1e-4, abs=1e-6)
    out = model.solve(torch.as_tensor(mol.coords))
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy, mol.nocc)
    ref = orc.gradients([0], out[1][:1], out[2][:1], atoms=[60])[0]
    assert np.max(np.abs(g[60] - ref[60])) <= 1e-5
