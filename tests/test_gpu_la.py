"""Device dense linear algebra against numpy: the Davidson subspace
eigensolver (Householder + multisection + inverse iteration)."""
import numpy as np
import pytest

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
@pytest.mark.parametrize("m,k", [(1, 1), (2, 2), (5, 3), (18, 10), (80, 20), (150, 20), (200, 12)])
def test_sym_eig_lowest(ris_mod, m, k):
    rng = np.random.default_rng(m)
    # Davidson-like: clustered low diagonal, small couplings, a few large entries
    d = np.sort(np.concatenate([0.27 + 0.02 * rng.random(min(m, 12)), 0.3 + 2 * rng.random(max(m - 12, 0))]))
    Q = rng.standard_normal((m, m)) * 1e-3
    H = np.diag(d) + 0.5 * (Q + Q.T)
    w, V = ris_mod.debug_sym_eig(H, k)
    wr, Vr = np.linalg.eigh(H)
    np.testing.assert_allclose(w, wr[:k], rtol=0, atol=1e-13)
    np.testing.assert_allclose(V @ V.T, np.eye(k), atol=1e-10)
    res = H @ V.T - V.T * w[None, :]
    assert np.max(np.abs(res)) < 1e-10
