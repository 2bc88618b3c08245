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


@gpu
@pytest.mark.parametrize("m,k", [(1, 1), (2, 2), (5, 3), (18, 10), (80, 20), (150, 20), (200, 12)])
def test_sym_eig_lowest_fp32_form(ris_mod, m, k):
    """FP32 eigensolver of the mixed form: residuals at FP32 level of ||H||,
    FP64 Rayleigh quotients (eigenvalue error ~ residual^2 / gap), unit
    vectors, near-orthogonality of the FP32 vectors."""
    rng = np.random.default_rng(m + 100)
    d = np.sort(np.concatenate([0.27 + 0.02 * rng.random(min(m, 12)), 0.3 + 2 * rng.random(max(m - 12, 0))]))
    Q = rng.standard_normal((m, m)) * 1e-3
    H = np.diag(d) + 0.5 * (Q + Q.T)
    w, V = ris_mod.debug_sym_eig(H, k, fp32=True)
    wr, Vr = np.linalg.eigh(H)
    hn = np.max(np.abs(wr))
    res = H @ V.T - V.T * w[None, :]
    assert np.max(np.abs(res)) < 2e-6 * hn
    np.testing.assert_allclose(w, wr[:k], rtol=0, atol=1e-9)
    G = V @ V.T
    np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-12)
    assert np.max(np.abs(G - np.eye(k))) < 1e-3


@gpu
def test_sym_eig_fp32_form_degenerate_pair(ris_mod):
    """An exactly degenerate pair and a pair 1e-6 apart: orthonormal vectors
    spanning the right spaces, Ritz values in FP64."""
    rng = np.random.default_rng(5)
    m = 40
    d = np.concatenate([[0.3, 0.3, 0.5, 0.5 + 1e-6], 0.8 + rng.random(m - 4)])
    Qm, _ = np.linalg.qr(rng.standard_normal((m, m)))
    H = (Qm * d) @ Qm.T
    H = 0.5 * (H + H.T)
    w, V = ris_mod.debug_sym_eig(H, 6, fp32=True)
    np.testing.assert_allclose(w[:4], d[:4], rtol=0, atol=1e-9)
    G = V @ V.T
    np.testing.assert_allclose(G[:2, :2], np.eye(2), atol=1e-12)   # within each cluster: FP64
    np.testing.assert_allclose(G[2:4, 2:4], np.eye(2), atol=1e-12)
    assert np.max(np.abs(G - np.eye(6))) < 1e-4                     # across: FP32 level
    for a, b in ((0, 2), (2, 4)):                                   # the right eigenspaces
        P = Qm[:, a:b] @ Qm[:, a:b].T
        assert np.max(np.abs(P @ V[a:b].T - V[a:b].T)) < 1e-5
    res = H @ V.T - V.T * w[None, :]
    assert np.max(np.abs(res)) < 2e-6 * np.max(np.abs(d))


# Shapes cover every tile family (8..64 rows, 16..128 columns), ragged edges,
# split k (few tiles, long k) and all four transposes.
_GEMM_SHAPES = [(1, 1, 1), (3, 5, 7), (10, 80, 31000), (10, 31000, 80), (71, 5000, 512),
                (80, 10, 4000), (16, 16, 16), (17, 33, 65), (64, 64, 1), (130, 257, 300),
                (8, 128, 2000), (5, 2, 100000)]


@gpu
@pytest.mark.parametrize("m,n,k", _GEMM_SHAPES)
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
def test_dgemm_shapes(ris_mod, m, n, k, ta, tb):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C0 = rng.standard_normal((m, n))
    alpha, beta = 0.75, -1.25
    got = ris_mod.debug_dgemm(A, B, C0, ta, tb, alpha, beta)
    ref = alpha * ((A.T if ta else A) @ (B.T if tb else B)) + beta * C0
    # FP64 sums of k products of unit normals: error ~ sqrt(k) eps per entry
    scale = np.sqrt(k) * (np.abs(alpha) + 1) + abs(beta) * np.abs(C0)
    assert np.max(np.abs(got - ref) / scale) <= 1e-13


@gpu
def test_dgemm_beta_zero_ignores_nan(ris_mod):
    A = np.ones((9, 40))
    B = np.ones((40, 11))
    C0 = np.full((9, 11), np.nan)
    got = ris_mod.debug_dgemm(A, B, C0, False, False, 1.0, 0.0)
    np.testing.assert_array_equal(got, np.full((9, 11), 40.0))
