"""The double-FP32 GEMM behind the mixed form's subspace products.

Stated error: |C - (alpha A op(B) + beta C0)| <= 3e-11 sum_k |A_ik| |op(B)_kj|
per element (the compensated dot product's bound over runs of 32 terms,
see ris_debug_gemm_ff), for operands inside the FP32 exponent range.  The
reference is an FP64 product summed pairwise term by term (numpy's pairwise
summation: error about log2(K) 2^-53 of sum |a b|, far below the bound),
not a BLAS call whose own rounding (K 2^-53) would reach the bound at long K.
"""
import numpy as np
import pytest

gpu = pytest.mark.gpu
BOUND = 3e-11


@pytest.fixture(scope="module")
def ris_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    return ris


def _reference(A, Bt):
    """sum_k A[i,k] Bt[j,k] by pairwise summation of the FP64 products, and
    sum_k |A[i,k] Bt[j,k]|."""
    M, N = A.shape[0], Bt.shape[0]
    C = np.empty((M, N))
    S = np.empty((M, N))
    for i in range(M):
        P = A[i][None, :] * Bt
        C[i] = P.sum(axis=1)
        S[i] = np.abs(P).sum(axis=1)
    return C, S


def _check(ris_mod, M, N, K, transB, alpha=1.0, beta=0.0, scale=None, seed=0, kind=None):
    rng = np.random.default_rng(seed + M + 3 * N + 7 * K)
    A = rng.standard_normal((M, K))
    Bt = rng.standard_normal((N, K))
    if scale is not None:
        A *= 10.0 ** rng.uniform(-scale, scale, A.shape)
        Bt *= 10.0 ** rng.uniform(-scale, scale, Bt.shape)
    C0 = rng.standard_normal((M, N))
    B = Bt if transB else np.ascontiguousarray(Bt.T)
    C, kd = ris_mod.debug_gemm_ff(A, B, transB=transB, alpha=alpha, beta=beta, C=C0)
    if kind is not None:
        assert kd == kind
    ref, S = _reference(A, Bt)
    ref = alpha * ref + beta * C0
    err = np.abs(C - ref)
    bound = BOUND * abs(alpha) * S + 4e-16 * (np.abs(ref) + abs(beta) * np.abs(C0))
    rel = float(np.max(err / (abs(alpha) * S)))
    print(f"\nff gemm {M}x{N}x{K} transB={transB} kind={kd}: max err / sum|ab| {rel:.1e}")
    assert np.all(err <= bound)
    return rel


@gpu
@pytest.mark.parametrize("M,N,K,transB", [
    (10, 90, 31311, True),     # projections T V^T over nocc*nvir (C20H22)
    (10, 102, 31311, False),   # X B^J
    (1, 1, 512, True), (32, 512, 700, True), (7, 33, 100003, False), (18, 18, 4097, True),
    (3, 129, 600, False)])
def test_long_k(ris_mod, M, N, K, transB):
    _check(ris_mod, M, N, K, transB, kind=1)


@gpu
@pytest.mark.parametrize("M,N,K,transB", [
    (10, 31311, 80, False),    # Ritz vectors S V
    (10, 31311, 102, True),    # (X B^J) B^J^T
    (1, 128, 1, False), (32, 1000, 256, True), (20, 4097, 33, False), (13, 300, 255, True),
    (2, 130, 7, True)])
def test_short_k(ris_mod, M, N, K, transB):
    _check(ris_mod, M, N, K, transB, kind=2)


@gpu
def test_alpha_beta_and_dynamic_range(ris_mod):
    # T -= Cc V form and Coulomb scaling; operands spanning 1e-12 .. 1e12
    _check(ris_mod, 10, 5000, 80, False, alpha=-1.0, beta=1.0, kind=2)
    _check(ris_mod, 10, 90, 20000, True, alpha=2.0, beta=-0.5, kind=1)
    _check(ris_mod, 8, 64, 3000, True, scale=12, kind=1)
    _check(ris_mod, 8, 640, 64, False, scale=12, kind=2)


@gpu
def test_typical_error_near_fp64(ris_mod):
    """Random operands sit far below the worst-case bound: the error is at
    the level of an FP64 product (u^2 per term of the pair arithmetic)."""
    rel = _check(ris_mod, 10, 90, 31311, True, seed=5, kind=1)
    assert rel <= 1e-13
    rel = _check(ris_mod, 10, 31311, 80, False, seed=5, kind=2)
    assert rel <= 1e-13


@gpu
def test_unhandled_shapes_rejected(ris_mod):
    A = np.ones((33, 600))
    with pytest.raises(ris_mod.RisError):
        ris_mod.debug_gemm_ff(A, np.ones((10, 600)), transB=True)   # M > 32
    with pytest.raises(ris_mod.RisError):
        ris_mod.debug_gemm_ff(np.ones((4, 300)), np.ones((10, 300)), transB=True)  # 256 < K < 512
