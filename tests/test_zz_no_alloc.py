"""The allocation-free GEMM entry point, for callers that cannot allocate
device memory at the point of the call: its output must match the
allocating entry point's on two calls in a row, it must reject problems
larger than its preallocated scratch, and repeated calls must not change
the device's free memory."""
import numpy as np
import pytest


@pytest.mark.gpu
def test_noalloc_gemm_matches_allocating_entry():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18233_gb300 import build, ris
    build.build()
    rng = np.random.default_rng(2024)
    cases = [(300, 200, 1000), (1278, 441, 700)]
    for M, N, K in cases:  # two calls in a row, on different data
        A = rng.standard_normal((M, K))
        B = rng.standard_normal((N, K))
        ref = ris.debug_gemm_tf32x3(A, B)
        A_t = torch.as_tensor(A, device="cuda")
        B_t = torch.as_tensor(B, device="cuda")
        C_t = torch.full((M, N), np.nan, dtype=torch.float64, device="cuda")
        assert ris.gemm_tf32x3_noalloc(A_t, B_t, C_t) == 0
        C = C_t.cpu().numpy()
        bound = np.abs(A) @ np.abs(B).T
        assert np.max(np.abs(C - ref) / bound) <= 2e-6
        assert np.max(np.abs(C - A @ B.T) / bound) <= 2e-6
    # the split-K case above (M = 300, N = 200: six tiles, K split across CTAs)
    # and repeated calls allocate nothing: the library's allocation counter
    # does not move
    A_t = torch.as_tensor(rng.standard_normal((300, 1000)), device="cuda")
    B_t = torch.as_tensor(rng.standard_normal((200, 1000)), device="cuda")
    C_t = torch.empty((300, 200), dtype=torch.float64, device="cuda")
    n0 = ris.debug_alloc_count()
    for _ in range(2):
        assert ris.gemm_tf32x3_noalloc(A_t, B_t, C_t) == 0
    assert ris.debug_alloc_count() == n0
    # misuse is caught before the call: wrong dtype, transposed view, shape
    with pytest.raises(ValueError):
        ris.gemm_tf32x3_noalloc(A_t.float(), B_t, C_t)
    with pytest.raises(ValueError):
        ris.gemm_tf32x3_noalloc(A_t, B_t.t(), C_t)
    with pytest.raises(ValueError):
        ris.gemm_tf32x3_noalloc(A_t, B_t, C_t[:, :100])
    # repeated calls leave the device's free memory unchanged
    A_t = torch.as_tensor(rng.standard_normal((256, 512)), device="cuda")
    B_t = torch.as_tensor(rng.standard_normal((192, 512)), device="cuda")
    C_t = torch.empty((256, 192), dtype=torch.float64, device="cuda")
    assert ris.gemm_tf32x3_noalloc(A_t, B_t, C_t) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert ris.gemm_tf32x3_noalloc(A_t, B_t, C_t) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # too large for the 8 Mi-float scratch: rejected, output untouched
    big_A = torch.zeros((4096, 1024), dtype=torch.float64, device="cuda")
    big_B = torch.zeros((4096, 1024), dtype=torch.float64, device="cuda")
    big_C = torch.full((4096, 4096), 7.0, dtype=torch.float64, device="cuda")
    assert ris.gemm_tf32x3_noalloc(big_A, big_B, big_C) == -1
    assert float(big_C[0, 0]) == 7.0
