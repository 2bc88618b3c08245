"""FP64-emulating tensor-core GEMM (exact operand splitting into FP16 digit
slices) against an extended-precision reference, and the mixed form's
Coulomb B build that runs on it.

Bound per element (ten 6-bit slices per row frame, frames 2^E with
max_k|x_rk| < 2^E <= 2 max_k|x_rk|, products of order > 11 dropped):
    |C - C_ref| <= K 2^-52 max_k|A_rk| max_k|B_ck| + 2^-51 |C_ref|,
which holds with room (the truncation terms sum to about K 2^-56 of the
frames' product), plus a few subnormal steps for results that underflow;
FP64 GEMM itself sits near K 2^-53 sum_k |A_rk B_ck|.
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


def _ref(A, B):
    """A B^T in extended precision (long double), rounded to FP64."""
    return (A.astype(np.longdouble) @ B.astype(np.longdouble).T).astype(np.float64)


def _check(C, A, B):
    ref = _ref(A, B)
    K = A.shape[1]
    tiny = np.nextafter(0.0, 1.0)  # results in the subnormal range keep absolute steps of this
    bound = (K * 2.0 ** -52 * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
             + 2.0 ** -51 * np.abs(ref) + 4 * tiny)
    assert np.all(np.abs(C - ref) <= bound), float(np.max(np.abs(C - ref) / np.maximum(bound, 1e-300)))


def _scaled(rng, rows, K, span):
    X = rng.standard_normal((rows, K))
    X *= 10.0 ** rng.uniform(-span, span, size=(rows, 1))   # row frames far apart
    X *= 10.0 ** rng.uniform(-3, 0, size=(1, K))            # and a range inside each row
    return X


@gpu
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (127, 17, 15), (129, 48, 16), (300, 49, 17),
                                   (200, 71, 512), (130, 96, 513), (260, 441, 1100)])
def test_emulated_gemm_within_bound(ris_mod, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = _scaled(rng, M, K, 100)
    B = _scaled(rng, N, K, 100)
    _check(ris_mod.debug_gemm_f64emu(A, B), A, B)


@gpu
def test_emulated_gemm_exact_cancellation_and_special_rows(ris_mod):
    rng = np.random.default_rng(3)
    K = 96
    A = rng.standard_normal((160, K))
    A[5] = 0.0                                     # zero row
    A[6] *= 1e-300                                 # row of tiny values
    A[7, :] = 0.0
    A[7, 3] = 5e-324                               # one subnormal
    B = rng.standard_normal((40, K)) * 1e10
    # rows whose products cancel exactly: a . [x, -x] with a = [y, y]
    A[10, : K // 2] = A[10, K // 2:]
    B[11, K // 2:] = -B[11, : K // 2]
    C = ris_mod.debug_gemm_f64emu(A, B)
    assert np.all(C[5] == 0.0)
    assert C[10, 11] == 0.0
    _check(C, A, B)


@gpu
def test_emulated_gemm_beats_tf32x3_on_cancelling_sums(ris_mod):
    """Large terms that cancel to a small result: the three-pass TF32 product
    (FP32 accumulation) loses it, the emulation keeps FP64 accuracy."""
    rng = np.random.default_rng(11)
    K = 256
    A = rng.standard_normal((128, K))
    B = rng.standard_normal((32, K))
    B -= (B @ A[:1].T) / (A[0] @ A[0]) * A[:1]     # rows of B orthogonal to A[0]
    ref = _ref(A, B)
    emu = ris_mod.debug_gemm_f64emu(A, B)
    tf = ris_mod.debug_gemm_tf32x3(A, B)
    err_emu = np.abs(emu[0] - ref[0]).max()
    err_tf = np.abs(tf[0] - ref[0]).max()
    assert err_emu <= K * 2.0 ** -52 * np.abs(A[0]).max() * np.abs(B).max()
    assert err_emu * 1e6 < err_tf


def _ctx(ris_mod, mol, **opt):
    c = ris_mod.Context(**opt)
    c.build_aux(mol.coords, mol.shells, mol.aux_j, mol.aux_k)
    c.build_B(mol.C, mol.mo_energy, mol.nocc)
    return c


@gpu
def test_mixed_coulomb_build_matches_oracle(ris_mod, oracle):
    """Without exchange (c_x = 0) the mixed A X differs from FP64 only
    through the Coulomb B build, which is then FP64-accurate."""
    mol = synth.workload(0)
    orc = oracle.RisOracle(mol.coords, mol.shells, mol.aux_j, mol.aux_k, mol.C, mol.mo_energy,
                           mol.nocc, cx=0.0)
    X = synth.random_amplitudes(3, mol.nocc, mol.nvir, seed=5)
    ref = orc.apply_A(X)
    for emu, tol in ((1, 1e-11), (0, 1e-12)):
        got = _ctx(ris_mod, mol, precision=ris_mod.MIXED, cx=0.0, emu_f64=emu).apply(X)
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@gpu
def test_mixed_coulomb_build_c20h22_fp64_accurate(ris_mod):
    """C20H22 (heavy cancellation in the MO transforms of the J integrals):
    the emulated build reproduces the FP64 build to FP64 rounding level."""
    mol = synth.workload(1)
    X = synth.random_amplitudes(3, mol.nocc, mol.nvir, seed=6)
    ref = _ctx(ris_mod, mol, cx=0.0).apply(X)
    got = _ctx(ris_mod, mol, precision=ris_mod.MIXED, cx=0.0).apply(X)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
