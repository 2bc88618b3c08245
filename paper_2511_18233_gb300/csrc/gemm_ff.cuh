// Double-FP32 GEMM for skinny products of the mixed form's Davidson
// iterations (Ritz vectors, the Coulomb part of the Davidson product).
#pragma once
#include "common.cuh"

namespace ris {

// C (m x n) = alpha * A op(B) + beta * C, row-major FP64 in and out; A is
// [m][k] (lda), op(B) = B ([k][n], ldb) or B^T (B [n][k], ldb) per transB.
// Each product is formed from FP32 pairs (hi, lo) cut from the FP64 operands
// and accumulated as an unevaluated FP32 pair with error-free transforms on
// the FP32 pipe; error per element at most about 3e-11 sum_k |a_ik||b_kj|
// (see gemm_ff.cu).
// Handles m <= 32 with either k <= 256 and n >= 128 (one thread per output
// column) or k >= 512 and n <= 512 (k split over CTAs, fixed-order
// reduction).  Returns false, launching nothing, for any other shape or a
// transposed A; the caller then runs the FP64 GEMM.
bool ffgemm(bool transA, bool transB, int m, int n, int k, double alpha, const double* A, int lda,
            const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t st);

// Which kernel ffgemm would run for the shape: 0 none, 1 the long-k kernel,
// 2 the short-k (row) kernel.
int ffgemm_kind(bool transA, int m, int n, int k);

}  // namespace ris
