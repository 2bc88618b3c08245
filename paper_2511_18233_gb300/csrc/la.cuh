// Dense linear algebra on the device: FP64 batched GEMM, Cholesky, triangular
// inverse, small symmetric eigensolver, vector utilities.
#pragma once
#include "common.cuh"

namespace ris {

// Row-major batched GEMM: C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b],
// op(A) is m x k, op(B) is k x n.  Batch index b = b1 * nb2 + b2 with
// per-level element strides (sA1, sA2), (sB1, sB2), (sC1, sC2).
struct GemmBatch {
  int nb1 = 1, nb2 = 1;
  long long sA1 = 0, sA2 = 0, sB1 = 0, sB2 = 0, sC1 = 0, sC2 = 0;
};
void dgemm(bool transA, bool transB, int m, int n, int k, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t st,
           const GemmBatch& bt = GemmBatch());

// In place lower Cholesky of an n x n row-major SPD matrix (upper part is
// zeroed).  Writes 0 to *info on success, or j+1 if the j-th pivot is not
// above 1e-13 times the diagonal element (singular or indefinite matrix).
void cholesky(double* A, int n, int* d_info, cudaStream_t st);
// Linv = L^{-1} for lower-triangular L (n x n, row-major).
void tri_inverse(const double* L, double* Linv, int n, cudaStream_t st);

// Lowest k eigenpairs of the symmetric m x m row-major matrix H (leading
// dimension ldH; only read).
// w[k] ascending; V[k][m] (row j = eigenvector j).  work: eig_work_size(m)
// doubles.  Three launches on st.
size_t eig_work_size(int m);
void sym_eig_lowest(const double* H, int ldH, int m, int k, double* w, double* V, double* work,
                    cudaStream_t st);
// The same in FP32 arithmetic with FP64 Rayleigh quotients (residuals of a
// few FP32 ulps of ||H||; close eigenvalues' vectors orthonormalised and
// rotated onto Ritz vectors in FP64).  Returns false (nothing launched) when
// m > 200.
bool sym_eig_lowest_f32(const double* H, int ldH, int m, int k, double* w, double* V, double* work,
                        cudaStream_t st);

// Utilities
void fill(double* x, double v, size_t n, cudaStream_t st);
void row_norms(const double* X, int nrow, long long ncol, double* out, cudaStream_t st);
void gemv_rows(const double* V, int nrow, long long ncol, const double* x, double* out,
               cudaStream_t st);  // out[i] = V[i] . x

}  // namespace ris
