// 3xTF32 tensor-core GEMM for sm_103a (tcgen05 + TMA), used by the mixed
// precision form of the ris contractions.
#pragma once
#include "common.cuh"

namespace ris {

// Operand in FP32 storage, split a = hi + lo with hi = tf32(a) and
// lo = tf32(a - hi), both stored as FP32 bit patterns.  Row-major [rows][ld]
// with the contraction index K contiguous (K-major); ld % 4 == 0 and the
// pointers 16-byte aligned (TMA).  Optional batch: rows of batch z start at
// z * bstride elements (bstride % 4 == 0); nb = 1 means shared.
struct TcOperand {
  const float* hi = nullptr;
  const float* lo = nullptr;
  int rows = 0, ld = 0;
  long long bstride = 0;
  int nb = 1;
};

// Epilogue: element (i, j) of batch z, i < M, j < N, is stored at
//   z * bsc + rpos(i) + cpos(j),
// rpos(i) = (i / rin) * rld + (i % rin) * rs when rin > 0 (row blocks of rin
// at stride rld), else i * rs;
// cpos(j) = (j / cin) * cld + (j % cin) * cs when cin > 0 (column blocks of
// cin at stride cld, e.g. a padded inner index), else j * cs.
//   kOutF64:   C64 = alpha * acc + beta * C64
//   kOutSplit: Chi/Clo = tf32 split of alpha * acc (FP32)
//   kOutF32:   C32 = alpha * acc + beta * C32 (FP32 arithmetic)
enum TcOut { kOutF64 = 0, kOutSplit = 1, kOutF32 = 2 };
struct TcEpilogue {
  int mode = kOutF64;
  double* c64 = nullptr;
  float* c32 = nullptr;
  float* chi = nullptr;
  float* clo = nullptr;
  long long rs = 0, cs = 1;
  long long bsc = 0;
  double alpha = 1.0, beta = 0.0;
  int cin = 0;
  long long cld = 0;
  int rin = 0;
  long long rld = 0;
};

// C[z] (M x N) = A[z] (M x K) . B[z]^T (N x K), batches z < nb.  With
// kOutF64 and nb == 1 the K range may be split across CTAs (deterministic
// two-pass reduction); with kOutF64 a K longer than 16384 runs as chunks
// whose results the epilogue sums in FP64 (the tensor core's FP32
// accumulation error grows with the number of K steps).  *d_err (device int) is set non-zero if a pipeline
// wait timed out.
// ws / ws_floats: optional caller-owned FP32 workspace for the split-K
// partial sums; with allow_alloc false the GEMM never allocates (it splits K
// only when ws is large enough).
void tc_gemm(int M, int N, int K, const TcOperand& A, const TcOperand& B, int nb,
             const TcEpilogue& ep, int* d_err, cudaStream_t st, float* ws = nullptr,
             size_t ws_floats = 0, bool allow_alloc = true);

// Split FP64 -> (hi, lo) FP32 with a row-major source [rows][cols] (leading
// dimension lds) into [rows][ldd] (padding columns zero-filled).
// nbatch matrices at source / destination batch strides sbs / dbs.
void split_f64(const double* src, int rows, int cols, long long lds, float* hi, float* lo, int ldd,
               cudaStream_t st, int nbatch = 1, long long sbs = 0, long long dbs = 0);
// Same with the source transposed: dst[c][r] = src[r][c].
void split_f64_t(const double* src, int rows, int cols, long long lds, float* hi, float* lo,
                 int ldd, cudaStream_t st, int nbatch = 1, long long sbs = 0, long long dbs = 0);

// Transpose + split: src X[r][c] (nr x nc, row-major) into dst[c][r / nin]
// [r % nin] with the innermost index padded to ldin (padding not written).
void split_f64_tpad(const double* src, long long nr, int nc, int nin, int ldin, float* hi,
                    float* lo, cudaStream_t st);

inline int ld4(int k) { return (k + 3) & ~3; }

}  // namespace ris
