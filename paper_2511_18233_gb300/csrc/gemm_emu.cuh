// FP64-accurate matrix products on the FP16 tensor cores of sm_103a by exact
// splitting of the operands into small-integer slices (Ozaki's scheme).
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace ris {

// Slicing: bits per slice and slices per operand.  A row r of an operand
// (contraction index k) is written in one fixed-point frame per row,
//   x_rk = 2^(E_r) * sum_{p=1..kEmuSlices} d_p(r,k) 2^(-kEmuBeta p),
// |d_p| < 2^kEmuBeta, E_r set by the row's largest magnitude; the digits
// are the first kEmuSlices * kEmuBeta bits of x_rk in that frame.
constexpr int kEmuBeta = 6;
constexpr int kEmuSlices = 10;
// Largest contraction length of one tensor-core pass: a sum of eight digit
// products over K stays below 2^24 (K * 63^2 * 8 < 2^24), so it is exact in
// the FP32 accumulators.  Longer contractions run as several passes.
constexpr int kEmuKChunk = 512;

// A sliced operand: digits as FP16 integers [kEmuSlices][rows][ldk] (K
// contiguous, ldk % 8 == 0, zero past K) and the row exponents E[rows].
struct EmuOperand {
  __half* s = nullptr;
  int* e = nullptr;
  int rows = 0, K = 0, ldk = 0;
};

// Slices src with element (r, k) at src[r * rs + k * ks], r < rows, k < K,
// into op (op.s / op.e must hold kEmuSlices * rows * ldk halves and rows
// ints; ldk = ld8(K)).
void emu_slice(const double* src, int rows, int K, long long rs, long long ks, EmuOperand& op,
               cudaStream_t st);

// Output placement: element (r, c) goes to
//   c64[(r / rin) * rld + (r % rin) * rs + (c / cin) * cld + (c % cin) * cs]
// (rin, cin = 0: no blocking), as alpha * (A B^T)_rc + beta * c64[...].
struct EmuEpilogue {
  double* c64 = nullptr;
  int rin = 0, cin = 0;
  long long rld = 0, rs = 0, cld = 0, cs = 1;
  double alpha = 1.0, beta = 0.0;
};

// C (M x N) = A (M x K) . B (N x K)^T from sliced operands; *d_err (device
// int) is set non-zero if a pipeline wait timed out.
void emu_gemm(int M, int N, const EmuOperand& A, const EmuOperand& B, const EmuEpilogue& ep,
              int* d_err, cudaStream_t st);

inline int ld8(int k) { return (k + 7) & ~7; }

}  // namespace ris
