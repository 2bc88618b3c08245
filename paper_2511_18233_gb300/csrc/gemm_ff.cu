// Double-FP32 ("float-float") GEMM on the FP32 pipe.
//
// GB300 retires FP32 fused multiply-adds about 72 times faster than FP64
// ones (76 against 1.06 TFLOP/s measured on this part), so a product whose
// operands and sums are carried as pairs of FP32 numbers runs several times
// faster than on the FP64 pipe while keeping close to FP64 accuracy.  The
// mixed form uses it for skinny products of its Davidson iterations that the
// FP64 pipe bounds: the Ritz vectors S V and S (A V) over the nocc*nvir index
// and the Coulomb part 2 (X B^J) B^J^T of the Davidson product (the
// orthogonalisation and the projected matrix stay FP64).
//
// Arithmetic (all FP32 operations round to nearest and are never contracted):
// * Split.  An FP64 element x becomes hi + lo with hi its leading 24
//   significand bits and lo the next 29 rounded to 24, by integer operations
//   on the bit pattern (no FP64 instruction); |x - hi - lo| <= 2^-47 |x|
//   for |x| >= 2^-74 (below, lo is dropped: error < 2^-97); |x| < 2^-126
//   flushes to zero and |x| >= 2^128 becomes +-inf.
// * Term.  a*b ~ ah*bh + (ah*bl + al*bh) (al*bl < 2^-46 |a b| dropped).  The
//   leading product is made exact as p + e with an FMA (e = ah*bh - p, the
//   "TwoProduct" of Dekker 1971); p is added to the running sum s by Knuth's
//   TwoSum, whose exact rounding error q goes, with e and the cross terms, to
//   a second accumulator c.  This is the compensated dot product "Dot2" of
//   Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005), fed split inputs.
// * Bounds.  Dot2's error over a run of L terms is at most about (L u)^2
//   times sum |a b| (u = 2^-24).  The row kernel renormalises (s, c) by
//   TwoSum every 32 terms and has k <= 256 (error <= 256 * 32 u^2 ~ 2.9e-11
//   of sum |a b|); the long-k kernel restarts (s, c) every 32 terms and adds
//   each run into a second pair (S, C) by float-float addition (error about
//   (32 u)^2 ~ 3.6e-12 of sum |a b| plus u^2 per run).  With the split
//   truncation (2^-46) the result is within 3e-11 sum_k |a_ik b_kj|.
// * Output.  The pair is widened to FP64 by integer operations and added in
//   FP64; alpha and beta are applied in FP64.
//
// Two kernels cover the shapes the subspace iterations need:
// * k_ff_rows (k <= 256, n large, m <= 32): a CTA owns 32 output columns,
//   its four warps split k and combine through shared memory; A is split
//   once per CTA into shared memory (broadcast reads), B is streamed once.
// * k_ff_long (k large, m <= 32, n <= 512): warp w of a CTA owns output rows
//   w, w + 8, ... and each lane TN columns; k is cut into chunks over CTAs, 32-deep
//   slices of A and B are split into shared memory, and every chunk writes
//   its (S, C) pairs; k_ff_reduce adds the chunks in a fixed order (the
//   result does not depend on scheduling).
#include "gemm_ff.cuh"
#include "ff_arith.cuh"

#include <algorithm>

namespace ris {

namespace {

__device__ __forceinline__ void ff_store(double* p, float s, float c, double alpha, double beta) {
  const double y = ff_widen(s) + ff_widen(c);
  *p = beta == 0.0 ? alpha * y : fma(alpha, y, beta * *p);
}

}  // namespace

// ------------------------------------------------------------------ short k
constexpr int kRowsKG = 4;  // warps per CTA, each a quarter of k

// Shared memory: A split [k][RM] (float2); with TB the CTA's 32 rows of B
// split and transposed, hi and lo [k][33]; the k-group partial sums
// [kRowsKG - 1][RM][32] (float2).
inline size_t rows_smem(int RM, bool TB, int k) {
  return (size_t)k * RM * 8 + (TB ? (size_t)k * 33 * 8 : 0) + (size_t)(kRowsKG - 1) * RM * 32 * 8;
}

template <int RM, bool TB>
__global__ void __launch_bounds__(32 * kRowsKG) k_ff_rows(int m, int n, int k, double alpha,
                                                          const double* __restrict__ A, int lda,
                                                          const double* __restrict__ B, int ldb,
                                                          double beta, double* __restrict__ C,
                                                          int ldc) {
  extern __shared__ float2 ff_sh[];
  float2* sA = ff_sh;
  float* sBh = (float*)(sA + (size_t)k * RM);
  float* sBl = sBh + (TB ? (size_t)k * 33 : 0);
  float2* sR = (float2*)(sBl + (TB ? (size_t)k * 33 : 0));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j0 = blockIdx.x * 32, j = j0 + lane;
  for (int e = threadIdx.x; e < k * RM; e += 32 * kRowsKG) {
    const int kk = e / RM, r = e - kk * RM;
    float h = 0.f, l = 0.f;
    if (r < m) ff_split(A[(size_t)r * lda + kk], h, l);
    sA[e] = make_float2(h, l);
  }
  if (TB) {
    // consecutive threads read consecutive k of one row of B (coalesced),
    // four loads in flight per thread before the splits
    constexpr int NT = 32 * kRowsKG;
    for (int e0 = threadIdx.x; e0 < 32 * k; e0 += 4 * NT) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = e0 + u * NT;
        const int jj = e / k, kk = e - jj * k;
        v[u] = e < 32 * k && j0 + jj < n ? B[(size_t)(j0 + jj) * ldb + kk] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = e0 + u * NT;
        const int jj = e / k, kk = e - jj * k;
        float h, l;
        ff_split(v[u], h, l);
        if (e < 32 * k) {
          sBh[kk * 33 + jj] = h;
          sBl[kk * 33 + jj] = l;
        }
      }
    }
  }
  __syncthreads();
  const int kper = (k + kRowsKG - 1) / kRowsKG;
  const int kb = min(k, w * kper), ke = min(k, kb + kper);
  float s[RM], c[RM];
#pragma unroll
  for (int r = 0; r < RM; r++) s[r] = c[r] = 0.f;
  if (TB || j < n) {
    for (int k0 = kb; k0 < ke; k0 += 32) {
      const int k1 = min(ke, k0 + 32);
#pragma unroll 4
      for (int kk = k0; kk < k1; kk++) {
        float bh, bl;
        if (TB) {
          bh = sBh[kk * 33 + lane];
          bl = sBl[kk * 33 + lane];
        } else {
          ff_split(B[(size_t)kk * ldb + j], bh, bl);
        }
        const float2* a = sA + (size_t)kk * RM;
#pragma unroll
        for (int r = 0; r < RM; r++) ff_term(a[r].x, a[r].y, bh, bl, s[r], c[r]);
      }
#pragma unroll
      for (int r = 0; r < RM; r++) ff_renorm(s[r], c[r]);
    }
  }
  if (w > 0) {
#pragma unroll
    for (int r = 0; r < RM; r++) sR[((w - 1) * RM + r) * 32 + lane] = make_float2(s[r], c[r]);
  }
  __syncthreads();
  if (w == 0 && j < n) {
#pragma unroll
    for (int g = 0; g < kRowsKG - 1; g++)
#pragma unroll
      for (int r = 0; r < RM; r++) {
        const float2 v = sR[(g * RM + r) * 32 + lane];
        ff_add(s[r], c[r], v.x, v.y);
      }
#pragma unroll
    for (int r = 0; r < RM; r++)
      if (r < m) ff_store(C + (size_t)r * ldc + j, s[r], c[r], alpha, beta);
  }
}

// ------------------------------------------------------------------ long k
// Grid (n tiles of 32*TN columns, k chunks); CTA of 256 threads: warp w owns
// output rows w, w + 8, ... (RW of them, m <= 8 RW), each lane TN columns,
// so that all eight warps stage the operands whatever m is.  ws[chunk][m][n]
// receives the chunk's (S, C) pairs.
constexpr int kLongT = 256;
template <int TN, int RW, bool TB>
__global__ void __launch_bounds__(kLongT) k_ff_long(int m, int n, int k, int kchunk,
                                                    const double* __restrict__ A, int lda,
                                                    const double* __restrict__ B, int ldb,
                                                    float2* __restrict__ ws) {
  constexpr int BN = 32 * TN;
  __shared__ float2 sA[32][33];      // [k][row]
  __shared__ float sBh[32][BN + 1];  // [k][column]
  __shared__ float sBl[32][BN + 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = blockIdx.x * BN;
  const int kb = blockIdx.y * kchunk, ke = min(k, kb + kchunk);
  float S[RW][TN], Cc[RW][TN];
#pragma unroll
  for (int i = 0; i < RW; i++)
#pragma unroll
    for (int t = 0; t < TN; t++) S[i][t] = Cc[i][t] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += 32) {
    const int kn = min(32, ke - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < m * 32; e += kLongT) {
      const int rr = e >> 5, kk = e & 31;
      float h = 0.f, l = 0.f;
      if (kk < kn) ff_split(A[(size_t)rr * lda + k0 + kk], h, l);
      sA[kk][rr] = make_float2(h, l);
    }
    // B: four loads in flight per thread before the splits
    for (int e0 = threadIdx.x; e0 < BN * 32; e0 += 4 * kLongT) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = e0 + u * kLongT;
        int jj, kk;
        if (TB) {  // B [n][k]: consecutive threads along k
          jj = e >> 5;
          kk = e & 31;
        } else {   // B [k][n]: consecutive threads along n
          kk = e / BN;
          jj = e - kk * BN;
        }
        v[u] = 0.0;
        if (e < BN * 32 && kk < kn && c0 + jj < n)
          v[u] = TB ? B[(size_t)(c0 + jj) * ldb + k0 + kk] : B[(size_t)(k0 + kk) * ldb + c0 + jj];
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = e0 + u * kLongT;
        const int jj = TB ? e >> 5 : e % BN, kk = TB ? e & 31 : e / BN;
        float h, l;
        ff_split(v[u], h, l);
        if (e < BN * 32) {
          sBh[kk][jj] = h;
          sBl[kk][jj] = l;
        }
      }
    }
    __syncthreads();
    float s[RW][TN], c[RW][TN];
#pragma unroll
    for (int i = 0; i < RW; i++)
#pragma unroll
      for (int t = 0; t < TN; t++) s[i][t] = c[i][t] = 0.f;
#pragma unroll 2
    for (int kk = 0; kk < 32; kk++) {  // rows past kn are zero
      float bh[TN], bl[TN];
#pragma unroll
      for (int t = 0; t < TN; t++) {
        bh[t] = sBh[kk][lane + 32 * t];
        bl[t] = sBl[kk][lane + 32 * t];
      }
#pragma unroll
      for (int i = 0; i < RW; i++) {
        if (w + 8 * i < m) {  // warp-uniform
          const float2 a = sA[kk][w + 8 * i];
#pragma unroll
          for (int t = 0; t < TN; t++) ff_term(a.x, a.y, bh[t], bl[t], s[i][t], c[i][t]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < RW; i++)
#pragma unroll
      for (int t = 0; t < TN; t++) ff_add(S[i][t], Cc[i][t], s[i][t], c[i][t]);
  }
#pragma unroll
  for (int i = 0; i < RW; i++) {
    const int r = w + 8 * i;
#pragma unroll
    for (int t = 0; t < TN; t++) {
      const int col = c0 + lane + 32 * t;
      if (r < m && col < n) ws[((size_t)blockIdx.y * m + r) * n + col] = make_float2(S[i][t], Cc[i][t]);
    }
  }
}

// C = alpha * sum_chunk ws[chunk] + beta * C, chunks added in order by eight
// warps (warp g takes chunks g, g + 8, ...), then the eight in order.
__global__ void __launch_bounds__(256) k_ff_reduce(int m, int n, int nchunk,
                                                   const float2* __restrict__ ws, double alpha,
                                                   double beta, double* __restrict__ C, int ldc) {
  __shared__ float2 red[8][32];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const long long mn = (long long)m * n;
  const long long o = (long long)blockIdx.x * 32 + lane;
  float S = 0.f, Cc = 0.f;
  if (o < mn)
    for (int z = g; z < nchunk; z += 8) {
      const float2 v = ws[(size_t)z * mn + o];
      ff_add(S, Cc, v.x, v.y);
    }
  red[g][lane] = make_float2(S, Cc);
  __syncthreads();
  if (g == 0 && o < mn) {
#pragma unroll
    for (int h = 1; h < 8; h++) ff_add(S, Cc, red[h][lane].x, red[h][lane].y);
    const int i = (int)(o / n), j = (int)(o % n);
    ff_store(C + (size_t)i * ldc + j, S, Cc, alpha, beta);
  }
}

// ------------------------------------------------------------------ dispatch
namespace {

constexpr int kRowsRM[] = {2, 4, 6, 8, 10, 12, 16, 20, 24, 32};

template <int RM, bool TB>
void launch_rows(int m, int n, int k, double alpha, const double* A, int lda, const double* B,
                 int ldb, double beta, double* C, int ldc, cudaStream_t st) {
  const size_t smem = rows_smem(RM, TB, k);
  ensure_smem_attr((const void*)k_ff_rows<RM, TB>, (int)rows_smem(RM, TB, 256));
  k_ff_rows<RM, TB><<<cdiv(n, 32), 32 * kRowsKG, smem, st>>>(m, n, k, alpha, A, lda, B, ldb, beta,
                                                             C, ldc);
}

template <bool TB>
void rows_dispatch(int m, int n, int k, double alpha, const double* A, int lda, const double* B,
                   int ldb, double beta, double* C, int ldc, cudaStream_t st) {
#define RIS_FF_RM(R)                                                                  \
  if (m <= R) return launch_rows<R, TB>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st);
  RIS_FF_RM(2) RIS_FF_RM(4) RIS_FF_RM(6) RIS_FF_RM(8) RIS_FF_RM(10) RIS_FF_RM(12)
  RIS_FF_RM(16) RIS_FF_RM(20) RIS_FF_RM(24) RIS_FF_RM(32)
#undef RIS_FF_RM
}

template <int TN, int RW, bool TB>
void launch_long(dim3 grid, int m, int n, int k, int kchunk, const double* A, int lda,
                 const double* B, int ldb, float2* ws, cudaStream_t st) {
  k_ff_long<TN, RW, TB><<<grid, kLongT, 0, st>>>(m, n, k, kchunk, A, lda, B, ldb, ws);
}

template <int TN, bool TB>
void long_rows(dim3 grid, int m, int n, int k, int kchunk, const double* A, int lda,
               const double* B, int ldb, float2* ws, cudaStream_t st) {
  if (m <= 8) return launch_long<TN, 1, TB>(grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
  if (m <= 16) return launch_long<TN, 2, TB>(grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
  return launch_long<TN, 4, TB>(grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
}

template <bool TB>
void long_dispatch(int tn, dim3 grid, int m, int n, int k, int kchunk, const double* A, int lda,
                   const double* B, int ldb, float2* ws, cudaStream_t st) {
  if (tn == 1) return long_rows<1, TB>(grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
  if (tn == 2) return long_rows<2, TB>(grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
  if (tn == 3) return long_rows<3, TB>(grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
  return long_rows<4, TB>(grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
}

}  // namespace

int ffgemm_kind(bool transA, int m, int n, int k) {
  if (transA || m < 1 || m > 32 || n < 1 || k < 1) return 0;
  if (k <= 256 && n >= 128) return 2;
  if (k >= 512 && n <= 512) return 1;
  return 0;
}

bool ffgemm(bool transA, bool transB, int m, int n, int k, double alpha, const double* A, int lda,
            const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t st) {
  const int kind = ffgemm_kind(transA, m, n, k);
  if (kind == 0) return false;
  prof_begin(kProfFF, st);
  if (kind == 2) {
    if (transB)
      rows_dispatch<true>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st);
    else
      rows_dispatch<false>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st);
    RIS_CHECK_LAUNCH();
  } else {
    const int tn = std::min(4, cdiv(n, 32));
    const int ntile = cdiv(n, 32 * tn);
    // about two CTAs per SM, chunks of at least 64 k
    const int want = std::max(1, cdiv(2 * 152, ntile));
    int kchunk = std::max(64, ((cdiv(k, want) + 31) / 32) * 32);
    const int nchunk = cdiv(k, kchunk);
    MemTrack* tr = nullptr;
    const size_t wsb = sizeof(float2) * (size_t)nchunk * m * n;
    float2* ws = (float2*)dev_alloc(wsb, st, &tr);
    const dim3 grid((unsigned)ntile, (unsigned)nchunk);
    if (transB)
      long_dispatch<true>(tn, grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
    else
      long_dispatch<false>(tn, grid, m, n, k, kchunk, A, lda, B, ldb, ws, st);
    RIS_CHECK_LAUNCH();
    k_ff_reduce<<<cdiv((long long)m * n, 32), 256, 0, st>>>(m, n, nchunk, ws, alpha, beta, C, ldc);
    RIS_CHECK_LAUNCH();
    dev_free(ws, wsb, st, tr);
  }
  prof_end(kProfFF, st, 2.0 * m * n * (double)k);
  return true;
}

}  // namespace ris

extern "C" int ris_debug_gemm_ff(int transB, int M, int N, int K, double alpha, const double* A,
                                 const double* B, double beta, double* C, int* kind) {
  using namespace ris;
  try {
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return (int)RIS_ERR_ARG;
    const int kd = ffgemm_kind(false, M, N, K);
    if (kind) *kind = kd;
    if (kd == 0) return (int)RIS_ERR_ARG;
    cudaStream_t st = 0;
    ffgemm(false, transB != 0, M, N, K, alpha, A, K, B, transB ? K : N, beta, C, N, st);
    RIS_CUDA(cudaStreamSynchronize(st));
    return 0;
  } catch (const Error& e) {
    fprintf(stderr, "ris_debug_gemm_ff: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}
