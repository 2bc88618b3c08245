// Dense FP64 linear algebra on the device.
//
// * dgemm: tiled FP64 GEMM (block tile from 8x32 to 64x64 fitted to the
//   problem, up to 4x4 per thread), batched over two strided levels,
//   transposes folded into the tile loads, split along k for few tiles.
// * cholesky / tri_inverse: the metric factor M = L L^T of Eq. (g_modified)
//   and L^{-1}; the factorisation on one CTA (the metric is at most a few
//   thousand functions for one molecule of the ris basis), the inverse one
//   warp per column over many CTAs.
// * sym_eig_lowest: lowest k eigenpairs of a small symmetric matrix (the
//   Davidson subspace problem): Householder reduction to tridiagonal form
//   (one CTA), then one CTA per eigenvalue for Sturm-sequence multisection,
//   inverse iteration and back-transformation (FP64 runs at about two FMAs
//   per clock per SM, so the per-eigenvalue work is spread over SMs), and
//   Gram-Schmidt inside clusters of close eigenvalues.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "la.cuh"

namespace ris {

// ------------------------------------------------------------------ GEMM
// FP64 runs at about two fused multiply-adds per clock per SM on this part,
// so the GEMM is bound by the FMA pipe alone and every padded (wasted) FMA
// costs time: the block tile is chosen per call from a family of shapes to
// fit the problem (the Davidson products have 5-40 rows), and a product with
// too few tiles is split along k to occupy all SMs.
//
// Block tile BM x BN = (THY*TM) x ((256/THY)*TN); thread (ty, tx) owns the
// TM x TN outputs (ty + THY*r, tx + THX*c).
constexpr int kBK = 16;

// With ksplit > 1 (single batch only) blockIdx.z selects a slice of k of
// length kchunk and the raw partial product is written to C + z*m*n
// (ldc = n); k_splitk_reduce then forms alpha*sum + beta*C in a fixed order.
template <bool TA, bool TB, int THY, int TM, int TN>
__global__ void __launch_bounds__(256) k_dgemm(int m, int n, int k, double alpha,
                                               const double* __restrict__ A, int lda,
                                               const double* __restrict__ B, int ldb, double beta,
                                               double* __restrict__ C, int ldc, GemmBatch bt,
                                               int ksplit, int kchunk) {
  constexpr int THX = 256 / THY;
  constexpr int BM = THY * TM, BN = THX * TN;
  int kbeg = 0, kend = k;
  if (ksplit > 1) {
    kbeg = blockIdx.z * kchunk;
    kend = min(k, kbeg + kchunk);
    C += (size_t)blockIdx.z * m * n;
  } else {
    const int bz = blockIdx.z;
    const int b1 = bz / bt.nb2, b2 = bz % bt.nb2;
    A += b1 * bt.sA1 + b2 * bt.sA2;
    B += b1 * bt.sB1 + b2 * bt.sB2;
    C += b1 * bt.sC1 + b2 * bt.sC2;
  }
  __shared__ double As[kBK][BM + 1];
  __shared__ double Bs[kBK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % THX, ty = tid / THX;
  // tiles linearised on grid.x (column tiles fastest): no 65535 limit on rows
  const int ntn = (n + BN - 1) / BN;
  const int row0 = (int)(blockIdx.x / ntn) * BM, col0 = (int)(blockIdx.x % ntn) * BN;
  double acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; r++)
#pragma unroll
    for (int c = 0; c < TN; c++) acc[r][c] = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += kBK) {
#pragma unroll
    for (int e = tid; e < BM * kBK; e += 256) {
      int i, kk;
      if (!TA) {
        i = e / kBK;
        kk = e % kBK;
      } else {
        kk = e / BM;
        i = e % BM;
      }
      const int gi = row0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < m && gk < kend) v = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
      As[kk][i] = v;
    }
#pragma unroll
    for (int e = tid; e < BN * kBK; e += 256) {
      int j, kk;
      if (!TB) {
        kk = e / BN;
        j = e % BN;
      } else {
        j = e / kBK;
        kk = e % kBK;
      }
      const int gj = col0 + j, gk = k0 + kk;
      double v = 0.0;
      if (gj < n && gk < kend) v = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk++) {
      double a[TM], b[TN];
#pragma unroll
      for (int r = 0; r < TM; r++) a[r] = As[kk][ty + THY * r];
#pragma unroll
      for (int c = 0; c < TN; c++) b[c] = Bs[kk][tx + THX * c];
#pragma unroll
      for (int r = 0; r < TM; r++)
#pragma unroll
        for (int c = 0; c < TN; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < TM; r++) {
    const int gi = row0 + ty + THY * r;
    if (gi >= m) continue;
#pragma unroll
    for (int c = 0; c < TN; c++) {
      const int gj = col0 + tx + THX * c;
      if (gj >= n) continue;
      if (ksplit > 1) {
        C[(size_t)gi * n + gj] = acc[r][c];
      } else {
        double* p = C + (size_t)gi * ldc + gj;
        *p = beta == 0.0 ? alpha * acc[r][c] : fma(alpha, acc[r][c], beta * *p);
      }
    }
  }
}

// 32 outputs per CTA; warp g adds the slices g, g + 8, ... in order, then
// warp 0 adds the eight sums in order (the FP64 adds of a skinny product's
// many slices spread over many SMs; same result every run).
__global__ void __launch_bounds__(256) k_splitk_reduce(int m, int n, int ksplit,
                                                       const double* __restrict__ ws, double alpha,
                                                       double beta, double* __restrict__ C, int ldc) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const long long mn = (long long)m * n;
  const long long t = (long long)blockIdx.x * 32 + lane;
  double s = 0.0;
  if (t < mn)
    for (int z = g; z < ksplit; z += 8) s += ws[(size_t)z * mn + t];
  red[g][lane] = s;
  __syncthreads();
  if (g != 0 || t >= mn) return;
#pragma unroll
  for (int h = 1; h < 8; h++) s += red[h][lane];
  const int i = (int)(t / n), j = (int)(t % n);
  double* p = C + (size_t)i * ldc + j;
  *p = beta == 0.0 ? alpha * s : fma(alpha, s, beta * *p);
}

namespace {

struct TileShape {
  int thy, tm, tn;
  int bm() const { return thy * tm; }
  int bn() const { return (256 / thy) * tn; }
};
constexpr TileShape kShapes[] = {{16, 4, 4}, {16, 4, 2}, {16, 2, 4}, {16, 2, 2}, {16, 4, 1},
                                 {16, 1, 4}, {16, 2, 1}, {16, 1, 2}, {16, 1, 1}, {8, 1, 4},
                                 {8, 1, 2}, {8, 1, 1}};

// The shape with the fewest padded multiply-adds; among equals the one with
// the largest tile (more reuse of each loaded element).
TileShape pick_shape(int m, int n) {
  TileShape best = kShapes[0];
  long long best_cost = -1;
  for (const TileShape& t : kShapes) {
    const long long cost = (long long)cdiv(m, t.bm()) * t.bm() * cdiv(n, t.bn()) * t.bn();
    const long long area = (long long)t.bm() * t.bn();
    const long long barea = (long long)best.bm() * best.bn();
    if (best_cost < 0 || cost < best_cost || (cost == best_cost && area > barea)) {
      best = t;
      best_cost = cost;
    }
  }
  return best;
}

template <bool TA, bool TB, int THY, int TM, int TN>
void launch_shape(dim3 grid, cudaStream_t st, int m, int n, int k, double alpha, const double* A,
                  int lda, const double* B, int ldb, double beta, double* C, int ldc,
                  const GemmBatch& bt, int ksplit, int kchunk) {
  k_dgemm<TA, TB, THY, TM, TN><<<grid, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                                     bt, ksplit, kchunk);
}

template <bool TA, bool TB>
void launch_t(const TileShape& s, dim3 grid, cudaStream_t st, int m, int n, int k, double alpha,
              const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
              const GemmBatch& bt, int ksplit, int kchunk) {
#define RIS_SHAPE(Y, M_, N_)                                                                     \
  if (s.thy == Y && s.tm == M_ && s.tn == N_)                                                    \
    return launch_shape<TA, TB, Y, M_, N_>(grid, st, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, \
                                           bt, ksplit, kchunk);
  RIS_SHAPE(16, 4, 4) RIS_SHAPE(16, 4, 2) RIS_SHAPE(16, 2, 4) RIS_SHAPE(16, 2, 2)
  RIS_SHAPE(16, 4, 1) RIS_SHAPE(16, 1, 4) RIS_SHAPE(16, 2, 1) RIS_SHAPE(16, 1, 2)
  RIS_SHAPE(16, 1, 1) RIS_SHAPE(8, 1, 4) RIS_SHAPE(8, 1, 2) RIS_SHAPE(8, 1, 1)
#undef RIS_SHAPE
}

}  // namespace

void dgemm(bool transA, bool transB, int m, int n, int k, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t st,
           const GemmBatch& bt) {
  if (m <= 0 || n <= 0) return;
  const int nb = bt.nb1 * bt.nb2;
  if (nb <= 0) return;
  RIS_REQUIRE(nb <= 65535, RIS_ERR_ARG, "dgemm: batch too large");
  if (k <= 0) {  // C = beta C
    RIS_REQUIRE(beta == 0.0, RIS_ERR_ARG, "dgemm: k = 0 with beta != 0");
  }
  const TileShape sh = pick_shape(m, n);
  const int tiles = cdiv(n, sh.bn()) * cdiv(m, sh.bm());
  // split k when a single product has too few tiles to occupy every SM twice
  int ksplit = 1, kchunk = k;
  if (nb == 1 && tiles < 2 * 152 && k >= 512) {
    ksplit = std::min(cdiv(2 * 152, tiles), k / 256);
    ksplit = std::max(1, std::min(ksplit, 512));
    kchunk = ((cdiv(k, ksplit) + kBK - 1) / kBK) * kBK;
    ksplit = cdiv(k, kchunk);
  }
  double* ws = nullptr;
  MemTrack* ws_tr = nullptr;
  if (ksplit > 1) ws = (double*)dev_alloc(sizeof(double) * (size_t)ksplit * m * n, st, &ws_tr);
  const long long ntiles = (long long)cdiv(n, sh.bn()) * cdiv(m, sh.bm());
  RIS_REQUIRE(ntiles < (1LL << 31), RIS_ERR_ARG, "dgemm: too many tiles");
  dim3 grid((unsigned)ntiles, 1, ksplit > 1 ? ksplit : nb);
  double* Cout = ksplit > 1 ? ws : C;
  prof_begin(kProfGemm, st);
  if (!transA && !transB)
    launch_t<false, false>(sh, grid, st, m, n, k, alpha, A, lda, B, ldb, beta, Cout, ldc, bt, ksplit, kchunk);
  else if (!transA && transB)
    launch_t<false, true>(sh, grid, st, m, n, k, alpha, A, lda, B, ldb, beta, Cout, ldc, bt, ksplit, kchunk);
  else if (transA && !transB)
    launch_t<true, false>(sh, grid, st, m, n, k, alpha, A, lda, B, ldb, beta, Cout, ldc, bt, ksplit, kchunk);
  else
    launch_t<true, true>(sh, grid, st, m, n, k, alpha, A, lda, B, ldb, beta, Cout, ldc, bt, ksplit, kchunk);
  RIS_CHECK_LAUNCH();
  if (ksplit > 1) {
    k_splitk_reduce<<<cdiv((long long)m * n, 32), 256, 0, st>>>(m, n, ksplit, ws, alpha, beta, C, ldc);
    RIS_CHECK_LAUNCH();
    dev_free(ws, sizeof(double) * (size_t)ksplit * m * n, st, ws_tr);
  }
  prof_end(kProfGemm, st, 2.0 * m * n * (double)std::max(k, 0) * nb);
}

// ------------------------------------------------------------------ reductions
// Sum over the block (NT threads) of v, returned to every thread; red holds
// 33 elements of shared memory.
template <int NT, class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x < 32) {
    s = threadIdx.x < NT / 32 ? red[threadIdx.x] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// ------------------------------------------------------------------ Cholesky
__global__ void __launch_bounds__(1024) k_cholesky(double* A, int n, int* info) {
  __shared__ double red[33];
  __shared__ double piv;
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; j++) {
    double part = 0.0;
    for (int k = tid; k < j; k += 1024) part += A[(size_t)j * n + k] * A[(size_t)j * n + k];
    const double s = block_sum<1024>(part, red);
    if (tid == 0) {
      const double ajj = A[(size_t)j * n + j];
      const double d = ajj - s;
      if (!(d > 1e-13 * ajj)) {  // (numerically) singular or indefinite
        bad = j + 1;
      } else {
        piv = sqrt(d);
        A[(size_t)j * n + j] = piv;
      }
    }
    __syncthreads();
    if (bad) break;
    const double pj = piv;
    for (int i = j + 1 + tid; i < n; i += 1024) {
      double acc = A[(size_t)i * n + j];
      for (int k = 0; k < j; k++) acc -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = acc / pj;
    }
    __syncthreads();
  }
  if (!bad) {
    for (size_t e = tid; e < (size_t)n * n; e += 1024) {
      const int i = (int)(e / n), j = (int)(e % n);
      if (j > i) A[e] = 0.0;
    }
  }
  if (tid == 0) *info = bad;
}

// Shared-memory form for n <= kSmemChol: right-looking, the trailing update
// spread over the block; the same relative pivot test as k_cholesky.
constexpr int kSmemChol = 160;
__global__ void __launch_bounds__(1024) k_cholesky_smem(double* A, int n, int* info) {
  extern __shared__ double S[];
  double* diag0 = S + (size_t)n * n;
  __shared__ double piv;
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (size_t e = tid; e < (size_t)n * n; e += 1024) S[e] = A[e];
  for (int j = tid; j < n; j += 1024) diag0[j] = A[(size_t)j * n + j];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; j++) {
    if (tid == 0) {
      const double d = S[(size_t)j * n + j];
      if (!(d > 1e-13 * diag0[j])) {
        bad = j + 1;
      } else {
        piv = sqrt(d);
        S[(size_t)j * n + j] = piv;
      }
    }
    __syncthreads();
    if (bad) break;
    const double pj = piv;
    for (int i = j + 1 + tid; i < n; i += 1024) S[(size_t)i * n + j] /= pj;
    __syncthreads();
    // trailing lower triangle: S[i][k] -= S[i][j] S[k][j], j < k <= i
    // (warps over rows, lanes over columns)
    for (int i = j + 1 + (tid >> 5); i < n; i += 32) {
      const double sij = S[(size_t)i * n + j];
      for (int k = j + 1 + (tid & 31); k <= i; k += 32) S[(size_t)i * n + k] -= sij * S[(size_t)k * n + j];
    }
    __syncthreads();
  }
  if (!bad) {
    for (size_t e = tid; e < (size_t)n * n; e += 1024) {
      const int i = (int)(e / n), k = (int)(e % n);
      A[e] = k > i ? 0.0 : S[e];
    }
  }
  if (tid == 0) *info = bad;
}

void cholesky(double* A, int n, int* d_info, cudaStream_t st) {
  if (n <= kSmemChol) {
    const size_t smem = ((size_t)n * n + n) * sizeof(double);
    ensure_smem_attr((const void*)k_cholesky_smem, (int)(((size_t)kSmemChol * kSmemChol + kSmemChol) * sizeof(double)));
    k_cholesky_smem<<<1, 1024, smem, st>>>(A, n, d_info);
  } else {
    k_cholesky<<<1, 1024, 0, st>>>(A, n, d_info);
  }
  RIS_CHECK_LAUNCH();
}

__global__ void k_tri_inverse(const double* __restrict__ L, double* __restrict__ X, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int i = 0; i < j; i++) X[(size_t)i * n + j] = 0.0;
  X[(size_t)j * n + j] = 1.0 / L[(size_t)j * n + j];
  for (int i = j + 1; i < n; i++) {
    double acc = 0.0;
    for (int k = j; k < i; k++) acc += L[(size_t)i * n + k] * X[(size_t)k * n + j];
    X[(size_t)i * n + j] = -acc / L[(size_t)i * n + i];
  }
}

// One warp per column j of X = L^-1 (four per CTA, CTAs over the columns):
// column-oriented forward substitution of L x = e_j.  Lane l holds the
// right-hand side of rows l, l + 32, ...; at step k the owner of row k
// forms x_k = b_k / L_kk (reciprocals of the diagonal formed once per CTA)
// and broadcasts it, and every lane updates its rows below k.  L is staged
// transposed in shared memory so that a step's reads are consecutive.
constexpr int kTriRB = 5;  // rows per lane: n <= 160
__global__ void __launch_bounds__(128) k_tri_inverse_cols(const double* __restrict__ L,
                                                          double* __restrict__ X, int n) {
  extern __shared__ double tri_sh[];
  double* Lt = tri_sh;  // Lt[k][i] = L[i][k]
  double* rd = Lt + (size_t)n * n;
  for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
    const int i = (int)(e / n), k = (int)(e % n);
    Lt[(size_t)k * n + i] = L[e];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) rd[i] = 1.0 / L[(size_t)i * n + i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (j >= n) return;  // whole warp
  double b[kTriRB];
#pragma unroll
  for (int r = 0; r < kTriRB; r++) b[r] = 32 * r + lane == j ? 1.0 : 0.0;
  for (int i = lane; i < j; i += 32) X[(size_t)i * n + j] = 0.0;
#pragma unroll
  for (int r = 0; r < kTriRB; r++) {
    for (int kk = 0; kk < 32; kk++) {
      const int k = 32 * r + kk;
      if (k >= n) break;
      if (k < j) continue;
      const double xk = __shfl_sync(0xffffffffu, b[r], kk) * rd[k];
      if (lane == kk) X[(size_t)k * n + j] = xk;
      const double* lk = Lt + (size_t)k * n;
#pragma unroll
      for (int r2 = r; r2 < kTriRB; r2++) {
        const int i = 32 * r2 + lane;
        if (i > k && i < n) b[r2] = fma(-lk[i], xk, b[r2]);
      }
    }
  }
}

void tri_inverse(const double* L, double* Linv, int n, cudaStream_t st) {
  if (n <= 32 * kTriRB) {
    const size_t smem = ((size_t)n * n + n) * sizeof(double);
    ensure_smem_attr((const void*)k_tri_inverse_cols,
                     (int)(((size_t)32 * kTriRB * 32 * kTriRB + 32 * kTriRB) * sizeof(double)));
    k_tri_inverse_cols<<<cdiv(n, 4), 128, smem, st>>>(L, Linv, n);
  } else {
    k_tri_inverse<<<cdiv(n, 32), 32, 0, st>>>(L, Linv, n);
  }
  RIS_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ eigensolver
constexpr int kEigT = 256;
constexpr int kEigMaxM = 256;  // largest subspace (Davidson caps it at 256)

size_t eig_work_size(int m) { return (size_t)m * m + 3 * (size_t)m + 64 + 64 * (size_t)m; }

// 1/q from the FP32 reciprocal refined by two Newton steps in FP64 (relative
// error ~1e-15), far cheaper than an FP64 division on this part; q outside the
// FP32 range takes the division.
__device__ __forceinline__ double rcp64(double q) {
  const double aq = fabs(q);
  if (!(aq > 1e-30 && aq < 1e30)) return 1.0 / q;
  double r = (double)__frcp_rn((float)q);
  r = r * fma(-q, r, 2.0);
  r = r * fma(-q, r, 2.0);
  return r;
}

// FP32 Sturm count (for the coarse bracket only): exact for T + dT with
// |dT| of a few FP32 ulps of ||T||, i.e. correct for every x farther than
// ~1e-6 ||T|| from an eigenvalue.
__device__ int sturm_count_f(const float* d, const float* e2, int m, float x) {
  int c = 0;
  float q = d[0] - x;
  if (q < 0.f) c++;
  for (int i = 1; i < m; i++) {
    if (q == 0.f) q = -1e-30f;
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (q < 0.f) c++;
  }
  return c;
}

// Number of eigenvalues of the tridiagonal (d, e) below x (e2 holds e[i]^2)
// from the signs of the leading principal minors p_i = det(T_i - x I):
// p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}, one sign change per
// eigenvalue below x (p_i / p_{i-1} is the i-th pivot of the LDL^T
// factorisation of T - x I; a zero minor counts as a change, as a zero pivot
// taken negative).  No division: per step one subtraction, one product and
// one FMA on the FP64 pipe, the dependent chain a single FMA (the pivot
// recurrence needs a reciprocal and three operations per step, which
// matters on this part's narrow FP64 pipe); signs and exponents are read
// from the bit patterns.  The pair
// (p_{i-1}, p_i) is rescaled by a power of two when the larger leaves
// [2^-500, 2^500] (exact; the signs are unchanged).
__device__ __forceinline__ int dexp(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}
__device__ int sturm_count_minors(const double* d, const double* e2, int m, double x) {
  double p0 = 1.0, p1 = d[0] - x;
  if (dexp(p1) == 0) p1 = -1e-300;  // zero (or subnormal): a change
  int c = __double_as_longlong(p1) < 0 ? 1 : 0;
  for (int i = 1; i < m; i++) {
    double p2 = fma(d[i] - x, p1, -(e2[i - 1] * p0));
    const long long b1 = __double_as_longlong(p1);
    if (dexp(p2) == 0) p2 = b1 < 0 ? 1e-300 : -1e-300;  // a zero minor: a change
    c += (__double_as_longlong(p2) < 0) != (b1 < 0);
    const int ex = max(dexp(p1), dexp(p2));
    if (ex > 1023 + 500 || ex < 1023 - 500) {
      const double sc = __longlong_as_double((long long)(2046 - ex) << 52);  // 2^(1023 - ex)
      p2 *= sc;
      p1 *= sc;
    }
    p0 = p1;
    p1 = p2;
  }
  return c;
}

// The work array holds A (m x m: Householder vectors below the diagonal),
// d, e, tau (m each), the eigenvalues (64) and the eigenvectors (k x m).
struct EigWork {
  double *A, *d, *e, *tau, *lam, *Z;
  __host__ __device__ EigWork(double* work, int m) {
    A = work;
    d = A + (size_t)m * m;
    e = d + m;
    tau = e + m;
    lam = tau + m;
    Z = lam + 64;
  }
};

// Gershgorin bounds of the tridiagonal matrix (d, e).
__device__ void tri_bounds(const double* d, const double* e, int m, double& glo, double& ghi) {
  for (int i = 0; i < m; i++) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
    const double lo = d[i] - r, hi = d[i] + r;
    if (i == 0 || lo < glo) glo = lo;
    if (i == 0 || hi > ghi) ghi = hi;
  }
}

// Stage 1 (one CTA): symmetrise H and reduce it to tridiagonal form
// T = Q^T H Q by Householder reflections (d, e; reflectors kept in A).
// No __restrict__: every array is carved out of `work`, and with
// restrict-qualified parameters the compiler reordered in-place updates.
__global__ void __launch_bounds__(kEigT) k_eig_tridiag(const double* H, int ldH, int m,
                                                       double* work, int use_smem) {
  extern __shared__ double sm_A[];
  __shared__ double red[33];
  __shared__ double sh_alpha, sh_tau;
  __shared__ double p[kEigMaxM];   // A_sub v of the current step
  __shared__ double vc[kEigMaxM];  // the current Householder vector (column c below the diagonal)
  EigWork W(work, m);
  double* A = use_smem ? sm_A : W.A;
  double* d = W.d;
  double* e = W.e;
  double* tau = W.tau;
  const int tid = threadIdx.x;
  for (size_t ij = tid; ij < (size_t)m * m; ij += kEigT) {
    const int i = (int)(ij / m), j = (int)(ij % m);
    A[ij] = 0.5 * (H[(size_t)i * ldH + j] + H[(size_t)j * ldH + i]);
  }
  __syncthreads();
  for (int c = 0; c + 2 < m; c++) {
    double part = 0.0;
    for (int i = c + 1 + tid; i < m; i += kEigT) part += A[(size_t)i * m + c] * A[(size_t)i * m + c];
    const double s = block_sum<kEigT>(part, red);
    if (tid == 0) {
      const double x0 = A[(size_t)(c + 1) * m + c];
      const double nrm = sqrt(s);
      d[c] = A[(size_t)c * m + c];
      if (nrm == 0.0) {
        sh_alpha = 0.0;
        sh_tau = 0.0;
      } else {
        const double alpha = x0 >= 0.0 ? -nrm : nrm;
        const double v0 = x0 - alpha;
        const double vn2 = s - x0 * x0 + v0 * v0;
        A[(size_t)(c + 1) * m + c] = v0;
        sh_alpha = alpha;
        sh_tau = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
      }
      e[c] = sh_alpha;
      tau[c] = sh_tau;
    }
    __syncthreads();
    const double t = sh_tau;
    if (t == 0.0) continue;
    for (int i = c + 1 + tid; i < m; i += kEigT) vc[i] = A[(size_t)i * m + c];
    __syncthreads();
    // p = t * A_sub v, using symmetry for coalesced reads: two threads per
    // row (alternate j), two partial sums each, so that the dependent FP64
    // chains are a quarter of the row long
    for (int i0 = c + 1; i0 < m; i0 += kEigT / 2) {  // uniform: the shuffle needs every lane
      const int i = i0 + (tid >> 1), h = tid & 1;
      double a0 = 0.0, a1 = 0.0;
      if (i < m) {
        int j = c + 1 + h;
        for (; j + 2 < m; j += 4) {
          a0 += A[(size_t)j * m + i] * vc[j];
          a1 += A[(size_t)(j + 2) * m + i] * vc[j + 2];
        }
        if (j < m) a0 += A[(size_t)j * m + i] * vc[j];
      }
      double acc = a0 + a1;
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (i < m && h == 0) p[i] = t * acc;
    }
    __syncthreads();
    part = 0.0;
    for (int i = c + 1 + tid; i < m; i += kEigT) part += p[i] * vc[i];
    const double K = 0.5 * t * block_sum<kEigT>(part, red);
    for (int i = c + 1 + tid; i < m; i += kEigT) p[i] -= K * vc[i];
    __syncthreads();
    // rank-2 update of the trailing block: warps over rows, lanes over columns
    for (int i = c + 1 + (tid >> 5); i < m; i += kEigT / 32) {
      const double vi = vc[i], pi = p[i];
      for (int j = c + 1 + (tid & 31); j < m; j += 32) A[(size_t)i * m + j] -= vi * p[j] + pi * vc[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      d[m - 2] = A[(size_t)(m - 2) * m + m - 2];
      e[m - 2] = A[(size_t)(m - 1) * m + m - 2];
      tau[m - 2] = 0.0;
    }
    d[m - 1] = A[(size_t)(m - 1) * m + m - 1];
    e[m - 1] = 0.0;
    tau[m - 1] = 0.0;
  }
  if (use_smem) {  // the reflectors are read back by the next stage
    for (size_t ij = tid; ij < (size_t)m * m; ij += kEigT) W.A[ij] = A[ij];
  }
}

constexpr int kEigVecT = 128;

// Stage 2 (one CTA per wanted eigenvalue j, so that the FP64 work of the
// eigenvalues runs on as many SMs): lambda_j by multisection on Sturm
// counts, 32 points per step (33-fold shrink): FP32 counts down to a
// bracket of 1e-5 ||T||, widened by 1e-5 ||T|| on each side (over 100 times
// the FP32 count error), then FP64 counts down to 3e-14 ||T||; the
// eigenvector of T by inverse iteration (Gaussian elimination with partial
// pivoting of T - lambda_j I, three solves), and its back-transformation
// x = H_0 ... H_{m-3} z.  Householder vectors in shared memory when
// a_smem is set (m x m doubles).
__global__ void __launch_bounds__(kEigVecT) k_eig_vec(int m, double* work, int a_smem) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  __shared__ double sh_lo, sh_hi;
  EigWork W(work, m);
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  double* d = sm;
  double* e = d + m;
  double* e2 = e + m;
  double* z = e2 + m;
  double* dl = z + m;
  double* dd = dl + m;
  double* du = dd + m;
  double* du2 = du + m;
  double* piv = du2 + m;
  double* tau = piv + m;
  float* df = (float*)(tau + m);
  float* e2f = df + m;
  double* As = tau + m + m;  // after the two float arrays (m doubles)
  for (int i = tid; i < m; i += kEigVecT) {
    d[i] = W.d[i];
    e[i] = W.e[i];
    e2[i] = W.e[i] * W.e[i];
    tau[i] = W.tau[i];
    df[i] = (float)W.d[i];
    e2f[i] = (float)(W.e[i] * W.e[i]);
  }
  if (a_smem)
    for (size_t t = tid; t < (size_t)m * m; t += kEigVecT) As[t] = W.A[t];
  const double* A = a_smem ? As : W.A;
  __syncthreads();
  // Gershgorin bounds by one thread (every thread repeating the FP64 scan
  // would load the SM's narrow FP64 pipe 128-fold)
  if (tid == 0) {
    double lo0 = 0.0, hi0 = 0.0;
    tri_bounds(d, e, m, lo0, hi0);
    sh_lo = lo0;
    sh_hi = hi0;
  }
  __syncthreads();
  const double glo = sh_lo, ghi = sh_hi;
  __syncthreads();  // sh_lo / sh_hi are reused for the bracket below
  const double tnorm = fmax(fmax(fabs(glo), fabs(ghi)), 1e-300);
  if (tid < 32) {
    const int lane = tid;
    double lo = glo - 1e-12 * tnorm, hi = ghi + 1e-12 * tnorm;
    // coarse: FP32 counts while the bracket is wider than 1e-5 ||T||
    const double coarse = 1e-5 * tnorm;
    for (int it = 0; it < 12 && hi - lo > coarse; it++) {
      const double h = (hi - lo) / 33.0;
      const float x = (float)(lo + h * (lane + 1));
      const bool above = sturm_count_f(df, e2f, m, x) > j;
      const unsigned mask = __ballot_sync(0xffffffffu, above);
      const int f = mask ? __ffs(mask) - 1 : 32;
      const double nlo = f == 0 ? lo : lo + h * f;
      const double nhi = f == 32 ? hi : lo + h * (f + 1);
      lo = nlo;
      hi = nhi;
    }
    lo = fmax(lo - coarse, glo - 1e-12 * tnorm);
    hi = fmin(hi + coarse, ghi + 1e-12 * tnorm);
    // fine: FP64 counts (the counts that decide the final bracket), down to
    // a bracket of 3e-14 ||T|| (the midpoint then within 1.5e-14 ||T||, far
    // below what the Davidson residuals resolve) or the FP64 resolution
    for (int it = 0; it < 40; it++) {
      const double h = (hi - lo) / 33.0;
      if (!(h > 0.0) || lo + h <= lo || hi - lo <= 3e-14 * tnorm) break;
      const double x = lo + h * (lane + 1);
      const bool above = sturm_count_minors(d, e2, m, x) > j;  // lambda_j < x
      const unsigned mask = __ballot_sync(0xffffffffu, above);
      const int f = mask ? __ffs(mask) - 1 : 32;  // first point above lambda_j
      const double nlo = f == 0 ? lo : lo + h * f;
      const double nhi = f == 32 ? hi : lo + h * (f + 1);
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) {
      sh_lo = lo;
      sh_hi = hi;
    }
  }
  __syncthreads();
  const double lj = 0.5 * (sh_lo + sh_hi);
  if (tid == 0) {
    const double tiny = 1e-15 * tnorm;
    for (int i = 0; i < m; i++) {
      dd[i] = d[i] - lj;
      dl[i] = i + 1 < m ? e[i] : 0.0;
      du[i] = i + 1 < m ? e[i] : 0.0;
      du2[i] = 0.0;
      piv[i] = 0.0;
    }
    for (int i = 0; i + 1 < m; i++) {
      if (fabs(dd[i]) >= fabs(dl[i])) {
        if (dd[i] == 0.0) dd[i] = tiny;
        const double f = dl[i] * rcp64(dd[i]);
        dl[i] = f;
        dd[i + 1] -= f * du[i];
      } else {
        const double f = dd[i] * rcp64(dl[i]);
        dd[i] = dl[i];
        dl[i] = f;
        const double tmp = du[i];
        du[i] = dd[i + 1];
        dd[i + 1] = tmp - f * dd[i + 1];
        if (i + 2 < m) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
        piv[i] = 1.0;
      }
    }
    if (dd[m - 1] == 0.0) dd[m - 1] = tiny;
    for (int i = 0; i < m; i++) dd[i] = rcp64(dd[i]);  // pivots kept as reciprocals
    // start vector depending on j: equal eigenvalues (a split T) give
    // different vectors of their eigenspace, which stage 3 orthonormalises
    for (int i = 0; i < m; i++) z[i] = 1.0 + 0.01 * (double)((i * (j + 1)) % 7);
    for (int it = 0; it < 3; it++) {
      for (int i = 0; i + 1 < m; i++) {
        if (piv[i] == 0.0) {
          z[i + 1] -= dl[i] * z[i];
        } else {
          const double t0 = z[i];
          z[i] = z[i + 1];
          z[i + 1] = t0 - dl[i] * z[i];
        }
      }
      z[m - 1] *= dd[m - 1];
      if (m >= 2) z[m - 2] = (z[m - 2] - du[m - 2] * z[m - 1]) * dd[m - 2];
      for (int i = m - 3; i >= 0; i--) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) * dd[i];
      double nrm = 0.0;
      for (int i = 0; i < m; i++) nrm += z[i] * z[i];
      nrm = 1.0 / sqrt(nrm);
      for (int i = 0; i < m; i++) z[i] *= nrm;
    }
    W.lam[j] = lj;
  }
  __syncthreads();
  // back-transformation, H_{m-3} applied first, by one warp (each lane owns
  // the same elements of z in the dot product and in the update, so the
  // steps need no barrier)
  if (tid < 32) {
    for (int c = m - 3; c >= 0; c--) {
      const double t = tau[c];
      if (t == 0.0) continue;
      double part = 0.0;
      for (int i = c + 1 + tid; i < m; i += 32) part += A[(size_t)i * m + c] * z[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      const double f = t * part;
      for (int i = c + 1 + tid; i < m; i += 32) z[i] -= f * A[(size_t)i * m + c];
    }
  }
  __syncthreads();
  for (int i = tid; i < m; i += kEigVecT) W.Z[(size_t)j * m + i] = z[i];
}

// Stage 3 (one CTA): Gram-Schmidt within clusters of close eigenvalues
// (inverse iteration alone does not separate them), then the output.
__global__ void __launch_bounds__(kEigT) k_eig_finish(int m, int k, double* w, double* V,
                                                      double* work) {
  __shared__ double red[33];
  __shared__ double lam[64], bnd[2];
  EigWork W(work, m);
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += kEigT) lam[i] = W.lam[i];
  if (tid == 0) {
    double glo = 0.0, ghi = 0.0;
    tri_bounds(W.d, W.e, m, glo, ghi);
    bnd[0] = glo;
    bnd[1] = ghi;
  }
  __syncthreads();
  const double tnorm = fmax(fmax(fabs(bnd[0]), fabs(bnd[1])), 1e-300);
  const double gap_tol = 1e-7 * tnorm;
  // close[j] bit i (i < j): lambda_i within gap_tol of lambda_j, one thread
  // per j (the test repeated by every thread would load the narrow FP64 pipe)
  __shared__ unsigned long long close[64];
  if (tid < k) {
    unsigned long long msk = 0ull;
    for (int i = 0; i < tid; i++)
      if (!(fabs(lam[tid] - lam[i]) > gap_tol)) msk |= 1ull << i;
    close[tid] = msk;
  }
  __syncthreads();
  double* Z = W.Z;
  for (int j = 1; j < k; j++) {
    const unsigned long long msk = close[j];
    if (!msk) continue;
    for (int i = 0; i < j; i++) {
      if (!((msk >> i) & 1ull)) continue;
      double part = 0.0;
      for (int q = tid; q < m; q += kEigT) part += Z[(size_t)i * m + q] * Z[(size_t)j * m + q];
      const double s = block_sum<kEigT>(part, red);
      for (int q = tid; q < m; q += kEigT) Z[(size_t)j * m + q] -= s * Z[(size_t)i * m + q];
      __syncthreads();
      part = 0.0;
      for (int q = tid; q < m; q += kEigT) part += Z[(size_t)j * m + q] * Z[(size_t)j * m + q];
      const double nn = block_sum<kEigT>(part, red);
      for (int q = tid; q < m; q += kEigT) Z[(size_t)j * m + q] /= sqrt(nn);
      __syncthreads();
    }
  }
  for (int j = tid; j < k; j += kEigT) w[j] = lam[j];
  for (size_t i = tid; i < (size_t)k * m; i += kEigT) V[i] = Z[i];
}

// ---------------------------------------------------- FP32 subspace eigensolver
// The same three stages in FP32 arithmetic for the mixed precision form: the
// Householder reduction and the eigenvectors of T are backward stable, so
// every returned vector has a residual |H z - theta z| of a few FP32 ulps
// of ||H|| (about 1e-7 ||H||, below the mixed form's Davidson tolerance);
// the Ritz values are FP64 Rayleigh quotients of the FP64-normalised
// vectors.  Vectors of close eigenvalues (within 1e-4 ||T||) are made
// orthonormal and rotated onto the Ritz vectors of their span in FP64.
constexpr int kEig32MaxM = 200;  // m^2 floats in shared memory

// Stage 1 in FP32: T = Q^T H Q; reflectors left as floats in the first m^2
// floats of the work array's A block, d, e, tau stored as doubles.
__global__ void __launch_bounds__(kEigT) k_eig_tridiag32(const double* H, int ldH, int m,
                                                         double* work) {
  extern __shared__ float sA32[];
  __shared__ float red[33];
  __shared__ float sh_alpha, sh_tau;
  __shared__ float p[kEigMaxM];
  __shared__ float vc[kEigMaxM];
  EigWork W(work, m);
  float* A = sA32;
  const int tid = threadIdx.x;
  for (size_t ij = tid; ij < (size_t)m * m; ij += kEigT) {
    const int i = (int)(ij / m), j = (int)(ij % m);
    A[ij] = (float)(0.5 * (H[(size_t)i * ldH + j] + H[(size_t)j * ldH + i]));
  }
  __syncthreads();
  for (int c = 0; c + 2 < m; c++) {
    float part = 0.f;
    for (int i = c + 1 + tid; i < m; i += kEigT) part += A[(size_t)i * m + c] * A[(size_t)i * m + c];
    const float s = block_sum<kEigT>(part, red);
    if (tid == 0) {
      const float x0 = A[(size_t)(c + 1) * m + c];
      const float nrm = sqrtf(s);
      W.d[c] = A[(size_t)c * m + c];
      if (nrm == 0.f) {
        sh_alpha = 0.f;
        sh_tau = 0.f;
      } else {
        const float alpha = x0 >= 0.f ? -nrm : nrm;
        const float v0 = x0 - alpha;
        const float vn2 = s - x0 * x0 + v0 * v0;
        A[(size_t)(c + 1) * m + c] = v0;
        sh_alpha = alpha;
        sh_tau = vn2 > 0.f ? 2.f / vn2 : 0.f;
      }
      W.e[c] = sh_alpha;
      W.tau[c] = sh_tau;
    }
    __syncthreads();
    const float tt = sh_tau;
    if (tt == 0.f) continue;
    for (int i = c + 1 + tid; i < m; i += kEigT) vc[i] = A[(size_t)i * m + c];
    __syncthreads();
    for (int i = c + 1 + tid; i < m; i += kEigT) {
      float acc = 0.f;
      for (int j = c + 1; j < m; j++) acc += A[(size_t)j * m + i] * vc[j];
      p[i] = tt * acc;
    }
    __syncthreads();
    part = 0.f;
    for (int i = c + 1 + tid; i < m; i += kEigT) part += p[i] * vc[i];
    const float K = 0.5f * tt * block_sum<kEigT>(part, red);
    for (int i = c + 1 + tid; i < m; i += kEigT) p[i] -= K * vc[i];
    __syncthreads();
    for (int i = c + 1 + (tid >> 5); i < m; i += kEigT / 32) {
      const float vi = vc[i], pi = p[i];
      for (int j = c + 1 + (tid & 31); j < m; j += 32) A[(size_t)i * m + j] -= vi * p[j] + pi * vc[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      W.d[m - 2] = A[(size_t)(m - 2) * m + m - 2];
      W.e[m - 2] = A[(size_t)(m - 1) * m + m - 2];
      W.tau[m - 2] = 0.0;
    }
    W.d[m - 1] = A[(size_t)(m - 1) * m + m - 1];
    W.e[m - 1] = 0.0;
    W.tau[m - 1] = 0.0;
  }
  float* Ag = (float*)W.A;
  for (size_t ij = tid; ij < (size_t)m * m; ij += kEigT) Ag[ij] = A[ij];
}

constexpr int kEig32VecT = 128;

// Stage 2 in FP32 (one CTA per wanted eigenvalue j): multisection on FP32
// Sturm counts down to FP32 resolution, inverse iteration, back
// transformation; then the vector in FP64, normalised, and its FP64
// Rayleigh quotient with H.
__global__ void __launch_bounds__(kEig32VecT) k_eig_vec32(int m, double* work, const double* H,
                                                          int ldH) {
  extern __shared__ float s32[];
  __shared__ double redd[33];
  __shared__ float sh_lo, sh_hi;
  EigWork W(work, m);
  const int j = blockIdx.x;
  const int tid = threadIdx.x;
  float* d = s32;
  float* e = d + m;
  float* e2 = e + m;
  float* tau = e2 + m;
  float* z = tau + m;
  float* dl = z + m;
  float* dd = dl + m;
  float* du = dd + m;
  float* du2 = du + m;
  float* piv = du2 + m;
  float* A = piv + m;
  double* zd = (double*)(A + (size_t)m * m + ((m * m) & 1));  // m doubles, 8-byte aligned
  for (int i = tid; i < m; i += kEig32VecT) {
    d[i] = (float)W.d[i];
    e[i] = (float)W.e[i];
    e2[i] = e[i] * e[i];
    tau[i] = (float)W.tau[i];
  }
  const float* Ag = (const float*)W.A;
  for (size_t q = tid; q < (size_t)m * m; q += kEig32VecT) A[q] = Ag[q];
  __syncthreads();
  if (tid < 32) {
    const int lane = tid;
    float glo = 0.f, ghi = 0.f;
    for (int i = 0; i < m; i++) {
      const float r = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i + 1 < m ? fabsf(e[i]) : 0.f);
      if (i == 0 || d[i] - r < glo) glo = d[i] - r;
      if (i == 0 || d[i] + r > ghi) ghi = d[i] + r;
    }
    const float tn = fmaxf(fmaxf(fabsf(glo), fabsf(ghi)), 1e-30f);
    float lo = glo - 1e-6f * tn, hi = ghi + 1e-6f * tn;
    for (int it = 0; it < 24; it++) {
      const float h = (hi - lo) / 33.f;
      if (!(h > 0.f) || lo + h <= lo || hi - h >= hi) break;
      const float x = lo + h * (float)(lane + 1);
      const bool above = sturm_count_f(d, e2, m, x) > j;
      const unsigned mask = __ballot_sync(0xffffffffu, above);
      const int f = mask ? __ffs(mask) - 1 : 32;
      const float nlo = f == 0 ? lo : lo + h * (float)f;
      const float nhi = f == 32 ? hi : lo + h * (float)(f + 1);
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) {
      sh_lo = lo;
      sh_hi = hi;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const float lj = 0.5f * (sh_lo + sh_hi);
    float tn = 0.f;
    for (int i = 0; i < m; i++) tn = fmaxf(tn, fabsf(d[i]) + 2.f * fabsf(e[i]));
    const float tiny = 1e-7f * fmaxf(tn, 1e-30f);
    for (int i = 0; i < m; i++) {
      dd[i] = d[i] - lj;
      dl[i] = i + 1 < m ? e[i] : 0.f;
      du[i] = i + 1 < m ? e[i] : 0.f;
      du2[i] = 0.f;
      piv[i] = 0.f;
    }
    for (int i = 0; i + 1 < m; i++) {
      if (fabsf(dd[i]) >= fabsf(dl[i])) {
        if (dd[i] == 0.f) dd[i] = tiny;
        const float f = dl[i] / dd[i];
        dl[i] = f;
        dd[i + 1] -= f * du[i];
      } else {
        const float f = dd[i] / dl[i];
        dd[i] = dl[i];
        dl[i] = f;
        const float tmp = du[i];
        du[i] = dd[i + 1];
        dd[i + 1] = tmp - f * dd[i + 1];
        if (i + 2 < m) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
        piv[i] = 1.f;
      }
    }
    if (dd[m - 1] == 0.f) dd[m - 1] = tiny;
    for (int i = 0; i < m; i++) dd[i] = 1.f / dd[i];
    for (int i = 0; i < m; i++) z[i] = 1.f + 0.01f * (float)((i * (j + 1)) % 7);
    for (int it = 0; it < 3; it++) {
      for (int i = 0; i + 1 < m; i++) {
        if (piv[i] == 0.f) {
          z[i + 1] -= dl[i] * z[i];
        } else {
          const float t0 = z[i];
          z[i] = z[i + 1];
          z[i + 1] = t0 - dl[i] * z[i];
        }
      }
      z[m - 1] *= dd[m - 1];
      if (m >= 2) z[m - 2] = (z[m - 2] - du[m - 2] * z[m - 1]) * dd[m - 2];
      for (int i = m - 3; i >= 0; i--) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) * dd[i];
      float mx = 0.f;
      for (int i = 0; i < m; i++) mx = fmaxf(mx, fabsf(z[i]));
      const float sc = mx > 0.f ? 1.f / mx : 1.f;
      for (int i = 0; i < m; i++) z[i] *= sc;
    }
  }
  __syncthreads();
  if (tid < 32) {  // back-transformation by one warp, H_{m-3} first
    for (int c = m - 3; c >= 0; c--) {
      const float tt = tau[c];
      if (tt == 0.f) continue;
      float part = 0.f;
      for (int i = c + 1 + tid; i < m; i += 32) part += A[(size_t)i * m + c] * z[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      const float f = tt * part;
      for (int i = c + 1 + tid; i < m; i += 32) z[i] -= f * A[(size_t)i * m + c];
    }
  }
  __syncthreads();
  // FP64: normalise, Rayleigh quotient z^T H z
  double part = 0.0;
  for (int i = tid; i < m; i += kEig32VecT) {
    zd[i] = (double)z[i];
    part += zd[i] * zd[i];
  }
  const double nn = block_sum<kEig32VecT>(part, redd);
  const double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  for (int i = tid; i < m; i += kEig32VecT) zd[i] *= sc;
  __syncthreads();
  part = 0.0;
  for (int i = tid; i < m; i += kEig32VecT) {
    double hz = 0.0;
    const double* Hi = H + (size_t)i * ldH;
    for (int q = 0; q < m; q++) hz += Hi[q] * zd[q];
    part += zd[i] * hz;
  }
  const double rq = block_sum<kEig32VecT>(part, redd);
  if (tid == 0) W.lam[j] = rq;
  for (int i = tid; i < m; i += kEig32VecT) W.Z[(size_t)j * m + i] = zd[i];
}

// Stage 3 for the FP32 vectors (one CTA): clusters of consecutive
// eigenvalues closer than 1e-4 ||T|| are orthonormalised (two Gram-Schmidt
// passes) and replaced by the Ritz vectors of their span with respect to H
// (FP64 projected matrix, cyclic Jacobi); then the output.
constexpr int kEigMaxCluster = 16;
__global__ void __launch_bounds__(kEigT) k_eig_finish32(int m, int k, double* w, double* V,
                                                        double* work, const double* H, int ldH) {
  __shared__ double red[33];
  __shared__ double lam[64];
  __shared__ double Hc[kEigMaxCluster][kEigMaxCluster], Qc[kEigMaxCluster][kEigMaxCluster];
  __shared__ double bnd[2];
  EigWork W(work, m);
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += kEigT) lam[i] = W.lam[i];
  if (tid == 0) {
    double glo = 0.0, ghi = 0.0;
    tri_bounds(W.d, W.e, m, glo, ghi);
    bnd[0] = glo;
    bnd[1] = ghi;
  }
  __syncthreads();
  const double tnorm = fmax(fmax(fabs(bnd[0]), fabs(bnd[1])), 1e-300);
  const double gap_tol = 1e-4 * tnorm;
  double* Z = W.Z;
  int j0 = 0;
  while (j0 < k) {
    int j1 = j0 + 1;
    while (j1 < k && j1 - j0 < kEigMaxCluster && fabs(lam[j1] - lam[j1 - 1]) <= gap_tol) j1++;
    const int c = j1 - j0;
    if (c > 1) {
      for (int pass = 0; pass < 2; pass++)
        for (int a = j0; a < j1; a++) {
          for (int b = j0; b < a; b++) {
            double part = 0.0;
            for (int q = tid; q < m; q += kEigT) part += Z[(size_t)a * m + q] * Z[(size_t)b * m + q];
            const double s = block_sum<kEigT>(part, red);
            for (int q = tid; q < m; q += kEigT) Z[(size_t)a * m + q] -= s * Z[(size_t)b * m + q];
            __syncthreads();
          }
          double part = 0.0;
          for (int q = tid; q < m; q += kEigT) part += Z[(size_t)a * m + q] * Z[(size_t)a * m + q];
          const double nn = block_sum<kEigT>(part, red);
          for (int q = tid; q < m; q += kEigT) Z[(size_t)a * m + q] /= sqrt(nn);
          __syncthreads();
        }
      // projected matrix Hc = Zc H Zc^T
      for (int a = 0; a < c; a++)
        for (int b = 0; b <= a; b++) {
          double part = 0.0;
          for (int i = tid; i < m; i += kEigT) {
            double hz = 0.0;
            const double* Hi = H + (size_t)i * ldH;
            for (int q = 0; q < m; q++) hz += Hi[q] * Z[(size_t)(j0 + b) * m + q];
            part += Z[(size_t)(j0 + a) * m + i] * hz;
          }
          const double s = block_sum<kEigT>(part, red);
          if (tid == 0) Hc[a][b] = Hc[b][a] = s;
        }
      __syncthreads();
      if (tid == 0) {  // cyclic Jacobi on the c x c matrix
        for (int a = 0; a < c; a++)
          for (int b = 0; b < c; b++) Qc[a][b] = a == b ? 1.0 : 0.0;
        for (int sweep = 0; sweep < 12; sweep++) {
          double off = 0.0;
          for (int a = 0; a < c; a++)
            for (int b = a + 1; b < c; b++) off += Hc[a][b] * Hc[a][b];
          if (off < 1e-30) break;
          for (int a = 0; a < c; a++)
            for (int b = a + 1; b < c; b++) {
              if (Hc[a][b] == 0.0) continue;
              const double th = 0.5 * (Hc[b][b] - Hc[a][a]) / Hc[a][b];
              const double tq = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
              const double cs = 1.0 / sqrt(tq * tq + 1.0), sn = tq * cs;
              for (int q = 0; q < c; q++) {  // columns a, b
                const double x = Hc[q][a], y = Hc[q][b];
                Hc[q][a] = cs * x - sn * y;
                Hc[q][b] = sn * x + cs * y;
              }
              for (int q = 0; q < c; q++) {  // rows a, b
                const double x = Hc[a][q], y = Hc[b][q];
                Hc[a][q] = cs * x - sn * y;
                Hc[b][q] = sn * x + cs * y;
              }
              for (int q = 0; q < c; q++) {
                const double x = Qc[q][a], y = Qc[q][b];
                Qc[q][a] = cs * x - sn * y;
                Qc[q][b] = sn * x + cs * y;
              }
            }
        }
        // ascending order of the Ritz values (selection sort on the columns)
        for (int a = 0; a < c; a++) {
          int best = a;
          for (int b = a + 1; b < c; b++)
            if (Hc[b][b] < Hc[best][best]) best = b;
          if (best != a) {
            const double t0 = Hc[a][a];
            Hc[a][a] = Hc[best][best];
            Hc[best][best] = t0;
            for (int q = 0; q < c; q++) {
              const double t1 = Qc[q][a];
              Qc[q][a] = Qc[q][best];
              Qc[q][best] = t1;
            }
          }
        }
        for (int a = 0; a < c; a++) lam[j0 + a] = Hc[a][a];
      }
      __syncthreads();
      // Z_c <- Qc^T Z_c, column by column of Z
      for (int q = tid; q < m; q += kEigT) {
        double zc[kEigMaxCluster];
        for (int a = 0; a < c; a++) zc[a] = Z[(size_t)(j0 + a) * m + q];
        for (int a = 0; a < c; a++) {
          double s = 0.0;
          for (int b = 0; b < c; b++) s += Qc[b][a] * zc[b];
          Z[(size_t)(j0 + a) * m + q] = s;
        }
      }
      __syncthreads();
    }
    j0 = j1;
  }
  for (int j = tid; j < k; j += kEigT) w[j] = lam[j];
  for (size_t i = tid; i < (size_t)k * m; i += kEigT) V[i] = Z[i];
}

bool sym_eig_lowest_f32(const double* H, int ldH, int m, int k, double* w, double* V, double* work,
                        cudaStream_t st) {
  if (m > kEig32MaxM || k > 64 || k < 1 || k > m) return false;
  const size_t smA = (size_t)m * m * sizeof(float);
  ensure_smem_attr((const void*)k_eig_tridiag32, 200 * 1024);
  ensure_smem_attr((const void*)k_eig_vec32, 200 * 1024);
  const size_t vec_smem = 10 * (size_t)m * sizeof(float) + smA + 8 + (size_t)m * sizeof(double);
  prof_begin(kProfEig, st);
  k_eig_tridiag32<<<1, kEigT, smA, st>>>(H, ldH, m, work);
  RIS_CHECK_LAUNCH();
  k_eig_vec32<<<k, kEig32VecT, vec_smem, st>>>(m, work, H, ldH);
  RIS_CHECK_LAUNCH();
  k_eig_finish32<<<1, kEigT, 0, st>>>(m, k, w, V, work, H, ldH);
  RIS_CHECK_LAUNCH();
  prof_end(kProfEig, st, 1.0);
  return true;
}

void sym_eig_lowest(const double* H, int ldH, int m, int k, double* w, double* V, double* work,
                    cudaStream_t st) {
  RIS_REQUIRE(k >= 1 && k <= 64 && k <= m, RIS_ERR_ARG, "sym_eig_lowest: bad k");
  RIS_REQUIRE(m <= kEigMaxM, RIS_ERR_ARG, "sym_eig_lowest: subspace larger than 256");
  const size_t smem_max = 200 * 1024;
  ensure_smem_attr((const void*)k_eig_tridiag, (int)smem_max);
  const size_t need = (size_t)m * m * sizeof(double);
  const int use_smem = need <= smem_max;
  size_t vec_smem = 11 * (size_t)m * sizeof(double);
  RIS_REQUIRE(vec_smem <= 200 * 1024, RIS_ERR_ARG, "sym_eig_lowest: subspace too large");
  const int a_smem = vec_smem + need <= 200 * 1024;
  if (a_smem) vec_smem += need;
  ensure_smem_attr((const void*)k_eig_vec, (int)(200 * 1024));
  prof_begin(kProfEig, st);
  k_eig_tridiag<<<1, kEigT, use_smem ? need : 0, st>>>(H, ldH, m, work, use_smem);
  RIS_CHECK_LAUNCH();
  k_eig_vec<<<k, kEigVecT, vec_smem, st>>>(m, work, a_smem);
  RIS_CHECK_LAUNCH();
  k_eig_finish<<<1, kEigT, 0, st>>>(m, k, w, V, work);
  RIS_CHECK_LAUNCH();
  prof_end(kProfEig, st, 1.0);
}

// ------------------------------------------------------------------ utilities
__global__ void k_fill(double* x, double v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] = v;
}
void fill(double* x, double v, size_t n, cudaStream_t st) {
  if (!n) return;
  k_fill<<<(unsigned)std::min<size_t>(cdiv(n, 256), 152 * 8), 256, 0, st>>>(x, v, n);
  RIS_CHECK_LAUNCH();
}

__global__ void k_row_dot(const double* __restrict__ V, long long ncol, const double* __restrict__ x,
                          double* __restrict__ out) {
  __shared__ double red[33];
  const double* v = V + (size_t)blockIdx.x * ncol;
  const double* y = x ? x : v;
  double part = 0.0;
  for (long long i = threadIdx.x; i < ncol; i += 256) part += v[i] * y[i];
  const double s = block_sum<256>(part, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// Long rows: nsplit CTAs per row write partial sums, k_row_dot_fin adds them
// in order (spreads the FP64 work over the SMs; same result every run).
__global__ void k_row_dot_part(const double* __restrict__ V, long long ncol,
                               const double* __restrict__ x, int nsplit, double* __restrict__ part) {
  __shared__ double red[33];
  const int row = blockIdx.y, sp = blockIdx.x;
  const double* v = V + (size_t)row * ncol;
  const double* y = x ? x : v;
  const long long per = (ncol + nsplit - 1) / nsplit;
  const long long b = (long long)sp * per, e = min(ncol, b + per);
  double s = 0.0;
  for (long long i = b + threadIdx.x; i < e; i += 256) s += v[i] * y[i];
  s = block_sum<256>(s, red);
  if (threadIdx.x == 0) part[(size_t)row * nsplit + sp] = s;
}

__global__ void k_row_dot_fin(const double* __restrict__ part, int nrow, int nsplit,
                              double* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  double s = 0.0;
  for (int z = 0; z < nsplit; z++) s += part[(size_t)r * nsplit + z];
  out[r] = s;
}

static void row_dots(const double* V, int nrow, long long ncol, const double* x, double* out,
                     cudaStream_t st) {
  if (nrow <= 0) return;
  const int nsplit = (int)std::min<long long>(32, ncol / 4096);
  if (nsplit < 2 || nrow > 65535) {
    k_row_dot<<<nrow, 256, 0, st>>>(V, ncol, x, out);
    RIS_CHECK_LAUNCH();
    return;
  }
  MemTrack* tr = nullptr;
  const size_t b = sizeof(double) * (size_t)nrow * nsplit;
  double* part = (double*)dev_alloc(b, st, &tr);
  k_row_dot_part<<<dim3(nsplit, nrow), 256, 0, st>>>(V, ncol, x, nsplit, part);
  RIS_CHECK_LAUNCH();
  k_row_dot_fin<<<cdiv(nrow, 64), 64, 0, st>>>(part, nrow, nsplit, out);
  RIS_CHECK_LAUNCH();
  dev_free(part, b, st, tr);
}

void row_norms(const double* X, int nrow, long long ncol, double* out, cudaStream_t st) {
  row_dots(X, nrow, ncol, nullptr, out, st);
}
void gemv_rows(const double* V, int nrow, long long ncol, const double* x, double* out,
               cudaStream_t st) {
  row_dots(V, nrow, ncol, x, out, st);
}

}  // namespace ris

// Test hook (declared in include/ris.h): lowest k eigenpairs of a symmetric
// m x m matrix with the device subspace eigensolver; device pointers.
extern "C" int ris_debug_dgemm(int transA, int transB, int m, int n, int k, double alpha,
                               const double* A, int lda, const double* B, int ldb, double beta,
                               double* C, int ldc) {
  using namespace ris;
  try {
    RIS_REQUIRE(m >= 0 && n >= 0 && k >= 0 && A && B && C, RIS_ERR_ARG, "bad dgemm arguments");
    dgemm(transA != 0, transB != 0, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0);
    RIS_CUDA(cudaDeviceSynchronize());
    return 0;
  } catch (const Error& e) {
    fprintf(stderr, "ris_debug_dgemm: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}

extern "C" int ris_debug_sym_eig_f32(int m, int k, const double* H, double* w, double* V) {
  using namespace ris;
  try {
    double* work = nullptr;
    RIS_ALLOC(cudaMalloc(&work, sizeof(double) * eig_work_size(m)));
    const bool ok = sym_eig_lowest_f32(H, m, m, k, w, V, work, 0);
    RIS_CUDA(cudaDeviceSynchronize());
    cudaFree(work);
    return ok ? 0 : (int)RIS_ERR_ARG;
  } catch (const Error& e) {
    fprintf(stderr, "ris_debug_sym_eig_f32: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}

extern "C" int ris_debug_sym_eig(int m, int k, const double* H, double* w, double* V) {
  using namespace ris;
  try {
    double* work = nullptr;
    RIS_ALLOC(cudaMalloc(&work, sizeof(double) * eig_work_size(m)));
    sym_eig_lowest(H, m, m, k, w, V, work, 0);
    RIS_CUDA(cudaDeviceSynchronize());
    cudaFree(work);
    return 0;
  } catch (const Error& e) {
    fprintf(stderr, "ris_debug_sym_eig: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}
