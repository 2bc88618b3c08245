// FP64-accurate GEMM on the FP16 tensor cores (tcgen05) of sm_103a by exact
// splitting of both operands into small-integer slices: the error-free
// transformation of matrix products of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012), with digit slices in one fixed-point frame
// per row.
//
// With x_rk = 2^(E_r) sum_{p=1..10} dA_p(r,k) 2^(-6p) and y_ck likewise,
//   (X Y^T)_rc = 2^(E_r + E_c) sum_{d=2..11} 2^(-6d) V_d(r,c),
//   V_d = sum_{p+q=d} sum_k dA_p(r,k) dB_q(c,k),
// products with p + q > 11 being dropped (below 2^-60 of the frame).
// Digits are FP16 integers of at most 6 bits, their products are exact and,
// for K <= 512, every V_d with d <= 9 (at most eight terms) stays below 2^24
// and is summed exactly in its FP32 tensor-memory accumulator; V_10 and
// V_11 (nine and ten terms) may lose their last bit, 2^-60 below the frame.
// The epilogue combines the ten accumulators in 64-bit integers and FP64.
//
// Kernel (one 128 x BN output tile per CTA, BN <= 48, 128 threads):
//   warp 0 / lane 0 : TMA producer, 4-stage ring; a stage is K = 16 of all
//                     ten slices of A (128 rows) and of B (BN rows), two
//                     3-D loads with 32-byte swizzle
//   warp 1          : allocates 512 TMEM columns (ten accumulators of BN
//                     columns); lane 0 issues the 55 slice products of each
//                     stage (tcgen05.mma.kind::f16, M = 128, N = BN, K = 16)
//   warps 0-3       : epilogue, one output row per thread
// Every mbarrier wait is bounded; a timeout sets the error flag, drains what
// the CTA has in flight and frees its tensor memory.
#include <cuda.h>

#include "gemm_emu.cuh"
#include "tc_ptx.cuh"

namespace ris {

namespace {
using namespace tcx;

constexpr int S = kEmuSlices;
constexpr int NG = S;  // accumulators, d = 2 .. S + 1
constexpr int kFracBits = kEmuBeta * S;  // fixed-point bits of a row frame
constexpr int EBM = 128, EBK = 16, EMAXBN = 48, ESTAGES = 4;
constexpr int A_SLICE = EBM * EBK * 2;  // 4 KB
constexpr int A_BYTES = S * A_SLICE;
constexpr int B_SLICE_MAX = EMAXBN * EBK * 2;
constexpr int ESTAGE = ((A_BYTES + S * B_SLICE_MAX) + 1023) & ~1023;
constexpr int ESMEM = ESTAGES * ESTAGE + 1024 + 256;
constexpr int TMEM_COLS = 512;
static_assert(NG * EMAXBN <= TMEM_COLS, "accumulators exceed tensor memory");
static_assert(ESMEM <= 232448, "pipeline exceeds shared memory");
static_assert(kFracBits <= 63, "row frame exceeds 64-bit integers");
static_assert(NG == 10 && kEmuBeta == 6, "the epilogue's integer combination assumes 10 x 6 bits");

// 3-D map {K, rows, slice} of FP16 digits, box {16, box_rows, S}, 32-byte swizzle.
CUtensorMap make_map(const EmuOperand& op, int box_rows) {
  RIS_REQUIRE(((uintptr_t)op.s & 15) == 0, RIS_ERR_ARG, "emu_gemm: slices not 16-byte aligned");
  RIS_REQUIRE(op.ldk % 8 == 0 && op.ldk >= op.K, RIS_ERR_ARG, "emu_gemm: ldk must be a multiple of 8");
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)op.ldk * 2, (cuuint64_t)op.ldk * op.rows * 2};
  cuuint32_t box[3] = {EBK, (cuuint32_t)box_rows, S};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void*)op.s, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  RIS_REQUIRE(r == CUDA_SUCCESS, RIS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// K-major operand tile, rows of 32 bytes with 32-byte swizzle: start
// address, leading offset unused (1), 256 B between 8-row groups,
// descriptor version 1, layout type 6 (SWIZZLE_32B).
__device__ __forceinline__ uint64_t desc_sw32(const void* p) {
  const uint64_t a = sa(p);
  return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46) |
         (6ull << 61);
}

// kind::f16 instruction descriptor: D FP32 (bit 4), A and B FP16 (0 at bits
// 7 and 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int bn) {
  return (1u << 4) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(EBM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// eight consecutive accumulator columns of this warp's 32 lanes, waited on
__device__ __forceinline__ void tmem_ld8_wait(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

struct EmuArgs {
  int M, N, K, bn;
  uint32_t idesc;
  const int* ea;
  const int* eb;
  EmuEpilogue ep;
  int* err;
};

__device__ __forceinline__ long long emu_off(int i, int in, long long ld, long long s) {
  return in > 0 ? (long long)(i / in) * ld + (long long)(i % in) * s : (long long)i * s;
}

__global__ void __launch_bounds__(128, 1) k_emu_gemm(const __grid_constant__ CUtensorMap mA,
                                                      const __grid_constant__ CUtensorMap mB,
                                                      EmuArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + ESTAGES * ESTAGE);
  uint64_t* empty = full + ESTAGES;
  uint64_t* done = empty + ESTAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bn = args.bn;
  const int n0 = blockIdx.x * bn, m0 = blockIdx.y * EBM;
  const int nk = (args.K + EBK - 1) / EBK;
  const uint32_t stage_tx = (uint32_t)(A_BYTES + S * bn * EBK * 2);

  if (threadIdx.x == 0) {
    for (int s = 0; s < ESTAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    int issued = 0;
    for (int i = 0; i < nk; i++) {
      const int s = i % ESTAGES;
      if (i >= ESTAGES && !mbar_wait(&empty[s], ((i / ESTAGES) - 1) & 1)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t* st = smem + s * ESTAGE;
      mbar_expect_tx(&full[s], stage_tx);
      tma_load(st, &mA, &full[s], i * EBK, m0, 0);
      tma_load(st + A_BYTES, &mB, &full[s], i * EBK, n0, 0);
      issued = i + 1;
    }
    for (int i = (issued > ESTAGES ? issued - ESTAGES : 0); i < issued; i++)
      mbar_wait(&full[i % ESTAGES], (i / ESTAGES) & 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: slice products p + q <= S - 1 (0-based) into accumulator p + q
    for (int i = 0; i < nk; i++) {
      const int s = i % ESTAGES;
      if (!mbar_wait(&full[s], (i / ESTAGES) & 1)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint8_t* st = smem + s * ESTAGE;
#pragma unroll
      for (int p = 0; p < S; p++) {
        const uint64_t da = desc_sw32(st + p * A_SLICE);
        for (int q = 0; q < S - p; q++) {
          const uint64_t db = desc_sw32(st + A_BYTES + q * bn * EBK * 2);
          mma_f16(tmem + (uint32_t)((p + q) * bn), da, db, args.idesc, (i > 0 || p > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  // epilogue
  const bool ok = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) *abort_flag = 1;
  __syncthreads();
  const bool good = *abort_flag == 0 && nk > 0;
  if (!good && threadIdx.x == 0 && nk > 0) atomicExch(args.err, 1);
  const int row = m0 + warp * 32 + lane;
  const EmuEpilogue& ep = args.ep;
  const bool live = good && row < args.M;
  const int er = live ? args.ea[row] : 0;
  const long long roff = emu_off(row, ep.rin, ep.rld, ep.rs);
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
  for (int c0 = 0; c0 < bn; c0 += 8) {
    float v[NG][8];
    __syncwarp();  // tcgen05.ld is warp-collective
#pragma unroll
    for (int g = 0; g < NG; g++) tmem_ld8_wait(lane_base + (uint32_t)(g * bn + c0), v[g]);
#pragma unroll
    for (int j = 0; j < 8 && live; j++) {
      const int col = n0 + c0 + j;
      if (col >= args.N) break;
      // sum_g V_g 2^(-6g) in 64-bit integers (the V_g are integers, below
      // 2^24 for g <= 7 and 2^25 for g = 8, 9): hi = V_0 2^12 + V_1 2^6 + V_2
      // and lo = sum_{g>=3} V_g 2^(6(9-g)) < 2^61, both exact; then two
      // conversions and one FMA in FP64
      const long long hi = __float2ll_rn(v[0][j]) * 4096 + __float2ll_rn(v[1][j]) * 64 +
                           __float2ll_rn(v[2][j]);
      long long lo = 0;
#pragma unroll
      for (int g = 3; g < NG; g++) lo += __float2ll_rn(v[g][j]) * (1ll << (kEmuBeta * (NG - 1 - g)));
      const double s = fma((double)hi, 0x1p-12, (double)lo * 0x1p-54);
      const double x = ldexp(s, er + args.eb[col] - 2 * kEmuBeta);
      double* p = ep.c64 + roff + emu_off(col, ep.cin, ep.cld, ep.cs);
      *p = ep.beta == 0.0 ? ep.alpha * x : fma(ep.alpha, x, ep.beta * *p);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

// Row exponents: E_r = 1 + max_k floor(log2 |x_rk|) (subnormals included;
// 0 for a row of zeros), so that every |x_rk| < 2^(E_r).
constexpr int kNoLead = -4096;
__device__ __forceinline__ int lead_exp(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7FF);
  if (ef) return ef - 1023;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  return m ? -1011 - __clzll(m) : kNoLead;  // -1074 + (63 - clz)
}
__device__ __forceinline__ int row_frame(int lead) { return lead == kNoLead ? 0 : lead + 1; }
__global__ void k_emu_rowexp(const double* __restrict__ src, int rows, int K, long long rs,
                             long long ks, int* __restrict__ E) {
  __shared__ int red[8][33];
  const int r = blockIdx.x * 32 + threadIdx.x;
  int m = kNoLead;
  if (r < rows)
    for (int k = threadIdx.y; k < K; k += 8) m = max(m, lead_exp(src[r * rs + k * ks]));
  red[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && r < rows) {
    for (int y = 1; y < 8; y++) m = max(m, red[y][threadIdx.x]);
    E[r] = row_frame(m);
  }
}
// Same for rows contiguous in k: one warp per row.
__global__ void k_emu_rowexp_rm(const double* __restrict__ src, int rows, int K, long long rs,
                                int* __restrict__ E) {
  const int r = blockIdx.x * 8 + threadIdx.y;
  if (r >= rows) return;
  int m = kNoLead;
  for (int k = threadIdx.x; k < K; k += 32) m = max(m, lead_exp(src[r * rs + k]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x == 0) E[r] = row_frame(m);
}

// Digits of one element in its row frame: X = floor(|x| 2^(F - E)) < 2^F
// with F = 6 S fraction bits (integer arithmetic on the FP64 fields),
// d_p = bits [F - 6p, F - 6p + 6) of X, signed like x.
__global__ void k_emu_digits(const double* __restrict__ src, int rows, int K, long long rs,
                             long long ks, const int* __restrict__ E, __half* __restrict__ out,
                             int ldk) {
  __shared__ double tile[32][33];  // [k][r]
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  if (ks == 1) {  // rows contiguous in k: lanes along k
    for (int rr = threadIdx.y; rr < 32; rr += 8) {
      const int r = r0 + rr, k = k0 + threadIdx.x;
      tile[threadIdx.x][rr] = (r < rows && k < K) ? src[r * rs + k] : 0.0;
    }
  } else {  // lanes along r
    for (int kk = threadIdx.y; kk < 32; kk += 8) {
      const int r = r0 + threadIdx.x, k = k0 + kk;
      tile[kk][threadIdx.x] = (r < rows && k < K) ? src[r * rs + k * ks] : 0.0;
    }
  }
  __syncthreads();
  const size_t plane = (size_t)rows * ldk;
  for (int rr = threadIdx.y; rr < 32; rr += 8) {
    const int r = r0 + rr, k = k0 + threadIdx.x;
    if (r >= rows || k >= ldk) continue;
    const unsigned long long b = (unsigned long long)__double_as_longlong(tile[threadIdx.x][rr]);
    const int ef = (int)((b >> 52) & 0x7FF);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    int q = -1074;  // |x| = m 2^q
    if (ef) {
      m |= 1ull << 52;
      q = ef - 1075;
    }
    // m 2^q < 2^E, so X = m 2^(q + F - E) < 2^F
    const int sh = q + kFracBits - E[r];
    const unsigned long long X = sh >= 0 ? (m << sh) : (sh <= -64 ? 0ull : (m >> -sh));
    const bool neg = (b >> 63) != 0;
    __half* o = out + (size_t)r * ldk + k;
#pragma unroll
    for (int p = 1; p <= S; p++) {
      const int d = (int)((X >> (kFracBits - kEmuBeta * p)) & 63);
      o[(size_t)(p - 1) * plane] = __int2half_rn(neg ? -d : d);
    }
  }
}

}  // namespace

void emu_slice(const double* src, int rows, int K, long long rs, long long ks, EmuOperand& op,
               cudaStream_t st) {
  RIS_REQUIRE(rows > 0 && K > 0 && op.s && op.e, RIS_ERR_ARG, "emu_slice: bad operand");
  op.rows = rows;
  op.K = K;
  op.ldk = ld8(K);
  if (ks == 1)
    k_emu_rowexp_rm<<<cdiv(rows, 8), dim3(32, 8), 0, st>>>(src, rows, K, rs, op.e);
  else
    k_emu_rowexp<<<cdiv(rows, 32), dim3(32, 8), 0, st>>>(src, rows, K, rs, ks, op.e);
  RIS_CHECK_LAUNCH();
  dim3 g((unsigned)cdiv(rows, 32), (unsigned)cdiv(op.ldk, 32));
  k_emu_digits<<<g, dim3(32, 8), 0, st>>>(src, rows, K, rs, ks, op.e, op.s, op.ldk);
  RIS_CHECK_LAUNCH();
}

void emu_gemm(int M, int N, const EmuOperand& A, const EmuOperand& B, const EmuEpilogue& ep,
              int* d_err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  RIS_REQUIRE(A.K == B.K && A.K > 0, RIS_ERR_ARG, "emu_gemm: contraction lengths differ");
  RIS_REQUIRE(A.rows >= M && B.rows >= N, RIS_ERR_ARG, "emu_gemm: operand rows");
  ensure_smem_attr((const void*)k_emu_gemm, ESMEM);
  // tile width: the tensor core reads the 128-row A slice from shared
  // memory for every product whatever BN, so a product costs about
  // (4096 + 32 BN) bytes of shared-memory traffic; take the width with the
  // least total over the column tiles
  int bn = EMAXBN;
  for (int c = EMAXBN; c >= 16; c -= 16)
    if ((long long)cdiv(N, c) * (4096 + 32 * c) < (long long)cdiv(N, bn) * (4096 + 32 * bn)) bn = c;
  const int K = A.K;
  EmuArgs a;
  a.M = M;
  a.N = N;
  a.bn = bn;
  a.idesc = idesc_f16(bn);
  a.ea = A.e;
  a.eb = B.e;
  a.err = d_err;
  dim3 grid(cdiv(N, bn), cdiv(M, EBM));
  prof_begin(kProfEmuGemm, st);
  for (int k0 = 0; k0 < K; k0 += kEmuKChunk) {
    // one exact pass per K chunk, accumulated in FP64 through the output
    EmuOperand ca = A, cb = B;
    ca.s = A.s + k0;
    cb.s = B.s + k0;
    ca.K = cb.K = std::min(kEmuKChunk, K - k0);
    const CUtensorMap mA = make_map(ca, EBM);
    const CUtensorMap mB = make_map(cb, bn);
    a.K = ca.K;
    a.ep = ep;
    if (k0 > 0) {
      a.ep.beta = 1.0;
    }
    k_emu_gemm<<<grid, 128, ESMEM, st>>>(mA, mB, a);
    RIS_CHECK_LAUNCH();
  }
  prof_end(kProfEmuGemm, st, 2.0 * M * N * (double)K);
}

}  // namespace ris

// Test hook (declared in include/ris.h): C = A B^T through the emulating
// GEMM for FP64 device operands on the current device.
extern "C" int ris_debug_gemm_f64emu(int M, int N, int K, const double* A, const double* B, double* C) {
  using namespace ris;
  try {
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return (int)RIS_ERR_ARG;
    cudaStream_t st = 0;
    const int lk = ld8(K);
    EmuOperand a, b;
    int* err;
    RIS_ALLOC(cudaMalloc(&a.s, sizeof(__half) * kEmuSlices * (size_t)M * lk));
    RIS_ALLOC(cudaMalloc(&b.s, sizeof(__half) * kEmuSlices * (size_t)N * lk));
    RIS_ALLOC(cudaMalloc(&a.e, sizeof(int) * (size_t)M));
    RIS_ALLOC(cudaMalloc(&b.e, sizeof(int) * (size_t)N));
    RIS_ALLOC(cudaMalloc(&err, sizeof(int)));
    RIS_CUDA(cudaMemset(err, 0, sizeof(int)));
    emu_slice(A, M, K, K, 1, a, st);
    emu_slice(B, N, K, K, 1, b, st);
    EmuEpilogue ep;
    ep.c64 = C;
    ep.rs = N;
    ep.cs = 1;
    emu_gemm(M, N, a, b, ep, err, st);
    int h_err = 0;
    RIS_CUDA(cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(a.s); cudaFree(b.s); cudaFree(a.e); cudaFree(b.e); cudaFree(err);
    return h_err ? (int)RIS_ERR_TIMEOUT : 0;
  } catch (const Error& e) {
    fprintf(stderr, "ris_debug_gemm_f64emu: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}
