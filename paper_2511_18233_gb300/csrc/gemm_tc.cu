// 3xTF32 GEMM on the 5th-generation tensor cores (tcgen05) of sm_103a.
//
// C = A . B^T with A [M][K] and B [N][K] in FP32 storage, each pre-split as
// x = x_hi + x_lo (x_hi = tf32(x), x_lo = tf32(x - x_hi)).  Every K step
// issues the three products hi.hi + hi.lo + lo.hi into one FP32 accumulator
// in tensor memory (the lo.lo term is below FP32 resolution), which keeps
// about FP32 accuracy at tensor-core rates.
//
// Kernel structure (one 128 x 128 output tile per CTA, 128 threads):
//   warp 0 / lane 0 : TMA producer, 3-stage ring of (A_hi, A_lo, B_hi, B_lo)
//                     tiles of 128 rows x 32 FP32 (128-byte swizzle)
//   warp 1          : allocates 128 TMEM columns; lane 0 issues
//                     tcgen05.mma.kind::tf32 (M=128, N=128, K=8) and commits
//                     each stage back to the producer through an mbarrier
//   warps 0-3       : epilogue, tcgen05.ld of TMEM lanes 32w..32w+31
// All mbarrier waits are bounded (about one second of clock64 cycles); a
// timeout sets the error flag, drains what this CTA has in flight and frees
// its TMEM before returning.
#include <cuda.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "gemm_tc.cuh"
#include "ff_arith.cuh"
#include "tc_ptx.cuh"

namespace ris {

namespace {
using namespace tcx;

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 4;                      // 16 KB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;                  // hi/lo of A and B
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;

// 3-D map {K, rows, batch} of FP32, box {32, 128, 1}, 128-byte swizzle.
CUtensorMap make_map(const float* base, int K, int rows, int ld, long long bstride, int nb) {
  RIS_REQUIRE(base != nullptr, RIS_ERR_ARG, "tc_gemm: null operand");
  RIS_REQUIRE(((uintptr_t)base & 15) == 0, RIS_ERR_ARG, "tc_gemm: operand not 16-byte aligned");
  RIS_REQUIRE(ld % 4 == 0 && (nb == 1 || bstride % 4 == 0), RIS_ERR_ARG,
              "tc_gemm: leading dimension / batch stride not a multiple of 16 bytes");
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)nb};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)(nb > 1 ? bstride : (long long)ld * rows) * 4};
  cuuint32_t box[3] = {BK, BM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  RIS_REQUIRE(r == CUDA_SUCCESS, RIS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// K-major operand tile of 128 rows x 128 bytes with 128-byte swizzle:
// start address, leading offset unused (1), stride 1024 B between 8-row
// groups, descriptor version 1, layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t desc_sw128(const void* p) {
  const uint64_t a = sa(p);
  return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// kind::tf32 instruction descriptor: D FP32 (bit 4), A and B TF32 (2 at bits
// 7 and 10), both K-major, N>>3 at bit 17, M>>4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct TcArgs {
  int M, N, K, nkb, ksplit, kb_per;
  int nbA, nbB;
  TcEpilogue ep;
  float* partial;  // split-K workspace [ksplit][M][N] (FP32) or null
  int* err;
};

__global__ void __launch_bounds__(128, 1) k_tc_gemm(const __grid_constant__ CUtensorMap mAh,
                                                     const __grid_constant__ CUtensorMap mAl,
                                                     const __grid_constant__ CUtensorMap mBh,
                                                     const __grid_constant__ CUtensorMap mBl,
                                                     TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  int z = blockIdx.z, ks = 0;
  if (args.ksplit > 1) {
    ks = z;
    z = 0;
  }
  const int kb0 = ks * args.kb_per, kb1 = min(args.nkb, kb0 + args.kb_per);
  const int zA = args.nbA > 1 ? z : 0, zB = args.nbB > 1 ? z : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int nk = kb1 - kb0;

  if (warp == 0 && lane == 0) {
    // producer
    int issued = 0;
    for (int i = 0; i < nk; i++) {
      const int s = i % STAGES;
      if (i >= STAGES && !mbar_wait(&empty[s], ((i / STAGES) - 1) & 1)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t* st = smem + s * STAGE_BYTES;
      const int kx = (kb0 + i) * BK;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load(st, &mAh, &full[s], kx, m0, zA);
      tma_load(st + TILE_BYTES, &mAl, &full[s], kx, m0, zA);
      tma_load(st + 2 * TILE_BYTES, &mBh, &full[s], kx, n0, zB);
      tma_load(st + 3 * TILE_BYTES, &mBl, &full[s], kx, n0, zB);
      issued = i + 1;
    }
    // drain: make sure every TMA this CTA issued has landed before exit
    for (int i = std::max(0, issued - STAGES); i < issued; i++)
      mbar_wait(&full[i % STAGES], (i / STAGES) & 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int i = 0; i < nk; i++) {
      const int s = i % STAGES;
      if (!mbar_wait(&full[s], (i / STAGES) & 1)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint8_t* st = smem + s * STAGE_BYTES;
      const uint64_t ah = desc_sw128(st), al = desc_sw128(st + TILE_BYTES);
      const uint64_t bh = desc_sw128(st + 2 * TILE_BYTES), bl = desc_sw128(st + 3 * TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 8; kk++) {
        const uint64_t off = (uint64_t)((kk * 32) >> 4);  // 32 bytes per K=8 step
        mma_tf32(tmem, ah + off, bl + off, (i > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, al + off, bh + off, 1u);
        mma_tf32(tmem, ah + off, bh + off, 1u);
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
  // Each warp owns 32 accumulator rows; a 32 x 32 block is read from TMEM
  // (one row per lane), transposed through shared memory (the pipeline
  // stages are idle now) and stored row by row with the lanes on consecutive
  // columns, so that every store instruction is coalesced.
  const TcEpilogue& ep = args.ep;
  float* tile = (float*)smem + warp * (32 * 33);
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int j = 0; j < 32; j++) tile[lane * 33 + j] = v[j];
    __syncwarp();
    const int col = n0 + c0 + lane;
    if (good && col < args.N) {
      const long long cpos = ep.cin > 0 ? (long long)(col / ep.cin) * ep.cld + (long long)(col % ep.cin) * ep.cs
                                        : (long long)col * ep.cs;
#pragma unroll 4
      for (int r = 0; r < 32; r++) {
        const int row = m0 + warp * 32 + r;
        if (row >= args.M) break;
        const float x = tile[r * 33 + lane];
        if (args.partial) {
          args.partial[((size_t)ks * args.M + row) * args.N + col] = x;
          continue;
        }
        const long long rpos = ep.rin > 0 ? (long long)(row / ep.rin) * ep.rld + (long long)(row % ep.rin) * ep.rs
                                          : (long long)row * ep.rs;
        const size_t off = (size_t)z * ep.bsc + (size_t)rpos + (size_t)cpos;
        if (ep.mode == kOutF64) {
          double* p = ep.c64 + off;
          *p = ep.beta == 0.0 ? ep.alpha * x : fma(ep.alpha, (double)x, ep.beta * *p);
        } else if (ep.mode == kOutF32) {
          float* p = ep.c32 + off;
          const float a = (float)ep.alpha, b = (float)ep.beta;
          *p = b == 0.f ? a * x : fmaf(a, x, b * *p);
        } else {
          const float y = (float)ep.alpha * x;
          const float h = to_tf32(y);
          ep.chi[off] = h;
          ep.clo[off] = to_tf32(y - h);
        }
      }
    }
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
  }
}

// The FP32 partial sums of the K slices are added in double-FP32 (TwoSum on
// the FP32 pipe, as exact as an FP64 sum) and widened once, so the FP64 pipe
// only applies alpha and beta.  32 outputs per CTA: warp g adds the slices
// g, g + 8, ... in order, then warp 0 the eight sums in order (a skinny
// product's many slices spread over many SMs; same result every run).
__global__ void __launch_bounds__(256) k_tc_reduce(int M, int N, int ksplit,
                                                   const float* __restrict__ part, double alpha,
                                                   double beta, double* __restrict__ C, int ldc) {
  __shared__ float2 red[8][32];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const long long mn = (long long)M * N;
  const long long t = (long long)blockIdx.x * 32 + lane;
  float S = 0.f, Cc = 0.f;
  if (t < mn)
    for (int z = g; z < ksplit; z += 8) ff_add(S, Cc, part[(size_t)z * mn + t], 0.f);
  red[g][lane] = make_float2(S, Cc);
  __syncthreads();
  if (g != 0 || t >= mn) return;
#pragma unroll
  for (int h = 1; h < 8; h++) ff_add(S, Cc, red[h][lane].x, red[h][lane].y);
  const int i = (int)(t / N), j = (int)(t % N);
  const double s = ff_widen(S) + ff_widen(Cc);
  double* p = C + (size_t)i * ldc + j;
  *p = beta == 0.0 ? alpha * s : fma(alpha, s, beta * *p);
}

__global__ void k_split(const double* __restrict__ src, int rows, int cols, long long lds, bool trans,
                        float* __restrict__ hi, float* __restrict__ lo, int ldd, long long sbs,
                        long long dbs) {
  // destination [rows'][ldd] with rows' = trans ? cols : rows, batch blockIdx.y
  const int drows = trans ? cols : rows, dcols = trans ? rows : cols;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)drows * ldd) return;
  src += (size_t)blockIdx.y * sbs;
  hi += (size_t)blockIdx.y * dbs;
  lo += (size_t)blockIdx.y * dbs;
  const int r = (int)(t / ldd), c = (int)(t % ldd);
  float x = 0.f;
  if (c < dcols) x = (float)(trans ? src[(size_t)c * lds + r] : src[(size_t)r * lds + c]);
  const float h = to_tf32(x);
  hi[t] = h;
  lo[t] = to_tf32(x - h);
}

// Tiled transpose + split: src X[r][c] (r < nr, c < nc, row length nc) to
// dst[c][r / nin][r % nin] with the inner index padded to ldin.
__global__ void k_split_tpad(const double* __restrict__ X, long long nr, int nc, int nin, int ldin,
                             float* __restrict__ hi, float* __restrict__ lo) {
  __shared__ float tile[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const long long r = r0 + y;
    const int c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (r < nr && c < nc) ? (float)X[(size_t)r * nc + c] : 0.f;
  }
  __syncthreads();
  const long long nouter = nr / nin;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int c = c0 + y;
    const long long r = r0 + threadIdx.x;
    if (c >= nc || r >= nr) continue;
    const float x = tile[threadIdx.x][y];
    const size_t d = ((size_t)c * nouter + (size_t)(r / nin)) * ldin + (size_t)(r % nin);
    const float h = to_tf32(x);
    hi[d] = h;
    lo[d] = to_tf32(x - h);
  }
}

}  // namespace

void split_f64_tpad(const double* src, long long nr, int nc, int nin, int ldin, float* hi,
                    float* lo, cudaStream_t st) {
  RIS_REQUIRE(nin > 0 && nr % nin == 0 && ldin >= nin, RIS_ERR_ARG, "split_f64_tpad: bad shape");
  dim3 g((unsigned)cdiv(nr, 32), (unsigned)cdiv(nc, 32));
  k_split_tpad<<<g, dim3(32, 8), 0, st>>>(src, nr, nc, nin, ldin, hi, lo);
  RIS_CHECK_LAUNCH();
}

void split_f64(const double* src, int rows, int cols, long long lds, float* hi, float* lo, int ldd,
               cudaStream_t st, int nbatch, long long sbs, long long dbs) {
  dim3 g(cdiv((long long)rows * ldd, 256), nbatch);
  k_split<<<g, 256, 0, st>>>(src, rows, cols, lds, false, hi, lo, ldd, sbs, dbs);
  RIS_CHECK_LAUNCH();
}
void split_f64_t(const double* src, int rows, int cols, long long lds, float* hi, float* lo, int ldd,
                 cudaStream_t st, int nbatch, long long sbs, long long dbs) {
  dim3 g(cdiv((long long)cols * ldd, 256), nbatch);
  k_split<<<g, 256, 0, st>>>(src, rows, cols, lds, true, hi, lo, ldd, sbs, dbs);
  RIS_CHECK_LAUNCH();
}

// Longest contraction accumulated in one TMEM accumulator.  The tensor
// core's FP32 accumulation loses precision with every MMA it adds (its
// error grows about linearly with the number of K steps), so longer
// contractions with an FP64 output run as chunks of at most this length
// whose results are summed in FP64 by the epilogue.
constexpr int kTcKChunk = 16384;

void tc_gemm(int M, int N, int K, const TcOperand& A, const TcOperand& B, int nb, const TcEpilogue& ep,
             int* d_err, cudaStream_t st, float* ws, size_t ws_floats, bool allow_alloc) {
  if (M <= 0 || N <= 0 || nb <= 0) return;
  RIS_REQUIRE(K > 0, RIS_ERR_ARG, "tc_gemm: K must be positive");
  if (ep.mode == kOutF64 && K > kTcKChunk) {
    for (int k0 = 0; k0 < K; k0 += kTcKChunk) {
      TcOperand a = A, b = B;
      a.hi += k0;
      a.lo += k0;
      b.hi += k0;
      b.lo += k0;
      TcEpilogue e = ep;
      if (k0 > 0) e.beta = 1.0;
      tc_gemm(M, N, std::min(kTcKChunk, K - k0), a, b, nb, e, d_err, st, ws, ws_floats, allow_alloc);
    }
    return;
  }
  RIS_REQUIRE(A.rows >= M && B.rows >= N, RIS_ERR_ARG, "tc_gemm: operand rows");
  RIS_REQUIRE(nb <= 65535, RIS_ERR_ARG, "tc_gemm: batch too large");
  ensure_smem_attr((const void*)k_tc_gemm, SMEM_BYTES);
  const CUtensorMap mAh = make_map(A.hi, K, M, A.ld, A.bstride, A.nb);
  const CUtensorMap mAl = make_map(A.lo, K, M, A.ld, A.bstride, A.nb);
  const CUtensorMap mBh = make_map(B.hi, K, N, B.ld, B.bstride, B.nb);
  const CUtensorMap mBl = make_map(B.lo, K, N, B.ld, B.bstride, B.nb);
  TcArgs a;
  a.M = M;
  a.N = N;
  a.K = K;
  a.nkb = cdiv(K, BK);
  a.nbA = A.nb;
  a.nbB = B.nb;
  a.ep = ep;
  a.err = d_err;
  a.partial = nullptr;
  a.ksplit = 1;
  a.kb_per = 1;
  const int tiles = cdiv(M, BM) * cdiv(N, BN);
  a.kb_per = a.nkb;
  if (nb == 1 && ep.mode == kOutF64 && ep.cs == 1 && ep.cin == 0 && ep.rin == 0 && tiles < 152 &&
      a.nkb >= 8) {
    int ks = std::max(1, std::min(std::max(1, 152 / tiles), a.nkb / 4));
    a.kb_per = cdiv(a.nkb, ks);
    a.ksplit = cdiv(a.nkb, a.kb_per);  // every slice non-empty
  }
  float* part = nullptr;
  bool own_part = false;
  MemTrack* part_tr = nullptr;
  if (a.ksplit > 1) {
    const size_t need = (size_t)a.ksplit * M * N;
    if (ws && ws_floats >= need) {
      part = ws;
    } else if (allow_alloc) {
      part = (float*)dev_alloc(sizeof(float) * need, st, &part_tr);
      own_part = true;
    } else {
      a.ksplit = 1;
      a.kb_per = a.nkb;
    }
    a.partial = part;
  }
  dim3 grid(cdiv(N, BN), cdiv(M, BM), a.ksplit > 1 ? a.ksplit : nb);
  prof_begin(kProfTcGemm, st);
  k_tc_gemm<<<grid, 128, SMEM_BYTES, st>>>(mAh, mAl, mBh, mBl, a);
  RIS_CHECK_LAUNCH();
  if (a.ksplit > 1) {
    k_tc_reduce<<<cdiv((long long)M * N, 32), 256, 0, st>>>(M, N, a.ksplit, part, ep.alpha, ep.beta,
                                                            ep.c64, (int)ep.rs);
    RIS_CHECK_LAUNCH();
    if (own_part) dev_free(part, sizeof(float) * (size_t)a.ksplit * M * N, st, part_tr);
  }
  prof_end(kProfTcGemm, st, 2.0 * M * N * (double)K * nb);
}

}  // namespace ris

// Test hook (declared in include/ris.h): C = A B^T in 3xTF32 on the
// tensor cores for FP64 inputs on the current device.
extern "C" int ris_debug_gemm_tf32x3(int M, int N, int K, const double* A, const double* B, double* C) {
  using namespace ris;
  try {
    cudaStream_t st = 0;
    const int ld = ld4(K);
    float *ah, *al, *bh, *bl;
    int* err;
    RIS_ALLOC(cudaMalloc(&ah, sizeof(float) * (size_t)M * ld));
    RIS_ALLOC(cudaMalloc(&al, sizeof(float) * (size_t)M * ld));
    RIS_ALLOC(cudaMalloc(&bh, sizeof(float) * (size_t)N * ld));
    RIS_ALLOC(cudaMalloc(&bl, sizeof(float) * (size_t)N * ld));
    RIS_ALLOC(cudaMalloc(&err, sizeof(int)));
    RIS_CUDA(cudaMemset(err, 0, sizeof(int)));
    split_f64(A, M, K, K, ah, al, ld, st);
    split_f64(B, N, K, K, bh, bl, ld, st);
    TcOperand a, b;
    a.hi = ah; a.lo = al; a.rows = M; a.ld = ld;
    b.hi = bh; b.lo = bl; b.rows = N; b.ld = ld;
    TcEpilogue ep;
    ep.mode = kOutF64;
    ep.c64 = C;
    ep.rs = N;
    tc_gemm(M, N, K, a, b, 1, ep, err, st);
    int h_err = 0;
    RIS_CUDA(cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(ah); cudaFree(al); cudaFree(bh); cudaFree(bl); cudaFree(err);
    return h_err ? (int)RIS_ERR_TIMEOUT : 0;
  } catch (const Error& e) {
    fprintf(stderr, "ris_debug_gemm_tf32x3: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the 3xTF32 GEMM (declared in include/ris.h).
//
// Its scratch lives in one file-scope device array, set aside when the
// library is loaded on a device and held until the process exits:
//   [0, 64)       the pipeline error flag (cleared at the start of each call)
//   [64, ...)     hi/lo FP32 splits of A and B, then split-K partial sums.
// Host code cannot use the array's name as a device address, so the first
// call on each device looks its address up with cudaGetSymbolAddress (with
// that device current) and caches it.
namespace ris {
namespace {
constexpr size_t kNoAllocFloats = (size_t)8 << 20;  // 8 Mi floats = 32 MiB
__device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

float* noalloc_scratch() {
  static std::mutex mu;
  static std::map<int, float*> addr;
  int dev = 0;
  RIS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(mu);
  auto it = addr.find(dev);
  if (it != addr.end()) return it->second;
  float* p = nullptr;
  RIS_CUDA(cudaGetSymbolAddress((void**)&p, g_noalloc_scratch));
  addr[dev] = p;
  return p;
}
}  // namespace
}  // namespace ris

extern "C" int ris_gemm_tf32x3_noalloc(int M, int N, int K, const double* A, const double* B,
                                       double* C, void* stream) {
  using namespace ris;
  try {
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return (int)RIS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ld = (size_t)ld4(K);
    const size_t need = 64 + 2 * ((size_t)M + N) * ld;
    if (need > kNoAllocFloats) {
      fprintf(stderr,
              "ris_gemm_tf32x3_noalloc: 2*(M+N)*ceil4(K) + 64 = %zu floats exceeds the "
              "preallocated scratch of %zu floats\n",
              need, kNoAllocFloats);
      return (int)RIS_ERR_ARG;
    }
    float* base = noalloc_scratch();
    int* err = (int*)base;
    float* ah = base + 64;
    float* al = ah + (size_t)M * ld;
    float* bh = al + (size_t)M * ld;
    float* bl = bh + (size_t)N * ld;
    float* ws = bl + (size_t)N * ld;
    RIS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    split_f64(A, M, K, K, ah, al, (int)ld, st);
    split_f64(B, N, K, K, bh, bl, (int)ld, st);
    TcOperand a, b;
    a.hi = ah; a.lo = al; a.rows = M; a.ld = (int)ld;
    b.hi = bh; b.lo = bl; b.rows = N; b.ld = (int)ld;
    TcEpilogue ep;
    ep.mode = kOutF64;
    ep.c64 = C;
    ep.rs = N;
    tc_gemm(M, N, K, a, b, 1, ep, err, st, ws, kNoAllocFloats - need, false);
    int h_err = 0;
    RIS_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
    return h_err ? (int)RIS_ERR_TIMEOUT : 0;
  } catch (const Error& e) {
    fprintf(stderr, "ris_gemm_tf32x3_noalloc: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}
