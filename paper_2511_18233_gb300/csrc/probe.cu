// Peak-rate probes of the arithmetic pipes the engine's kernels are bound by:
// FP64 and FP32 FMA (the integral recursions and SIMT GEMMs), FP64 MMA
// (mma.sync m16n8k4, the only FP64 tensor instruction), and the tcgen05
// tensor pipe in kind::tf32 (the 3xTF32 products) and kind::f16 (the
// FP64-emulating digit-slice products).  Each probe issues independent
// operations back to back and is timed with CUDA events; the rates are the
// denominators of the kernels' roofline fractions.
#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace ris {
namespace {
using namespace tcx;

constexpr int kChains = 8;  // independent FMA chains per thread

template <class T>
__global__ void __launch_bounds__(256) k_probe_fma(int iters, T x, T y, T* sink) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) a[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = a[c] * x + y;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += a[c];
  if (s == (T)-1.2345) sink[0] = s;  // keeps the chains live
}

// FP64 mma.sync m16n8k4 (per thread: two A, one B, four C/D elements):
// four independent accumulators per warp.
__global__ void __launch_bounds__(256) k_probe_dmma(int iters, double* sink) {
  const double a0 = 1.0 + 1e-3 * threadIdx.x, a1 = 1.0 - 2e-3 * threadIdx.x,
               b = 1.0 - 1e-3 * threadIdx.x;
  double d[4][4] = {};
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < 4; c++)
      asm volatile(
          "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
          "{%0,%1,%2,%3};"
          : "+d"(d[c][0]), "+d"(d[c][1]), "+d"(d[c][2]), "+d"(d[c][3])
          : "d"(a0), "d"(a1), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < 4; c++) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
  if (s == -1.2345) sink[0] = s;
}

// tcgen05 MMA issue loop: one CTA per SM, one thread issues `iters`
// M = 128, N = 256 MMAs from fixed shared-memory operands (128-byte swizzled
// K-major tiles) into one TMEM accumulator, commits, and waits (bounded).
constexpr int kPM = 128, kPN = 256;
constexpr int kPA = kPM * 128, kPB = kPN * 128;  // bytes: 128 bytes of K per row
constexpr int kPSmem = kPA + kPB + 1024 + 64;

__device__ __forceinline__ uint64_t pdesc(const void* p) {
  const uint64_t a = sa(p);
  return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// kind: 0 = tf32 (K = 8 per instruction), 1 = f16 (K = 16)
__global__ void __launch_bounds__(128, 1) k_probe_tc(int iters, int kind, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* done = (uint64_t*)(smem + kPA + kPB);
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  const int warp = threadIdx.x >> 5;
  // operand tiles: small nonzero values (a hashed pattern) so that the pipe
  // switches like it does on real data
  for (int i = threadIdx.x; i < (kPA + kPB) / 4; i += blockDim.x) {
    const uint32_t h = (uint32_t)i * 2654435761u;
    if (kind == 0) {
      ((float*)smem)[i] = 0.5f + (float)(h >> 9) * 1e-8f;
    } else {
      const __half v = __float2half(0.5f + (float)(h >> 12) * 1e-6f);
      ((__half*)smem)[2 * i] = v;
      ((__half*)smem)[2 * i + 1] = v;
    }
  }
  if (threadIdx.x == 0) {
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                 "r"(kPN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (threadIdx.x == 0) {
    const uint64_t da = pdesc(smem), db = pdesc(smem + kPA);
    const uint32_t idesc = kind == 0
                               ? ((1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kPN >> 3) << 17) |
                                  ((uint32_t)(kPM >> 4) << 24))
                               : ((1u << 4) | ((uint32_t)(kPN >> 3) << 17) | ((uint32_t)(kPM >> 4) << 24));
    for (int i = 0; i < iters; i++) {
      // step through the four 32-byte K slices of the 128-byte rows
      const uint64_t off = (uint64_t)(((i & 3) * 32) >> 4);
      const uint32_t acc = i > 0 ? 1u : 0u;
      if (kind == 0)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da + off), "l"(db + off), "r"(idesc), "r"(acc)
            : "memory");
      else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da + off), "l"(db + off), "r"(idesc), "r"(acc)
            : "memory");
    }
    mma_commit(done);
    if (!mbar_wait(done, 0)) {
      atomicExch(err, 1);
      mbar_wait(done, 0);  // the MMAs must finish before TMEM is released
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPN) : "memory");
}

}  // namespace
}  // namespace ris

// Test hook (declared in include/ris.h): measured rate of one pipe.
extern "C" int ris_debug_peak_probe(int kind, int reps, double* tflops, double* ms_out) {
  using namespace ris;
  if (kind < 0 || kind > 4 || reps < 1 || !tflops) return (int)RIS_ERR_ARG;
  try {
    int dev = 0, nsm = 0;
    RIS_CUDA(cudaGetDevice(&dev));
    RIS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = 0;
    void* sink = nullptr;
    RIS_ALLOC(cudaMalloc(&sink, 64));
    RIS_CUDA(cudaMemset(sink, 0, 64));
    cudaEvent_t e0, e1;
    RIS_CUDA(cudaEventCreate(&e0));
    RIS_CUDA(cudaEventCreate(&e1));
    if (kind >= 3) ensure_smem_attr((const void*)k_probe_tc, kPSmem);
    double best = 0.0, best_ms = 0.0;
    for (int r = 0; r < reps + 1; r++) {  // the first run warms up
      double flops = 0.0;
      RIS_CUDA(cudaEventRecord(e0, st));
      if (kind == 0 || kind == 1) {
        const int blocks = nsm * 8, iters = kind == 0 ? 2048 : 16384;
        if (kind == 0)
          k_probe_fma<double><<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7, (double*)sink);
        else
          k_probe_fma<float><<<blocks, 256, 0, st>>>(iters, 0.9999f, 1e-5f, (float*)sink);
        flops = 2.0 * kChains * (double)iters * blocks * 256;
      } else if (kind == 2) {
        const int blocks = nsm * 8, iters = 2048;
        k_probe_dmma<<<blocks, 256, 0, st>>>(iters, (double*)sink);
        flops = 4.0 * 2.0 * 16 * 8 * 4 * (double)iters * blocks * 8;  // 8 warps per block
      } else {
        const int iters = kind == 3 ? 100000 : 50000;
        k_probe_tc<<<nsm, 128, kPSmem, st>>>(iters, kind - 3, (int*)sink);
        flops = 2.0 * kPM * kPN * (kind == 3 ? 8 : 16) * (double)iters * nsm;
      }
      RIS_CHECK_LAUNCH();
      RIS_CUDA(cudaEventRecord(e1, st));
      RIS_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      RIS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      const double rate = flops / (ms * 1e-3) / 1e12;
      if (r > 0 && rate > best) {
        best = rate;
        best_ms = ms;
      }
    }
    int h_err = 0;
    if (kind >= 3) RIS_CUDA(cudaMemcpy(&h_err, sink, sizeof(int), cudaMemcpyDeviceToHost));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (h_err) return (int)RIS_ERR_TIMEOUT;
    *tflops = best;
    if (ms_out) *ms_out = best_ms;
    return 0;
  } catch (const Error& e) {
    fprintf(stderr, "ris_debug_peak_probe: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}
