// Common definitions for the TDDFT-ris sm_103a library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ris.h"

namespace ris {

// Highest angular momenta handled by the integral kernels.
constexpr int kMaxLAO = 2;   // AO shells up to d
constexpr int kMaxLAux = 2;  // auxiliary shells up to d
// Boys table: F_m(k*dT) for m <= kBoysM, k*dT <= kBoysTmax.
constexpr int kBoysM = 16;
constexpr double kBoysDT = 0.05;
constexpr double kBoysTmax = 40.0;
constexpr int kBoysNT = 801;  // kBoysTmax/kBoysDT + 1
constexpr int kBoysTaylor = 8;

struct Error {
  ris_status code;
  std::string msg;
};

#define RIS_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw ::ris::Error{RIS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// Every kernel launch is followed by RIS_CHECK_LAUNCH, which also counts it.
extern std::atomic<long long> g_launches;
// Device allocations made by the library since it was loaded (every
// cudaMalloc / cudaMallocAsync goes through RIS_ALLOC or dev_alloc).
extern std::atomic<long long> g_allocs;
#define RIS_ALLOC(call)  \
  do {                   \
    ++::ris::g_allocs;   \
    RIS_CUDA(call);      \
  } while (0)
#define RIS_CHECK_LAUNCH()        \
  do {                            \
    ++::ris::g_launches;          \
    RIS_CUDA(cudaGetLastError()); \
  } while (0)

// Optional per-kernel-class timing with CUDA events on the launching stream
// (enabled by the profile option; off by default).
enum ProfClass {
  kProfGemm = 0, kProfInt3c, kProfInt3cDeriv, kProfContract, kProfEig, kProfTcGemm, kProfEmuGemm,
  kProfFF, kProfN
};
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st, double work);
void prof_attach(cudaStream_t st);  // time the classes launched on st
void prof_detach(cudaStream_t st);
// sums per class of the records on the given streams since their last collect
void prof_collect(const cudaStream_t* sts, int n, double* ms, double* work);

#define RIS_REQUIRE(cond, code, text)                    \
  do {                                                   \
    if (!(cond)) throw ::ris::Error{code, std::string(text)}; \
  } while (0)

__host__ __device__ inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Device bytes a context holds: now and the high-water mark since it was
// created or last trimmed.  A context is driven by one host thread at a time,
// so the counters need no atomics.
struct MemTrack {
  long long cur = 0, peak = 0;
  void add(long long b) {
    cur += b;
    if (cur > peak) peak = cur;
  }
};
// Tracker of the context the calling thread is serving (set per API call).
extern thread_local MemTrack* t_track;

// Stream-ordered allocation from the device's default pool (no device-wide
// synchronisation, unlike cudaMalloc / cudaFree), counted against t_track.
// Throws RIS_ERR_OOM.
void* dev_alloc(size_t bytes, cudaStream_t st, MemTrack** owner);
void dev_free(void* p, size_t bytes, cudaStream_t st, MemTrack* owner);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (kernel, device),
// safe to call from several threads.
void ensure_smem_attr(const void* func, int bytes);

}  // namespace ris
