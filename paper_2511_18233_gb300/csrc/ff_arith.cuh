// Double-FP32 arithmetic: FP64 values carried as unevaluated sums of two
// FP32 numbers, with error-free transforms on the FP32 pipe (GB300 issues
// FP32 operations about 72 times faster than FP64 ones).  Every FP32
// operation here rounds to nearest and is never contracted (intrinsics).
// Used by the double-FP32 GEMM (gemm_ff.cu) and by the tensor-core GEMM's
// split-K reduction.
#pragma once
#include "common.cuh"

namespace ris {

// x = hi + lo + r: hi the leading 24 significand bits of x and lo the next
// 29 rounded to 24, by integer operations on the bit pattern (no FP64
// instruction); |r| <= 2^-47 |x| for |x| >= 2^-74.  Below that lo would
// leave the FP32 normal range and is dropped (|r| < 2^-97); |x| < 2^-126
// flushes to zero and |x| >= 2^128 becomes +-inf.
__device__ __forceinline__ void ff_split(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const unsigned long long f = b & 0xfffffffffffffULL;
  if (e < -126) {  // zero, FP64 subnormal, or below the FP32 normal range
    hi = 0.f;
    lo = 0.f;
    return;
  }
  if (e > 127) {  // beyond the FP32 range (or inf / nan)
    hi = __uint_as_float(sgn | 0x7f800000u);
    lo = 0.f;
    return;
  }
  hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (unsigned)(f >> 29));
  const unsigned r = (unsigned)(f & 0x1fffffffu);  // value r * 2^(e-52)
  if (r == 0u || e < -74) {  // 2^(e-52) below the FP32 normal range: lo < 2^-97, dropped
    lo = 0.f;
    return;
  }
  const float sc = __uint_as_float((unsigned)(e + 75) << 23);  // 2^(e-52)
  lo = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(r), sc)) | sgn);
}

// FP32 -> FP64 by the bit pattern (FP32 subnormals flush to zero).
__device__ __forceinline__ double ff_widen(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u) return 0.0;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long e64 = ex == 0xffu ? 0x7ffULL : (unsigned long long)(ex + 896u);
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(s | (e64 << 52) | m));
}

// (s, c) += (ah + al) (bh + bl)
__device__ __forceinline__ void ff_term(float ah, float al, float bh, float bl, float& s, float& c) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e))));
}

// (s, c) <- TwoSum(s, c) + c's remainder
__device__ __forceinline__ void ff_renorm(float& s, float& c) {
  const float t = __fadd_rn(s, c);
  const float z = __fsub_rn(t, s);
  c = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(c, z));
  s = t;
}

// (S, C) += (s, c)
__device__ __forceinline__ void ff_add(float& S, float& C, float s, float c) {
  const float t = __fadd_rn(S, s);
  const float z = __fsub_rn(t, S);
  const float q = __fadd_rn(__fsub_rn(S, __fsub_rn(t, z)), __fsub_rn(s, z));
  S = t;
  C = __fadd_rn(C, __fadd_rn(q, c));
}

}  // namespace ris
