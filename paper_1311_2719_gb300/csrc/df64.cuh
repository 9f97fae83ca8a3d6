// df64: a real number held as an unevaluated sum hi + lo of two FP32 values (|lo| <= ulp(hi)/2),
// carrying a 48-bit significand. Its arithmetic runs on the FP32 pipes, which on GB300 have
// about 58x the throughput of the FP64 pipe; it gives the half-lattice operator FP64-level
// accuracy (relative error ~1e-14) at HBM speed instead of the FP64-pipe limit.
//
// The operations are the classical error-free transformations (Dekker 1971; Knuth, TAOCP vol. 2,
// sec. 4.2.2): two-sum for additions and the FMA form of the exact product, a*b = p + e with
// e = fma(a, b, -p). Every step uses explicitly rounded intrinsics so that the compiler cannot
// contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace qcd {

struct df64 {
  float hi, lo;
  __host__ __device__ constexpr df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df64(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ df64(float v) : hi(v), lo(0.f) {}
  // nearest df64 to d: hi = round(d), lo = round(d - hi) (d - hi is exact in FP64)
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly (Knuth's two-sum, no ordering assumption)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, given |a| >= |b| (fast two-sum)
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df64 r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);           // exact error of a.hi * b.hi
  e = __fmaf_rn(a.hi, b.lo, e);                  // cross terms; a.lo * b.lo is below 2^-48
  e = __fmaf_rn(a.lo, b.hi, e);
  df64 r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }

// a * b + c with one renormalisation at the end.
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  float s, e;
  two_sum(p, c.hi, s, e);                         // s + e = p + c.hi exactly
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  df64 r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ bool isfinite(df64 a) { return ::isfinite(a.hi) && ::isfinite(a.lo); }

// The df64 overloads above would hide the CUDA math functions for unqualified calls inside
// namespace qcd; these forwarders keep float and double on the hardware instructions.
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fma(float a, float b, float c) { return ::fmaf(a, b, c); }
__host__ __device__ __forceinline__ bool isfinite(double a) { return ::isfinite(a); }
__host__ __device__ __forceinline__ bool isfinite(float a) { return ::isfinite(a); }

}  // namespace qcd
