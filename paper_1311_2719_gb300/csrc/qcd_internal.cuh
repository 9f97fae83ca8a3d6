// Internal types shared by the library's translation units: lattice geometry on the device,
// complex colour algebra, packed field / link accessors for every precision, and the
// deterministic block reduction used by the fused CG epilogues.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qcd.h"
#include "df64.cuh"

namespace qcd {

constexpr int kBlock = 128;           // threads per block of the site kernels
constexpr int kSpreadBlockMax = 512;  // widest block of the CG kernels on lattices below one wave
constexpr int kMaxPartials = 8192;    // per-reduction partial slots in the workspace
constexpr int kMaxRhs = 16;
// shared-link multi-RHS operators (staggered and Wilson): tiles of kShTile sites, kShWarps warps
constexpr int kShTile = 32;
constexpr int kShWarps = 8;
constexpr int kShThreads = kShTile * kShWarps;
constexpr int kRhsShared = -1;  // the rhs_block option value that selects them
static_assert(2 * kShWarps >= kMaxRhs, "two right-hand sides per warp cover every RHS");

// ------------------------------------------------------------------------------------------
// Host-side handle.
// ------------------------------------------------------------------------------------------
struct LinkSet {
  void* ptr = nullptr;  // caller-owned packed links
  int recon = 0;        // 0 = not loaded
};

}  // namespace qcd

struct qcd_lattice {
  int L[4];
  long long V;
  long long Vh;
  int tbc;
  int device;
  qcd::LinkSet links[4];  // indexed by precision
  void* wilson_links[4] = {nullptr, nullptr, nullptr, nullptr};  // Wilson operator links by precision
                                                                 // (FP64, FP32, -, df64; caller-owned)
};

namespace qcd {

// ------------------------------------------------------------------------------------------
// Device geometry: even-odd index <-> coordinates and neighbours (the paper's iup/idn, computed).
// ------------------------------------------------------------------------------------------
// Division of a non-negative int by a run-time constant d >= 1 as a multiply-high and shifts
// (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994, §4:
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0)
// with t = the high half of m n; exact for every 32-bit unsigned n). Every site kernel turns its
// index into coordinates with three divisions and two remainders by the extents; compiled as
// integer divisions they are long instruction sequences in kernels that are issue-limited.
struct FastDiv {
  unsigned d, m;
  int s1, s2;
};
inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (unsigned)((((1ull << l) - d) << 32) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}
__host__ __device__ __forceinline__ unsigned umulhi32(unsigned a, unsigned b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (unsigned)(((unsigned long long)a * b) >> 32);
#endif
}
__host__ __device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
  const unsigned t = umulhi32(f.m, (unsigned)n);
  return (int)((t + (((unsigned)n - t) >> f.s1)) >> f.s2);
}

struct Geom {
  int L0, L1, L2, L3;
  int Vh;
  float tbc;  // +1 or -1
  FastDiv d0, d1, d2, d3;  // division by L0 .. L3
};

inline Geom make_geom(const qcd_lattice* lat) {
  Geom g;
  g.L0 = lat->L[0]; g.L1 = lat->L[1]; g.L2 = lat->L[2]; g.L3 = lat->L[3];
  g.Vh = (int)lat->Vh;
  g.tbc = (float)lat->tbc;
  g.d0 = make_fastdiv((unsigned)g.L0);
  g.d1 = make_fastdiv((unsigned)g.L1);
  g.d2 = make_fastdiv((unsigned)g.L2);
  g.d3 = make_fastdiv((unsigned)g.L3);
  return g;
}

struct Site {
  int x0, x1, x2, x3;
  int lex;  // canonical index
};

// Coordinates of even-odd site k of parity `par`: the canonical pair (2k, 2k+1) shares x1..x3
// and holds one site of each parity because L0 is even.
__device__ __forceinline__ Site site_of(const Geom& g, int k, int par) {
  Site s;
  int j = 2 * k;
  int t = fdiv(j, g.d0);
  int x0e = j - t * g.L0;
  const int t1 = fdiv(t, g.d1);
  s.x1 = t - t1 * g.L1;
  s.x3 = fdiv(t1, g.d2);
  s.x2 = t1 - s.x3 * g.L2;
  s.x0 = x0e + ((s.x1 + s.x2 + s.x3 + par) & 1);
  s.lex = j + (s.x0 - x0e);
  return s;
}

// Even-odd index of the forward (n + mu) and backward (n - mu) neighbours.
__device__ __forceinline__ void neighbours(const Geom& g, const Site& s, int fwd[4], int bwd[4]) {
  const int st1 = g.L0, st2 = g.L0 * g.L1, st3 = g.L0 * g.L1 * g.L2;
  fwd[0] = (s.x0 == g.L0 - 1 ? s.lex - (g.L0 - 1) : s.lex + 1) >> 1;
  bwd[0] = (s.x0 == 0 ? s.lex + (g.L0 - 1) : s.lex - 1) >> 1;
  fwd[1] = (s.x1 == g.L1 - 1 ? s.lex - (g.L1 - 1) * st1 : s.lex + st1) >> 1;
  bwd[1] = (s.x1 == 0 ? s.lex + (g.L1 - 1) * st1 : s.lex - st1) >> 1;
  fwd[2] = (s.x2 == g.L2 - 1 ? s.lex - (g.L2 - 1) * st2 : s.lex + st2) >> 1;
  bwd[2] = (s.x2 == 0 ? s.lex + (g.L2 - 1) * st2 : s.lex - st2) >> 1;
  fwd[3] = (s.x3 == g.L3 - 1 ? s.lex - (g.L3 - 1) * st3 : s.lex + st3) >> 1;
  bwd[3] = (s.x3 == 0 ? s.lex + (g.L3 - 1) * st3 : s.lex - st3) >> 1;
}

// eta_mu(n) * zeta_mu(n) of the link U_mu(n) (forward) and of U_mu(n - mu) (backward), as +-1.
__device__ __forceinline__ float fwd_sign(const Geom& g, const Site& s, int mu) {
  int e = 0;
  if (mu >= 1) e += s.x0;
  if (mu >= 2) e += s.x1;
  if (mu >= 3) e += s.x2;
  float sg = (e & 1) ? -1.f : 1.f;
  if (mu == 3 && s.x3 == g.L3 - 1) sg *= g.tbc;
  return sg;
}
__device__ __forceinline__ float bwd_sign(const Geom& g, const Site& s, int mu) {
  // eta_mu(n - mu) = eta_mu(n); zeta of the link at n - mu is tbc when x3(n) == 0.
  int e = 0;
  if (mu >= 1) e += s.x0;
  if (mu >= 2) e += s.x1;
  if (mu >= 3) e += s.x2;
  float sg = (e & 1) ? -1.f : 1.f;
  if (mu == 3 && s.x3 == 0) sg *= g.tbc;
  return sg;
}

// ------------------------------------------------------------------------------------------
// Complex colour algebra in the compute type T (double or float).
// ------------------------------------------------------------------------------------------
template <typename T>
struct cplx {
  T re, im;
};

template <typename T>
struct cvec3 {
  cplx<T> c[3];
};

template <typename T>
struct su3 {
  cplx<T> e[3][3];
};

template <typename T>
__device__ __forceinline__ void zero(cvec3<T>& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) v.c[a].re = v.c[a].im = T(0);
}

// acc += U x
template <typename T>
__device__ __forceinline__ void mul_add(cvec3<T>& acc, const su3<T>& U, const cvec3<T>& x) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      acc.c[a].re = fma(U.e[a][b].re, x.c[b].re, acc.c[a].re);
      acc.c[a].re = fma(-U.e[a][b].im, x.c[b].im, acc.c[a].re);
      acc.c[a].im = fma(U.e[a][b].re, x.c[b].im, acc.c[a].im);
      acc.c[a].im = fma(U.e[a][b].im, x.c[b].re, acc.c[a].im);
    }
  }
}

// acc -= U^dagger x
template <typename T>
__device__ __forceinline__ void adj_mul_sub(cvec3<T>& acc, const su3<T>& U, const cvec3<T>& x) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // conj(U_ba) x_b = (U_re - i U_im)(x_re + i x_im)
      acc.c[a].re = fma(-U.e[b][a].re, x.c[b].re, acc.c[a].re);
      acc.c[a].re = fma(-U.e[b][a].im, x.c[b].im, acc.c[a].re);
      acc.c[a].im = fma(-U.e[b][a].re, x.c[b].im, acc.c[a].im);
      acc.c[a].im = fma(U.e[b][a].im, x.c[b].re, acc.c[a].im);
    }
  }
}

// w = U x
template <typename T>
__device__ __forceinline__ cvec3<T> mul(const su3<T>& U, const cvec3<T>& x) {
  cvec3<T> w;
  zero(w);
  mul_add(w, U, x);
  return w;
}

// w = U^dagger x
template <typename T>
__device__ __forceinline__ cvec3<T> adj_mul(const su3<T>& U, const cvec3<T>& x) {
  cvec3<T> w;
  zero(w);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      w.c[a].re = fma(U.e[b][a].re, x.c[b].re, w.c[a].re);
      w.c[a].re = fma(U.e[b][a].im, x.c[b].im, w.c[a].re);
      w.c[a].im = fma(U.e[b][a].re, x.c[b].im, w.c[a].im);
      w.c[a].im = fma(-U.e[b][a].im, x.c[b].re, w.c[a].im);
    }
  }
  return w;
}

// ---- df64 colour products with lazy accumulation. An output component of U x is a sum of six
// real products plus the accumulator. Each product a*b is formed exactly as p + e (e by FMA, the
// cross terms a.hi b.lo + a.lo b.hi folded into e); the six p's and the accumulator's hi part are
// added by two-sums in a fixed tree, every rounding error and e and the accumulator's lo part are
// collected in one float, and the result is renormalised once. The generic form renormalises after
// every multiply-add, a chain of six dependent 14-operation steps per component; here the products
// are independent and the chain is three two-sums deep. Error: a few units of 2^-48 of the largest
// term, as before.
__device__ __forceinline__ void df64_prod(df64 a, df64 b, float& p, float& e) {
  p = __fmul_rn(a.hi, b.hi);
  e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
}
// c + sum_k a_k b_k over six terms
__device__ __forceinline__ df64 df64_dot6_add(const df64 (&a)[6], const df64 (&b)[6], df64 c) {
  float p[6], e[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) df64_prod(a[k], b[k], p[k], e[k]);
  float s01, t01, s23, t23, s45, t45, s03, t03, s05, t05, s, t;
  two_sum(p[0], p[1], s01, t01);
  two_sum(p[2], p[3], s23, t23);
  two_sum(p[4], p[5], s45, t45);
  two_sum(s01, s23, s03, t03);
  two_sum(s03, s45, s05, t05);
  two_sum(c.hi, s05, s, t);
  const float err = __fadd_rn(
      __fadd_rn(__fadd_rn(__fadd_rn(e[0], e[1]), __fadd_rn(e[2], e[3])), __fadd_rn(__fadd_rn(e[4], e[5]), c.lo)),
      __fadd_rn(__fadd_rn(__fadd_rn(t01, t23), __fadd_rn(t45, t03)), __fadd_rn(t05, t)));
  df64 r;
  quick_two_sum(s, err, r.hi, r.lo);
  return r;
}

// acc += U x
__device__ __forceinline__ void mul_add(cvec3<df64>& acc, const su3<df64>& U, const cvec3<df64>& x) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const df64 ure[6] = {U.e[a][0].re, -U.e[a][0].im, U.e[a][1].re, -U.e[a][1].im, U.e[a][2].re, -U.e[a][2].im};
    const df64 xre[6] = {x.c[0].re, x.c[0].im, x.c[1].re, x.c[1].im, x.c[2].re, x.c[2].im};
    const df64 uim[6] = {U.e[a][0].re, U.e[a][0].im, U.e[a][1].re, U.e[a][1].im, U.e[a][2].re, U.e[a][2].im};
    const df64 xim[6] = {x.c[0].im, x.c[0].re, x.c[1].im, x.c[1].re, x.c[2].im, x.c[2].re};
    acc.c[a].re = df64_dot6_add(ure, xre, acc.c[a].re);
    acc.c[a].im = df64_dot6_add(uim, xim, acc.c[a].im);
  }
}

// acc -= U^dagger x: conj(U_ba) x_b = (U_re x_re + U_im x_im) + i (U_re x_im - U_im x_re)
__device__ __forceinline__ void adj_mul_sub(cvec3<df64>& acc, const su3<df64>& U, const cvec3<df64>& x) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const df64 ure[6] = {-U.e[0][a].re, -U.e[0][a].im, -U.e[1][a].re, -U.e[1][a].im, -U.e[2][a].re, -U.e[2][a].im};
    const df64 xre[6] = {x.c[0].re, x.c[0].im, x.c[1].re, x.c[1].im, x.c[2].re, x.c[2].im};
    const df64 uim[6] = {-U.e[0][a].re, U.e[0][a].im, -U.e[1][a].re, U.e[1][a].im, -U.e[2][a].re, U.e[2][a].im};
    const df64 xim[6] = {x.c[0].im, x.c[0].re, x.c[1].im, x.c[1].re, x.c[2].im, x.c[2].re};
    acc.c[a].re = df64_dot6_add(ure, xre, acc.c[a].re);
    acc.c[a].im = df64_dot6_add(uim, xim, acc.c[a].im);
  }
}

// w = U x
__device__ __forceinline__ cvec3<df64> mul(const su3<df64>& U, const cvec3<df64>& x) {
  cvec3<df64> w;
  zero(w);
  mul_add(w, U, x);
  return w;
}

// w = U^dagger x
__device__ __forceinline__ cvec3<df64> adj_mul(const su3<df64>& U, const cvec3<df64>& x) {
  cvec3<df64> w;
  zero(w);
  adj_mul_sub(w, U, x);
#pragma unroll
  for (int a = 0; a < 3; ++a) w.c[a] = {-w.c[a].re, -w.c[a].im};
  return w;
}

// acc += s * w
template <typename T>
__device__ __forceinline__ void axpy(cvec3<T>& acc, T s, const cvec3<T>& w) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc.c[a].re = fma(s, w.c[a].re, acc.c[a].re);
    acc.c[a].im = fma(s, w.c[a].im, acc.c[a].im);
  }
}

template <typename T>
__device__ __forceinline__ T norm2(const cvec3<T>& v) {
  T s = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) s = fma(v.c[a].re, v.c[a].re, fma(v.c[a].im, v.c[a].im, s));
  return s;
}

// Third row of an SU(3) matrix from the first two: c = conj(a x b).
template <typename T>
__device__ __forceinline__ void reconstruct_row2(su3<T>& U) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    // a_j b_k - a_k b_j
    T re = U.e[0][j].re * U.e[1][k].re - U.e[0][j].im * U.e[1][k].im;
    T im = U.e[0][j].re * U.e[1][k].im + U.e[0][j].im * U.e[1][k].re;
    re = fma(-U.e[0][k].re, U.e[1][j].re, re);
    re = fma(U.e[0][k].im, U.e[1][j].im, re);
    im = fma(-U.e[0][k].re, U.e[1][j].im, im);
    im = fma(-U.e[0][k].im, U.e[1][j].re, im);
    U.e[2][i].re = re;
    U.e[2][i].im = -im;
  }
}

// Two 16-bit fixed-point reals (q = round(v * 2^15) + 2^15, low and high half of w) to floats.
// The byte permutation places q under the exponent bits of 1.5 * 2^23, so that the float is exactly
// 12582912 + q; scaled by 2^-15 that is 384 + q / 2^15 (24 significant bits: exact), and 385
// subtracted gives (q - 2^15) / 2^15 = v. One permutation and one FMA per real, no conversion unit.
__device__ __forceinline__ float2 fx16x2_to_float2(unsigned w) {
  const float lo = __uint_as_float(__byte_perm(w, 0x4B40u, 0x5410));
  const float hi = __uint_as_float(__byte_perm(w, 0x4B40u, 0x5432));
  return make_float2(fmaf(lo, 0x1p-15f, -385.0f), fmaf(hi, 0x1p-15f, -385.0f));
}
__host__ __device__ __forceinline__ unsigned fx16_of(float v) {
  float t = rintf(v * 32768.0f);
  t = t < -32768.0f ? -32768.0f : (t > 32767.0f ? 32767.0f : t);
  return (unsigned)((int)t + 32768);
}
__host__ __device__ __forceinline__ unsigned float2_to_fx16x2(float re, float im) {
  return fx16_of(re) | (fx16_of(im) << 16);
}

__device__ __forceinline__ float2 u32_to_float2(unsigned u) {
  return __half22float2(__halves2half2(__ushort_as_half((unsigned short)(u & 0xffffu)),
                                       __ushort_as_half((unsigned short)(u >> 16))));
}
__device__ __forceinline__ unsigned float2_to_u32(float a, float b) {
  return (unsigned)__half_as_ushort(__float2half_rn(a)) | ((unsigned)__half_as_ushort(__float2half_rn(b)) << 16);
}

// ------------------------------------------------------------------------------------------
// Packed fields. One parity, V/2 sites, structure of arrays.
// ------------------------------------------------------------------------------------------
template <int PREC>
struct Field;

template <>
struct Field<QCD_PREC_DOUBLE> {
  using T = double;
  static constexpr int kElemsPerSite = 3;
  double2* p;  // [3][Vh]
  int Vh;
  __device__ __forceinline__ cvec3<double> load(int k) const {
    cvec3<double> v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double2 d = __ldg(p + (size_t)a * Vh + k);
      v.c[a].re = d.x; v.c[a].im = d.y;
    }
    return v;
  }
  __device__ __forceinline__ cvec3<double> load_cg(int k) const {
    cvec3<double> v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double2 d = __ldcg(p + (size_t)a * Vh + k);
      v.c[a].re = d.x; v.c[a].im = d.y;
    }
    return v;
  }
  __device__ __forceinline__ void store(int k, const cvec3<double>& v) const {
#pragma unroll
    for (int a = 0; a < 3; ++a) p[(size_t)a * Vh + k] = make_double2(v.c[a].re, v.c[a].im);
  }
  static size_t bytes(long long Vh) { return (size_t)Vh * 3 * sizeof(double2); }
};

template <>
struct Field<QCD_PREC_SINGLE> {
  using T = float;
  static constexpr int kElemsPerSite = 3;
  float2* p;  // [3][Vh]
  int Vh;
  __device__ __forceinline__ cvec3<float> load(int k) const {
    cvec3<float> v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 d = __ldg(p + (size_t)a * Vh + k);
      v.c[a].re = d.x; v.c[a].im = d.y;
    }
    return v;
  }
  __device__ __forceinline__ cvec3<float> load_cg(int k) const {
    cvec3<float> v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 d = __ldcg(p + (size_t)a * Vh + k);
      v.c[a].re = d.x; v.c[a].im = d.y;
    }
    return v;
  }
  __device__ __forceinline__ void store(int k, const cvec3<float>& v) const {
#pragma unroll
    for (int a = 0; a < 3; ++a) p[(size_t)a * Vh + k] = make_float2(v.c[a].re, v.c[a].im);
  }
  static size_t bytes(long long Vh) { return (size_t)Vh * 3 * sizeof(float2); }
};

// 16 bytes per site: three half2 colour components scaled by a per-site float.
template <>
struct Field<QCD_PREC_HALF> {
  using T = float;
  static constexpr int kElemsPerSite = 1;
  uint4* p;  // [Vh]
  int Vh;
  __device__ __forceinline__ cvec3<float> load(int k) const { return decode(__ldg(p + k)); }
  __device__ __forceinline__ cvec3<float> load_cg(int k) const { return decode(__ldcg(p + k)); }
  // The colour vector without its scale, and the scale: an operator that multiplies its hop
  // result by a coefficient anyway applies the scale there, once, instead of to six reals.
  __device__ __forceinline__ cvec3<float> load_raw(int k, float& s) const {
    const uint4 q = __ldg(p + k);
    s = __uint_as_float(q.w);
    cvec3<float> v;
    const unsigned w[3] = {q.x, q.y, q.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 f = u32_to_float2(w[a]);
      v.c[a].re = f.x; v.c[a].im = f.y;
    }
    return v;
  }
  __device__ __forceinline__ static cvec3<float> decode(uint4 q) {
    const float s = __uint_as_float(q.w);
    cvec3<float> v;
    const unsigned w[3] = {q.x, q.y, q.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 f = u32_to_float2(w[a]);
      v.c[a].re = f.x * s; v.c[a].im = f.y * s;
    }
    return v;
  }
  __device__ __forceinline__ void store(int k, const cvec3<float>& v) const {
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) m = fmaxf(m, fmaxf(fabsf(v.c[a].re), fabsf(v.c[a].im)));
    const float inv = m > 0.f ? 1.f / m : 0.f;
    unsigned w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) w[a] = float2_to_u32(v.c[a].re * inv, v.c[a].im * inv);
    p[k] = make_uint4(w[0], w[1], w[2], __float_as_uint(m));
  }
  static size_t bytes(long long Vh) { return (size_t)Vh * sizeof(uint4); }
};

// FP64-accuracy field as float-float pairs: float4 {re.hi, re.lo, im.hi, im.lo} per colour.
template <>
struct Field<QCD_PREC_DF64> {
  using T = df64;
  static constexpr int kElemsPerSite = 3;
  float4* p;  // [3][Vh]
  int Vh;
  __device__ __forceinline__ static cvec3<df64> decode3(float4 a, float4 b, float4 c) {
    cvec3<df64> v;
    v.c[0].re = df64(a.x, a.y); v.c[0].im = df64(a.z, a.w);
    v.c[1].re = df64(b.x, b.y); v.c[1].im = df64(b.z, b.w);
    v.c[2].re = df64(c.x, c.y); v.c[2].im = df64(c.z, c.w);
    return v;
  }
  __device__ __forceinline__ cvec3<df64> load(int k) const {
    return decode3(__ldg(p + k), __ldg(p + (size_t)Vh + k), __ldg(p + 2 * (size_t)Vh + k));
  }
  __device__ __forceinline__ cvec3<df64> load_cg(int k) const {
    return decode3(__ldcg(p + k), __ldcg(p + (size_t)Vh + k), __ldcg(p + 2 * (size_t)Vh + k));
  }
  __device__ __forceinline__ void store(int k, const cvec3<df64>& v) const {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      p[(size_t)a * Vh + k] = make_float4(v.c[a].re.hi, v.c[a].re.lo, v.c[a].im.hi, v.c[a].im.lo);
  }
  static size_t bytes(long long Vh) { return (size_t)Vh * 3 * sizeof(float4); }
};

inline size_t field_bytes(int prec, long long Vh) {
  switch (prec) {
    case QCD_PREC_DOUBLE: return Field<QCD_PREC_DOUBLE>::bytes(Vh);
    case QCD_PREC_SINGLE: return Field<QCD_PREC_SINGLE>::bytes(Vh);
    case QCD_PREC_HALF: return Field<QCD_PREC_HALF>::bytes(Vh);
    case QCD_PREC_DF64: return Field<QCD_PREC_DF64>::bytes(Vh);
  }
  return 0;
}

// Precision of the CG solution accumulator for an inner precision.
__host__ __device__ constexpr int x_prec(int prec) {
  return prec == QCD_PREC_DOUBLE ? QCD_PREC_DOUBLE : (prec == QCD_PREC_DF64 ? QCD_PREC_DF64 : QCD_PREC_SINGLE);
}

// A field whose loads go to L2 (coherent), for data that other blocks write during the same
// launch; the default loads use the read-only path, valid only for data fixed during a launch.
template <class FieldT>
struct Coherent {
  using T = typename FieldT::T;
  static constexpr int kElemsPerSite = FieldT::kElemsPerSite;
  FieldT f;
  __device__ __forceinline__ cvec3<T> load(int k) const { return f.load_cg(k); }
  __device__ __forceinline__ void store(int k, const cvec3<T>& v) const { f.store(k, v); }
};

// ------------------------------------------------------------------------------------------
// Link loads with an L2 eviction priority. A half-lattice operator reads every link exactly once per
// launch; when the links are larger than the L2 they evict the CG's vector fields (which every
// launch re-reads) before being evicted themselves. Loading them with an evict-first policy keeps
// the fields resident instead (measured on GB300, 32^4 FP32 recon-12 mixed CG: 329.6 -> 295 ms per
// solve; FP16 recon-12 318 -> 299 ms). Where the links fit in L2 they are reused from it by the next
// launch, and the normal policy is kept (evict-first measured 6 % slower at 16^4 FP64).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t l2_policy(int evict_first) {
  uint64_t first, normal;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(first));
  asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(normal));
  return evict_first ? first : normal;
}
__device__ __forceinline__ float4 ld_link(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float2 ld_link(const float2* p, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_link(const double2* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint4 ld_link(const uint4* p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint2 ld_link(const uint2* p, uint64_t pol) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
  return v;
}

// ------------------------------------------------------------------------------------------
// Packed links. Array of (parity, mu) blocks of V/2 sites each; link (par, mu, k) is U_mu at
// even-odd site k of parity par. Recon 18 stores 1/2*eta*zeta*U; recon 12 stores rows 0, 1 of U.
// ------------------------------------------------------------------------------------------
template <int PREC, int RECON>
struct Links;

template <>
struct Links<QCD_PREC_DOUBLE, 18> {
  using T = double;
  static constexpr bool kFolded = true;
  const double2* p;  // [2][4][9][Vh]
  int Vh;
  int stream = 0;  // 1: load with the L2 evict-first policy
  __device__ __forceinline__ su3<double> load(int par, int mu, int k) const {
    su3<double> U;
    const uint64_t pol = l2_policy(stream);
    const double2* b = p + (size_t)(par * 4 + mu) * 9 * Vh + k;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      double2 d = ld_link(b + (size_t)e * Vh, pol);
      U.e[e / 3][e % 3].re = d.x; U.e[e / 3][e % 3].im = d.y;
    }
    return U;
  }
  static size_t bytes(long long Vh) { return (size_t)2 * 4 * 9 * Vh * sizeof(double2); }
};

template <>
struct Links<QCD_PREC_SINGLE, 18> {
  using T = float;
  static constexpr bool kFolded = true;
  const float2* p;  // [2][4][9][Vh]
  int Vh;
  int stream = 0;  // 1: load with the L2 evict-first policy
  __device__ __forceinline__ su3<float> load(int par, int mu, int k) const {
    su3<float> U;
    const uint64_t pol = l2_policy(stream);
    const float2* b = p + (size_t)(par * 4 + mu) * 9 * Vh + k;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      float2 d = ld_link(b + (size_t)e * Vh, pol);
      U.e[e / 3][e % 3].re = d.x; U.e[e / 3][e % 3].im = d.y;
    }
    return U;
  }
  static size_t bytes(long long Vh) { return (size_t)2 * 4 * 9 * Vh * sizeof(float2); }
};

template <>
struct Links<QCD_PREC_SINGLE, 12> {
  using T = float;
  static constexpr bool kFolded = false;
  const float4* p;  // [2][4][3][Vh]: (a0 a1) (a2 b0) (b1 b2)
  int Vh;
  int stream = 0;  // 1: load with the L2 evict-first policy
  __device__ __forceinline__ su3<float> load(int par, int mu, int k) const {
    su3<float> U;
    const float4* b = p + (size_t)(par * 4 + mu) * 3 * Vh + k;
    const uint64_t pol = l2_policy(stream);
    float4 q0 = ld_link(b, pol), q1 = ld_link(b + Vh, pol), q2 = ld_link(b + 2 * (size_t)Vh, pol);
    U.e[0][0] = {q0.x, q0.y}; U.e[0][1] = {q0.z, q0.w};
    U.e[0][2] = {q1.x, q1.y}; U.e[1][0] = {q1.z, q1.w};
    U.e[1][1] = {q2.x, q2.y}; U.e[1][2] = {q2.z, q2.w};
    reconstruct_row2(U);
    return U;
  }
  static size_t bytes(long long Vh) { return (size_t)2 * 4 * 3 * Vh * sizeof(float4); }
};

template <>
struct Links<QCD_PREC_HALF, 12> {
  using T = float;
  static constexpr bool kFolded = false;
  // 16-bit fixed point: every real of rows 0 and 1 as q = round(v * 2^15) + 2^15 in [0, 65535]
  // (|v| <= 1 for an SU(3) element; v = 1 saturates at 65535), (re, im) in the low and high half
  // of a 32-bit word. Absolute error <= 2^-16 (2^-15 next to v = 1), 8 to 16 times below IEEE
  // FP16's on elements of magnitude 0.25 to 1: the CG's iteration count grows with the operator's
  // rounding error.
  const uint4* p;  // [2][4][Vh] words of (a0 a1 a2 b0), then uint2 [2][4][Vh] words of (b1 b2)
  const uint2* q;
  int Vh;
  int stream = 0;  // 1: load with the L2 evict-first policy
  __device__ __forceinline__ su3<float> load(int par, int mu, int k) const {
    su3<float> U;
    const size_t o = (size_t)(par * 4 + mu) * Vh + k;
    const uint64_t pol = l2_policy(stream);
    uint4 a = ld_link(p + o, pol);
    uint2 b = ld_link(q + o, pol);
    const unsigned w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const float2 f = fx16x2_to_float2(w[e]);
      U.e[e / 3][e % 3].re = f.x; U.e[e / 3][e % 3].im = f.y;
    }
    reconstruct_row2(U);
    return U;
  }
  static size_t bytes(long long Vh) { return (size_t)2 * 4 * Vh * (sizeof(uint4) + sizeof(uint2)); }
};

template <>
struct Links<QCD_PREC_DF64, 18> {
  using T = df64;
  static constexpr bool kFolded = true;
  const float4* p;  // [2][4][9][Vh] of {re.hi, re.lo, im.hi, im.lo}
  int Vh;
  int stream = 0;  // 1: load with the L2 evict-first policy
  __device__ __forceinline__ su3<df64> load(int par, int mu, int k) const {
    su3<df64> U;
    const uint64_t pol = l2_policy(stream);
    const float4* b = p + (size_t)(par * 4 + mu) * 9 * Vh + k;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float4 d = ld_link(b + (size_t)e * Vh, pol);
      U.e[e / 3][e % 3].re = df64(d.x, d.y);
      U.e[e / 3][e % 3].im = df64(d.z, d.w);
    }
    return U;
  }
  static size_t bytes(long long Vh) { return (size_t)2 * 4 * 9 * Vh * sizeof(float4); }
};

inline size_t links_bytes(int prec, int recon, long long Vh) {
  if (prec == QCD_PREC_DOUBLE && recon == 18) return Links<QCD_PREC_DOUBLE, 18>::bytes(Vh);
  if (prec == QCD_PREC_SINGLE && recon == 18) return Links<QCD_PREC_SINGLE, 18>::bytes(Vh);
  if (prec == QCD_PREC_SINGLE && recon == 12) return Links<QCD_PREC_SINGLE, 12>::bytes(Vh);
  if (prec == QCD_PREC_HALF && recon == 12) return Links<QCD_PREC_HALF, 12>::bytes(Vh);
  if (prec == QCD_PREC_DF64 && recon == 18) return Links<QCD_PREC_DF64, 18>::bytes(Vh);
  return 0;
}

// Whether single-RHS operator launches should stream the links of (prec, recon) with the L2
// evict-first policy: when they take more than half of the L2.
inline int stream_links(int prec, int recon, long long Vh) {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0)
    return 0;
  return links_bytes(prec, recon, Vh) > (size_t)l2 / 2 ? 1 : 0;
}

// Per-thread partial sums of the norms: FP32 in FP32-arithmetic kernels (a thread adds a few
// sites' values; converted to FP64 once, at the block sum), FP64 otherwise. Keeps the FP64
// pipe, 1/64 of the FP32 rate on GB300, out of the per-site work.
template <class T>
struct Accum {
  using type = double;
};
template <>
struct Accum<float> {
  using type = float;
};
__device__ __forceinline__ void accum(float& r, float v) { r += v; }
__device__ __forceinline__ void accum(double& r, double v) { r += v; }
__device__ __forceinline__ void accum(double& r, float v) { r += (double)v; }
__device__ __forceinline__ void accum(double& r, df64 v) { r += (double)v; }

// ------------------------------------------------------------------------------------------
// Deterministic reductions: per-block partial sums in FP64, the last block to finish sums the
// partials in a fixed order (so results do not depend on block scheduling).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV values over the block; thread 0 returns the totals in v.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sm[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) sm[j][warp] = v[j];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double t = lane < nw ? sm[j][lane] : 0.0;
      v[j] = warp_sum(t);
    }
  }
  __syncthreads();
}

// The same sums for FP32 per-thread values, carried as float pairs hi + lo (Knuth's two-sum on the
// FP32 pipes, ~48 significant bits) and returned as FP64. GB300's FP64 pipe runs at 1/64 of the FP32
// rate: the FP64 shuffle tree (5 adds per warp and value) of every block of a one-wave launch kept
// that pipe busy ~6k cycles per SM at the end of each FP32 or FP16 CG operator launch (ncu: FP64
// pipe 15 % active in a kernel with no other FP64 arithmetic).
__device__ __forceinline__ df64 warp_sum_pair(df64 t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    t = t + df64(__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o));
  return t;
}
__device__ __forceinline__ double warp_sum(float v) {
  const df64 t = warp_sum_pair(df64(v, 0.f));
  return (double)t.hi + (double)t.lo;
}
template <int NV>
__device__ __forceinline__ void block_sum(const float (&x)[NV], double (&v)[NV]) {
  __shared__ float2 sm[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  df64 t[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) t[j] = warp_sum_pair(df64(x[j], 0.f));
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) sm[j][warp] = make_float2(t[j].hi, t[j].lo);
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const float2 q = lane < nw ? sm[j][lane] : make_float2(0.f, 0.f);
      const df64 u = warp_sum_pair(df64(q.x, q.y));
      v[j] = (double)u.hi + (double)u.lo;
    }
  }
  __syncthreads();
}
template <int NV>
__device__ __forceinline__ void block_sum(const double (&x)[NV], double (&v)[NV]) {
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = x[j];
  block_sum<NV>(v);
}

// Sum of partials[j * kMaxPartials + b] over b < n, for j < NV, by the whole block (thread 0 gets
// the totals). The order is fixed by n and blockDim.x alone: thread t adds the blocks t + q*B in four
// chains (q mod 4), the chains in pairs, then the block. The four chains keep a thread's loads in
// flight together: one L2 round trip per four partials instead of one per partial, which is what the
// whole grid waits for at the end of every reducing launch (measured on GB300: the summing block's
// SM stayed busy ~19k cycles longer than the others with one chain and two sums in a row).
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, int n, double (&s)[NV]) {
  const int B = blockDim.x;
  double a[NV][4];
#pragma unroll
  for (int j = 0; j < NV; ++j) a[j][0] = a[j][1] = a[j][2] = a[j][3] = 0.0;
  int b = threadIdx.x;
  for (; b + 3 * B < n; b += 4 * B) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const double* p = partials + (size_t)j * kMaxPartials + b;
      const double v0 = __ldcg(p), v1 = __ldcg(p + B), v2 = __ldcg(p + 2 * B), v3 = __ldcg(p + 3 * B);
      a[j][0] += v0; a[j][1] += v1; a[j][2] += v2; a[j][3] += v3;
    }
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) {  // at most three left
    const double* p = partials + (size_t)j * kMaxPartials + b;
    const double v0 = b < n ? __ldcg(p) : 0.0, v1 = b + B < n ? __ldcg(p + B) : 0.0,
                 v2 = b + 2 * B < n ? __ldcg(p + 2 * B) : 0.0;
    a[j][0] += v0; a[j][1] += v1; a[j][2] += v2;
    s[j] = (a[j][0] + a[j][1]) + (a[j][2] + a[j][3]);
  }
  block_sum<NV>(s);
}

// Write this block's partials; returns true in the block that finished last, after which
// `tot` holds the grid-wide sums (valid in every thread of that block).
// A is float (the FP32-arithmetic kernels' per-thread sums, reduced as float pairs) or double.
template <int NV, class A>
__device__ __forceinline__ bool grid_sum_last_block(const A (&x)[NV], double* partials, unsigned* counter,
                                                    double (&tot)[NV]) {
  __shared__ bool am_last;
  __shared__ double res[NV];
  double v[NV];
  block_sum<NV>(x, v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) partials[(size_t)j * kMaxPartials + blockIdx.x] = v[j];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double s[NV];
  sum_partials<NV>(partials, (int)gridDim.x, s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) res[j] = s[j];
    *counter = 0u;  // ready for the next launch
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = res[j];
  return true;
}

// ------------------------------------------------------------------------------------------
// Error plumbing (host).
// ------------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define QCD_CUDA(call)                                         \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::qcd::cuda_fail(e_, #call); \
  } while (0)

inline int grid_for(long long n, int block = kBlock) { return (int)((n + block - 1) / block); }

}  // namespace qcd
