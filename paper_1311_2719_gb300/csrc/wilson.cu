// Wilson fermions (the paper's second program, §2/§6): the hopping term D_W on the full lattice,
// M = 1 - kappa D_W, M^dagger = gamma5 M gamma5, and CGNR (CG on M^dagger M x = M^dagger b) with
// FP64 (or df64) reliable updates when the recursion runs in FP32.
//
// Spin projection: (1 -+ gamma_mu)/2 are rank-2 projectors. In the DeGrand-Rossi basis every
// gamma_mu has one non-zero entry per row, ph(r) in {+-1, +-i} at column col(r), with col(r) in
// {2, 3} for r in {0, 1}. So (1 + s gamma_mu) psi is fixed by its upper two rows
// h_r = psi_r + s ph(r) psi_col(r) (r = 0, 1), and its lower rows are s ph(r) h_col(r) (gamma^2 = 1).
// A hop therefore multiplies two colour vectors by the link instead of four.
#include <chrono>
#include <cmath>
#include <vector>

#include "cg_common.cuh"

namespace qcd {

// ---------------------------------------------------------------- gamma tables (DeGrand-Rossi)
// column and phase of the non-zero entry of row r of gamma_mu; phase code: 0 -> 1, 1 -> i,
// 2 -> -1, 3 -> -i
__host__ __device__ constexpr int gcol(int mu, int r) {
  constexpr int c[4][4] = {{3, 2, 1, 0}, {3, 2, 1, 0}, {2, 3, 0, 1}, {2, 3, 0, 1}};
  return c[mu][r];
}
__host__ __device__ constexpr int gph(int mu, int r) {
  constexpr int p[4][4] = {{1, 1, 3, 3}, {2, 0, 0, 2}, {1, 3, 3, 1}, {0, 0, 0, 0}};
  return p[mu][r];
}

// v * (i^code)
template <typename T>
__device__ __forceinline__ cplx<T> times_phase(const cplx<T>& v, int code) {
  switch (code & 3) {
    case 0: return v;
    case 1: return {-v.im, v.re};
    case 2: return {-v.re, -v.im};
    default: return {v.im, -v.re};
  }
}

template <typename T>
struct spinor {
  cvec3<T> s[4];
};

template <typename T>
__device__ __forceinline__ void zero(spinor<T>& v) {
#pragma unroll
  for (int r = 0; r < 4; ++r) zero(v.s[r]);
}

template <typename T>
__device__ __forceinline__ T norm2(const spinor<T>& v) {
  T t = T(0);
#pragma unroll
  for (int r = 0; r < 4; ++r) t = t + norm2(v.s[r]);
  return t;
}

// ---------------------------------------------------------------- fields (full lattice, V sites)
template <int PREC>
struct WField;

template <>
struct WField<QCD_PREC_DOUBLE> {
  using T = double;
  double2* p;  // [12][V]: component (spin, colour) = 3 s + c
  int V;
  __device__ __forceinline__ spinor<double> load(int i) const {
    spinor<double> v;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const double2 d = __ldg(p + (size_t)q * V + i);
      v.s[q / 3].c[q % 3] = {d.x, d.y};
    }
    return v;
  }
  __device__ __forceinline__ void store(int i, const spinor<double>& v) const {
#pragma unroll
    for (int q = 0; q < 12; ++q) p[(size_t)q * V + i] = make_double2(v.s[q / 3].c[q % 3].re, v.s[q / 3].c[q % 3].im);
  }
  static size_t bytes(long long V) { return (size_t)V * 12 * sizeof(double2); }
  __host__ __device__ WField at(int r) const { return {p + (size_t)r * 12 * V, V}; }  // RHS r of a multi-RHS field
};

template <>
struct WField<QCD_PREC_SINGLE> {
  using T = float;
  float4* p;  // [6][V]: float4 q holds components 2q and 2q+1
  int V;
  __device__ __forceinline__ spinor<float> load(int i) const {
    spinor<float> v;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float4 d = __ldg(p + (size_t)q * V + i);
      v.s[(2 * q) / 3].c[(2 * q) % 3] = {d.x, d.y};
      v.s[(2 * q + 1) / 3].c[(2 * q + 1) % 3] = {d.z, d.w};
    }
    return v;
  }
  __device__ __forceinline__ void store(int i, const spinor<float>& v) const {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const cplx<float> a = v.s[(2 * q) / 3].c[(2 * q) % 3], b = v.s[(2 * q + 1) / 3].c[(2 * q + 1) % 3];
      p[(size_t)q * V + i] = make_float4(a.re, a.im, b.re, b.im);
    }
  }
  static size_t bytes(long long V) { return (size_t)V * 6 * sizeof(float4); }
  __host__ __device__ WField at(int r) const { return {p + (size_t)r * 6 * V, V}; }
};

// df64: float4 [12][V] {re.hi, re.lo, im.hi, im.lo}, the 16 bytes per complex of FP64. The
// mixed CGNR can keep its solution accumulator, b, M^dagger b and the reliable-update residual in
// this form: the operator on them then runs on the FP32 pipes instead of the FP64 pipe.
template <>
struct WField<QCD_PREC_DF64> {
  using T = df64;
  float4* p;
  int V;
  __device__ __forceinline__ spinor<df64> load(int i) const {
    spinor<df64> v;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const float4 d = __ldg(p + (size_t)q * V + i);
      v.s[q / 3].c[q % 3] = {df64(d.x, d.y), df64(d.z, d.w)};
    }
    return v;
  }
  __device__ __forceinline__ void store(int i, const spinor<df64>& v) const {
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const cplx<df64> c = v.s[q / 3].c[q % 3];
      p[(size_t)q * V + i] = make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo);
    }
  }
  static size_t bytes(long long V) { return (size_t)V * 12 * sizeof(float4); }
  __host__ __device__ WField at(int r) const { return {p + (size_t)r * 12 * V, V}; }
};

// links [mu][9][V], zeta folded into the t-links of the last time slice (no staggered phases)
template <int PREC>
struct WLinks;
template <>
struct WLinks<QCD_PREC_DOUBLE> {
  using T = double;
  const double2* p;
  int V;
  __device__ __forceinline__ su3<double> load(int mu, int i) const {
    su3<double> U;
    const double2* b = p + (size_t)mu * 9 * V + i;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const double2 d = __ldg(b + (size_t)e * V);
      U.e[e / 3][e % 3] = {d.x, d.y};
    }
    return U;
  }
  static size_t bytes(long long V) { return (size_t)4 * 9 * V * sizeof(double2); }
};
template <>
struct WLinks<QCD_PREC_SINGLE> {
  using T = float;
  const float2* p;
  int V;
  __device__ __forceinline__ su3<float> load(int mu, int i) const {
    su3<float> U;
    const float2* b = p + (size_t)mu * 9 * V + i;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float2 d = __ldg(b + (size_t)e * V);
      U.e[e / 3][e % 3] = {d.x, d.y};
    }
    return U;
  }
  static size_t bytes(long long V) { return (size_t)4 * 9 * V * sizeof(float2); }
};

template <>
struct WLinks<QCD_PREC_DF64> {
  using T = df64;
  const float4* p;  // [mu][9][V] {re.hi, re.lo, im.hi, im.lo}
  int V;
  __device__ __forceinline__ su3<df64> load(int mu, int i) const {
    su3<df64> U;
    const float4* b = p + (size_t)mu * 9 * V + i;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float4 d = __ldg(b + (size_t)e * V);
      U.e[e / 3][e % 3] = {df64(d.x, d.y), df64(d.z, d.w)};
    }
    return U;
  }
  static size_t bytes(long long V) { return (size_t)4 * 9 * V * sizeof(float4); }
};

size_t wfield_bytes(int prec, long long V) {
  switch (prec) {
    case QCD_PREC_DOUBLE: return WField<QCD_PREC_DOUBLE>::bytes(V);
    case QCD_PREC_SINGLE: return WField<QCD_PREC_SINGLE>::bytes(V);
    case QCD_PREC_DF64: return WField<QCD_PREC_DF64>::bytes(V);
    default: return 0;
  }
}
size_t wlinks_bytes(int prec, long long V) {
  switch (prec) {
    case QCD_PREC_DOUBLE: return WLinks<QCD_PREC_DOUBLE>::bytes(V);
    case QCD_PREC_SINGLE: return WLinks<QCD_PREC_SINGLE>::bytes(V);
    case QCD_PREC_DF64: return WLinks<QCD_PREC_DF64>::bytes(V);
    default: return 0;
  }
}

// ---------------------------------------------------------------- geometry (full lattice)
__device__ __forceinline__ void full_site(const Geom& g, int i, int c[4]) {
  int t = i;
  const int t0 = fdiv(t, g.d0);
  c[0] = t - t0 * g.L0;
  const int t1 = fdiv(t0, g.d1);
  c[1] = t0 - t1 * g.L1;
  c[3] = fdiv(t1, g.d2);
  c[2] = t1 - c[3] * g.L2;
}

// ---------------------------------------------------------------- the hopping term at site i
// neighbour of site i (coordinates c) in direction mu: dir 0 forward, dir 1 backward (periodic wrap)
__device__ __forceinline__ int w_neighbour(const Geom& g, int i, const int c[4], int mu, int dir) {
  const int L[4] = {g.L0, g.L1, g.L2, g.L3};
  const int st[4] = {1, g.L0, g.L0 * g.L1, g.L0 * g.L1 * g.L2};
  return dir == 0 ? (c[mu] == L[mu] - 1 ? i - (L[mu] - 1) * st[mu] : i + st[mu])
                  : (c[mu] == 0 ? i + (L[mu] - 1) * st[mu] : i - st[mu]);
}

// One hop into acc: forward (dir 0) adds (1 - gamma_mu) U psi, backward (dir 1) adds
// (1 + gamma_mu) U^dagger psi, through the two-row spin projection. G5IN: psi is read as gamma5 psi
// (spins 2, 3 negated) — used for M^dagger.
template <bool G5IN, typename T>
__device__ __forceinline__ void hop_accumulate(spinor<T>& acc, const su3<T>& Ul, spinor<T> psi, int mu, int dir) {
  const int sgn = dir == 0 ? 2 : 0;  // phase code of s: -1 -> 2, +1 -> 0
  if constexpr (G5IN) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      psi.s[2].c[a] = {-psi.s[2].c[a].re, -psi.s[2].c[a].im};
      psi.s[3].c[a] = {-psi.s[3].c[a].re, -psi.s[3].c[a].im};
    }
  }
  cvec3<T> h[2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cplx<T> t = times_phase(psi.s[gcol(mu, r)].c[a], sgn + gph(mu, r));
      h[r].c[a] = {psi.s[r].c[a].re + t.re, psi.s[r].c[a].im + t.im};
    }
  cvec3<T> w[2];
  w[0] = dir == 0 ? mul(Ul, h[0]) : adj_mul(Ul, h[0]);
  w[1] = dir == 0 ? mul(Ul, h[1]) : adj_mul(Ul, h[1]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc.s[0].c[a].re += w[0].c[a].re; acc.s[0].c[a].im += w[0].c[a].im;
    acc.s[1].c[a].re += w[1].c[a].re; acc.s[1].c[a].im += w[1].c[a].im;
#pragma unroll
    for (int r = 2; r < 4; ++r) {
      const cplx<T> t = times_phase(w[gcol(mu, r)].c[a], sgn + gph(mu, r));
      acc.s[r].c[a].re += t.re;
      acc.s[r].c[a].im += t.im;
    }
  }
}

template <class LinksT, class FieldT, bool G5IN>
__device__ __forceinline__ spinor<typename LinksT::T> wilson_hop(const Geom& g, const LinksT& U, const FieldT& in, int i) {
  using T = typename LinksT::T;
  int c[4];
  full_site(g, i, c);
  spinor<T> acc;
  zero(acc);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const int nb = w_neighbour(g, i, c, mu, dir);
      hop_accumulate<G5IN>(acc, U.load(mu, dir == 0 ? i : nb), in.load(nb), mu, dir);
    }
  return acc;
}

// resident 128-thread blocks per SM: 4 (a cap of 128 registers). In FP64 that keeps 16 warps on
// the FP64 pipe; in FP32 the compiler spends the registers above its own choice (80) on loads in
// flight, which the latency-bound kernel needs more than a fifth and sixth block.
template <typename T>
struct WMinBlocks { static constexpr int value = 4; };
// df64: a spinor accumulator of 48 FP32 pairs does not fit 128 registers without spills; 3 blocks
// (168 registers) keep 12 warps per SM on the FP32 pipes.
template <>
struct WMinBlocks<df64> { static constexpr int value = 3; };

template <class LinksT, class FieldT, bool G5IN, class Epi>
__global__ void __launch_bounds__(kBlock, WMinBlocks<typename LinksT::T>::value) wilson_kernel(Geom g, int V, LinksT U, FieldT in, Epi epi) {
  if (epi.skip()) return;
  using A = typename Accum<typename LinksT::T>::type;
  A red[Epi::NV > 0 ? Epi::NV : 1];
#pragma unroll
  for (int j = 0; j < (Epi::NV > 0 ? Epi::NV : 1); ++j) red[j] = A(0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    auto acc = wilson_hop<LinksT, FieldT, G5IN>(g, U, in, i);
    epi.site(i, acc, red);
  }
  if constexpr (Epi::NV > 0) epi.finish(red);
}

// ---------------------------------------------------------------- epilogues
template <class FieldT>
struct WStore {  // out = D_W in
  static constexpr int NV = 0;
  FieldT out;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class T, class A>
  __device__ __forceinline__ void site(int i, spinor<T>& acc, A*) const { out.store(i, acc); }
  template <class A>
  __device__ __forceinline__ void finish(A*) const {}
};

// out = in - kappa acc            (M in, when the kernel computes acc = D_W in)
// out = in - kappa gamma5 acc     (M^dagger in, when acc = D_W gamma5 in: G5IN)
template <class FieldT, bool DAG>
__device__ __forceinline__ spinor<typename FieldT::T> m_combine(const FieldT& in, int i, const spinor<typename FieldT::T>& acc,
                                                                typename FieldT::T kappa) {
  using T = typename FieldT::T;
  spinor<T> v = in.load(i);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const T k = (DAG && r >= 2) ? -kappa : kappa;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v.s[r].c[a].re = fma(-k, acc.s[r].c[a].re, v.s[r].c[a].re);
      v.s[r].c[a].im = fma(-k, acc.s[r].c[a].im, v.s[r].c[a].im);
    }
  }
  return v;
}

template <class FieldT, bool DAG>
struct WApplyM {  // out = M in or M^dagger in
  static constexpr int NV = 0;
  FieldT in, out;
  double kappa;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class T, class A>
  __device__ __forceinline__ void site(int i, spinor<T>& acc, A*) const {
    out.store(i, m_combine<FieldT, DAG>(in, i, acc, (T)kappa));
  }
  template <class A>
  __device__ __forceinline__ void finish(A*) const {}
};

// resident 128-thread blocks per SM for a register block of RB right-hand sides (register caps
// 128 for RB <= 2 and 170 for RB = 4 in FP32; 170 / 255 in FP64)
template <typename T, int RB>
struct WMrhsMinBlocks {
  static constexpr int value = sizeof(T) == 8 ? (RB == 1 ? 3 : 2) : (RB <= 2 ? 4 : 3);
};

// ---------------------------------------------------------------- multi-RHS operator kernel
// One thread per site (1-D grid, one wave). For its site a thread walks the right-hand sides in
// register blocks of RB: each loaded link is applied to the RB spinors of a block, and the next
// block reloads the same links (fields of all RHS back to back, WField::at). The epilogue sees one
// (site, RHS) pair at a time; reducing epilogues keep per-thread, per-RHS partials in shared memory
// and finish with one deterministic sum per RHS.
// (Measured on 32^3x64 with 8 RHS, FP32: this layout with RB = 1 beats one grid row per register
// block, whose rows each stream the links from DRAM, and one lane per register block, which spreads
// a warp's neighbour gathers over the fields and thrashes L2.)
template <class LinksT, class FieldT, bool G5IN, int RB, class Epi>
__global__ void __launch_bounds__(kBlock, WMrhsMinBlocks<typename LinksT::T, RB>::value) wilson_mrhs_kernel(Geom g, int V, LinksT U, FieldT in, int nrhs, Epi epi) {
  using T = typename LinksT::T;
  using A = typename Accum<T>::type;
  __shared__ A spart[Epi::kReduce ? kMaxRhs : 1][kBlock];
  unsigned run = 0;
  for (int q = 0; q < nrhs; ++q)
    if (epi.running(q)) run |= 1u << q;
  if constexpr (Epi::kReduce)
    for (int q = 0; q < nrhs; ++q) spart[q][threadIdx.x] = A(0);
  if (run) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
      int c[4];
      full_site(g, i, c);
#pragma unroll 1
      for (int r0 = 0; r0 < nrhs; r0 += RB) {
        const unsigned active = (run >> r0) & ((1u << RB) - 1u);
        if (!active) continue;
        // an opaque copy of the links pointer keeps the link loads inside this loop (hoisting all
        // eight links out of it would hold 144 registers)
        LinksT Ur = U;
        asm volatile("" : "+l"(Ur.p));
        spinor<T> acc[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) zero(acc[j]);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
#pragma unroll
          for (int dir = 0; dir < 2; ++dir) {
            const int nb = w_neighbour(g, i, c, mu, dir);
            const su3<T> Ul = Ur.load(mu, dir == 0 ? i : nb);
#pragma unroll
            for (int j = 0; j < RB; ++j)
              if ((active >> j) & 1u) hop_accumulate<G5IN>(acc[j], Ul, in.at(r0 + j).load(nb), mu, dir);
          }
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if ((active >> j) & 1u) {
            A part = A(0);
            epi.site(i, r0 + j, acc[j], part);
            if constexpr (Epi::kReduce) spart[r0 + j][threadIdx.x] += part;
          }
      }
    }
  }
  if constexpr (Epi::kReduce) {
    __shared__ bool am_last;
    for (int q = 0; q < nrhs; ++q) {
      const A x[1] = {spart[q][threadIdx.x]};
      double v[1];
      block_sum<1>(x, v);
      if (threadIdx.x == 0) epi.partials[(size_t)q * kMaxPartials + blockIdx.x] = v[0];
    }
    if (threadIdx.x == 0) {
      __threadfence();
      am_last = atomicAdd(epi.counter(), 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (am_last) {
      __shared__ double tot[kMaxRhs];
      mrhs_totals(nrhs, epi.partials, tot);
      // one thread per right-hand side (each update is a chain of dependent global loads and stores)
      if (threadIdx.x < nrhs && epi.running(threadIdx.x)) epi.update(threadIdx.x, tot[threadIdx.x]);
      if (threadIdx.x == 0) *epi.counter() = 0u;
    }
  }
}

// ---------------------------------------------------------------- multi-RHS operator with shared links
// A block of kShWarps warps takes a tile of kShTile consecutive sites. Warp w loads link slot w of the
// tile (direction w / 2: the forward link U_mu(i) or the backward link U_mu(i - mu)) once, one lane
// per site, into shared memory; after a barrier warp w applies the tile's eight links to right-hand
// sides w and w + kShWarps (through the two-row spin projection, the link read back from shared
// memory for each RHS). Every link is read from memory once per launch; dslash-style register
// blocking instead reloads the links for every block of RHS (measured at 32^3 x 64 x 8 RHS: K1 moved
// 1.6 times its algorithmic bytes).
template <typename T>
struct WShMinBlocks {  // 256-thread blocks per SM: 2 (128 registers) for FP32, 1 for 64-bit types
  static constexpr int value = sizeof(T) == 4 ? 2 : 1;
};

// The order in which the tiles visit the sites: rows of L0 sites taken in (x1, x2 within a chunk of
// zc, x3, chunk) order instead of lexicographically. A site's x3 (t) neighbours then come
// L0 L1 zc sites later in the sweep instead of a whole L0 L1 L2 time slice later, and are still in
// L2 when they are needed; only the x2 hops that cross a chunk boundary (1/zc of them) reach back
// further. Memory layout and coalescing are unchanged (a tile is 32 consecutive sites of a row
// when L0 >= 32). Returns the site and its coordinates for sweep index j.
__device__ __forceinline__ int w_sweep_site(const Geom& g, int zc, int j, int c[4]) {
  int r = fdiv(j, g.d0);
  c[0] = j - r * g.L0;
  const int r1 = fdiv(r, g.d1);
  c[1] = r - r1 * g.L1;
  const int zz = r1 & (zc - 1);  // zc is a power of two
  r = r1 >> (__ffs(zc) - 1);
  const int r3 = fdiv(r, g.d3);
  c[3] = r - r3 * g.L3;
  c[2] = r3 * zc + zz;
  return c[0] + g.L0 * (c[1] + g.L1 * (c[2] + g.L2 * c[3]));
}

// The x2 chunk of the sweep (a power of two): the largest of 16, 8, 4, 2 dividing L2 whose L0 L1 zc sites stay
// within 4096, else 1 (lexicographic). Measured on GB300, 32^3x64 x 8 RHS (FP32 CGNR, df64 reliable
// updates), per solve: lexicographic 374 ms, zc = 16 (16384 sites) 366 ms, 8: 357 ms, 4: 354 ms; a
// site's input is used over twice the chunk distance in the sweep, and ~8 MB of fields and links
// per 4096 sites have to stay in L2 meanwhile.
inline int w_sweep_chunk(const Geom& g) {
  for (int zc : {16, 8, 4, 2})
    if (g.L2 % zc == 0 && (long long)g.L0 * g.L1 * zc <= 4096) return zc;
  return 1;
}

template <class LinksT, class FieldT, bool G5IN, class Epi>
__global__ void __launch_bounds__(kShThreads, WShMinBlocks<typename LinksT::T>::value)
    wilson_mrhs_shared_kernel(Geom g, int V, LinksT U, FieldT in, int nrhs, Epi epi, int zc) {
  using T = typename LinksT::T;
  using A = typename Accum<T>::type;
  __shared__ __align__(16) unsigned char sl_raw[kShWarps * 9 * kShTile * sizeof(cplx<T>)];
  cplx<T>* sl = reinterpret_cast<cplx<T>*>(sl_raw);  // [slot][element][site of the tile]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned run = 0;
  for (int q = 0; q < nrhs; ++q)
    if (epi.running(q)) run |= 1u << q;
  if (!run) return;  // every block reads the same flags: none of them arrives below
  A part[2] = {A(0), A(0)};
  const int ntiles = (V + kShTile - 1) / kShTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * kShTile + lane;
    const bool valid = j < V;
    int c[4] = {0, 0, 0, 0};
    const int i = valid ? w_sweep_site(g, zc, j, c) : 0;
    if (valid) {
      const int mu = w >> 1, dir = w & 1;
      const su3<T> L = U.load(mu, dir == 0 ? i : w_neighbour(g, i, c, mu, 1));
#pragma unroll
      for (int e = 0; e < 9; ++e) sl[(w * 9 + e) * kShTile + lane] = L.e[e / 3][e % 3];
    }
    __syncthreads();
    if (valid) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int q = w + j * kShWarps;
        if (q >= nrhs || !((run >> q) & 1u)) continue;
        spinor<T> acc;
        zero(acc);
#pragma unroll
        for (int slot = 0; slot < kShWarps; ++slot) {
          const int mu = slot >> 1, dir = slot & 1;
          su3<T> Ul;
#pragma unroll
          for (int e = 0; e < 9; ++e) Ul.e[e / 3][e % 3] = sl[(slot * 9 + e) * kShTile + lane];
          hop_accumulate<G5IN>(acc, Ul, in.at(q).load(w_neighbour(g, i, c, mu, dir)), mu, dir);
        }
        A pt = A(0);
        epi.site(i, q, acc, pt);
        part[j] += pt;
      }
    }
    __syncthreads();  // the slots are refilled by the next tile
  }
  if constexpr (Epi::kReduce) {
    // the block's partial for RHS q is warp (q mod kShWarps)'s sum; its writer fences before the
    // barrier, thread 0 arrives for the block
    __shared__ bool am_last;
    const double v0 = warp_sum(part[0]), v1 = warp_sum(part[1]);
    if (lane == 0) {
      if (w < nrhs) epi.partials[(size_t)w * kMaxPartials + blockIdx.x] = v0;
      if (w + kShWarps < nrhs) epi.partials[(size_t)(w + kShWarps) * kMaxPartials + blockIdx.x] = v1;
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) am_last = atomicAdd(epi.counter(), 1u) == gridDim.x - 1;
    __syncthreads();
    if (am_last) {
      __shared__ double tot[kMaxRhs];
      mrhs_totals(nrhs, epi.partials, tot);
      if (threadIdx.x < nrhs && epi.running(threadIdx.x)) epi.update(threadIdx.x, tot[threadIdx.x]);
      if (threadIdx.x == 0) *epi.counter() = 0u;
    }
  }
}

// one wave of the shared-link kernel's blocks (at most one per tile)
template <class KernelT>
static int w_shared_grid(KernelT kernel, int V) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kShThreads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  long long gx = (long long)sms * per_sm;
  const long long tiles = (V + kShTile - 1) / kShTile;
  if (gx > tiles) gx = tiles;
  if (gx > kMaxPartials) gx = kMaxPartials;
  return (int)gx;
}

// counter slots of sc[0] used by the multi-RHS CGNR kernels (the FP64 residual epilogue uses slot 4 of sc[r])
enum { kCtrWT = 9, kCtrWU = 10 };

// out_r = D_W in_r (op 0), M in_r (op 1), M^dagger in_r (op 2, with G5IN)
template <class FieldT, int OP>
struct WOpM {
  static constexpr bool kReduce = false;
  FieldT in, out;
  double kappa;
  double* partials;
  __device__ __forceinline__ bool running(int) const { return true; }
  __device__ __forceinline__ unsigned* counter() const { return nullptr; }
  template <class T, class A>
  __device__ __forceinline__ void site(int i, int r, const spinor<T>& acc, A&) const {
    if constexpr (OP == 0) out.at(r).store(i, acc);
    else out.at(r).store(i, m_combine<FieldT, OP == 2>(in.at(r), i, acc, (T)kappa));
  }
  __device__ __forceinline__ void update(int, double) const {}
};

// CGNR K1: t_r = M p_r, |t_r|^2 -> alpha_r = rr_r / |t_r|^2
template <class FieldT>
struct WEpiT {
  static constexpr bool kReduce = true;
  FieldT p, t;
  double kappa;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool running(int r) const { return sc[r].done == kRunning; }
  __device__ __forceinline__ unsigned* counter() const { return &sc[0].counter[kCtrWT]; }
  template <class T, class A>
  __device__ __forceinline__ void site(int i, int r, const spinor<T>& acc, A& red) const {
    const spinor<T> v = m_combine<FieldT, false>(p.at(r), i, acc, (T)kappa);
    t.at(r).store(i, v);
    accum(red, norm2(v));
  }
  __device__ __forceinline__ void update(int r, double tt) const {
    CgScalars& s = sc[r];
    const double alpha = s.rr / tt;
    if (!(tt > 0.0) || !isfinite(alpha)) s.done = kBreakdown;
    else s.alpha = alpha;
  }
};

// CGNR K2: s = M^dagger t_r; x_r += alpha_r p_r; r_r -= alpha_r s; |r_r|^2 -> beta_r and the exit tests
template <class FieldT, class XFieldT>
struct WEpiUpdate {
  static constexpr bool kReduce = true;
  FieldT t, p, r;
  XFieldT x;
  double kappa;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool running(int q) const { return sc[q].done == kRunning; }
  __device__ __forceinline__ unsigned* counter() const { return &sc[0].counter[kCtrWU]; }
  template <class T, class A>
  __device__ __forceinline__ void site(int i, int q, const spinor<T>& acc, A& red) const {
    using TX = typename XFieldT::T;
    const spinor<T> s = m_combine<FieldT, true>(t.at(q), i, acc, (T)kappa);
    const T alpha = (T)sc[q].alpha;
    const FieldT rf = r.at(q);
    const XFieldT xf = x.at(q);
    const spinor<T> pv = p.at(q).load(i);
    spinor<T> rv = rf.load(i);
    spinor<TX> xv = xf.load(i);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        rv.s[u].c[a].re = fma(-alpha, s.s[u].c[a].re, rv.s[u].c[a].re);
        rv.s[u].c[a].im = fma(-alpha, s.s[u].c[a].im, rv.s[u].c[a].im);
        xv.s[u].c[a].re = fma((TX)alpha, (TX)pv.s[u].c[a].re, xv.s[u].c[a].re);
        xv.s[u].c[a].im = fma((TX)alpha, (TX)pv.s[u].c[a].im, xv.s[u].c[a].im);
      }
    rf.store(i, rv);
    xf.store(i, xv);
    accum(red, norm2(rv));
  }
  __device__ __forceinline__ void update(int q, double rr) const {
    CgScalars& s = sc[q];
    s.iter += 1;
    s.since_ru += 1;
    s.rr_prev = s.rr;
    s.rr = rr;
    if (!isfinite(rr)) { s.done = kBreakdown; return; }
    s.beta = rr / s.rr_prev;
    if (rr > s.rmax2) s.rmax2 = rr;
    if (rr < s.delit) s.done = kConverged;
    else if (s.iter >= s.max_iter) s.done = kMaxIter;
    else if (s.mixed && (s.since_ru >= s.ru_interval || rr < s.delta2 * s.rmax2)) s.done = kReliable;
  }
};

// Residual of the normal equations at the high precision (FP64 or df64, HiT): res = rhs -
// M^dagger t (t = M x); r_lo <- res; |res|^2. Used for the convergence check and the final report.
template <class HiT, class FieldT, bool FINAL>
struct WEpiResidual {
  static constexpr int NV = 1;
  HiT t, rhs;
  FieldT r_lo;
  double kappa;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class TH, class A>
  __device__ __forceinline__ void site(int i, spinor<TH>& acc, A* red) const {
    using T = typename FieldT::T;
    const spinor<TH> s = m_combine<HiT, true>(t, i, acc, (TH)kappa);
    const spinor<TH> b = rhs.load(i);
    spinor<TH> res;
    spinor<T> rl;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        res.s[q].c[a] = {b.s[q].c[a].re - s.s[q].c[a].re, b.s[q].c[a].im - s.s[q].c[a].im};
        rl.s[q].c[a] = {(T)res.s[q].c[a].re, (T)res.s[q].c[a].im};
      }
    if (!FINAL) r_lo.store(i, rl);
    accum(red[0], norm2(res));
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    const A v[1] = {red[0]};
    double tot[1];
    if (grid_sum_last_block<1>(v, partials, &sc->counter[4], tot) && threadIdx.x == 0) {
      const double rr = tot[0];
      sc->res2 = rr;
      if (FINAL) return;
      if (!isfinite(rr)) { sc->done = kBreakdown; return; }
      sc->beta = sc->iter > 0 ? rr / sc->rr_prev : 0.0;
      sc->rr = rr;
      sc->rmax2 = rr;
      sc->since_ru = 0;
      if (sc->iter > 0) sc->ru_count += 1;
      if (rr < sc->delit) sc->done = kTrueConverged;
      else if (sc->iter >= sc->max_iter) sc->done = kMaxIter;
      else sc->done = kRunning;
    }
  }
};

// Reliable update of the mixed recursion, in two launches:
//   (1) high precision (FP64 or df64): s = b - M x_hi, the true residual of M x = b (where the
//       cancellation happens), stored at the inner precision;
//   (2) inner precision: r_lo = M^dagger s, |r_lo|^2 and the restart of the recursion.
// The error of (2) is relative to the current residual (rounding of order eps_inner * cond(M)), the
// same order as storing r_lo at the inner precision; convergence is only declared after the
// high-precision residual of the normal equations (WEpiResidual) confirms it.
template <class HiT, class FieldT>
struct WEpiSysResidual {
  static constexpr int NV = 0;
  HiT x, b;
  FieldT s_lo;
  double kappa;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class TH, class A>
  __device__ __forceinline__ void site(int i, spinor<TH>& acc, A*) const {
    using T = typename FieldT::T;
    const spinor<TH> mx = m_combine<HiT, false>(x, i, acc, (TH)kappa);
    const spinor<TH> bv = b.load(i);
    spinor<T> sv;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int a = 0; a < 3; ++a)
        sv.s[u].c[a] = {(T)(bv.s[u].c[a].re - mx.s[u].c[a].re), (T)(bv.s[u].c[a].im - mx.s[u].c[a].im)};
    s_lo.store(i, sv);
  }
  template <class A>
  __device__ __forceinline__ void finish(A*) const {}
};

template <class FieldT>
struct WEpiReliableInner {
  static constexpr int NV = 1;
  FieldT s, r_lo;
  double kappa;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class T, class A>
  __device__ __forceinline__ void site(int i, spinor<T>& acc, A* red) const {
    const spinor<T> v = m_combine<FieldT, true>(s, i, acc, (T)kappa);
    r_lo.store(i, v);
    accum(red[0], norm2(v));
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    const A v[1] = {red[0]};
    double tot[1];
    if (grid_sum_last_block<1>(v, partials, &sc->counter[4], tot) && threadIdx.x == 0) {
      const double rr = tot[0];
      if (!isfinite(rr)) { sc->done = kBreakdown; return; }
      sc->beta = sc->iter > 0 ? rr / sc->rr_prev : 0.0;
      sc->rr = rr;
      sc->rmax2 = rr;
      sc->since_ru = 0;
      sc->ru_count += 1;
      // below the tolerance: hand over to the full FP64 check (kConverged), never stop here
      if (rr < sc->delit) sc->done = kConverged;
      else if (sc->iter >= sc->max_iter) sc->done = kMaxIter;
      else sc->done = kRunning;
    }
  }
};

// ---------------------------------------------------------------- small streaming kernels
// p_r = r_r + beta_r p_r for every running RHS (grid.y = RHS)
template <class FieldT>
__global__ void __launch_bounds__(kBlock) w_p_kernel(int V, FieldT r_all, FieldT p_all, const CgScalars* sc) {
  using T = typename FieldT::T;
  const int q = blockIdx.y;
  if (sc[q].done != kRunning) return;
  const T beta = (T)sc[q].beta;
  const FieldT r = r_all.at(q), p = p_all.at(q);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const spinor<T> rv = r.load(i);
    spinor<T> pv = p.load(i);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pv.s[u].c[a].re = fma(beta, pv.s[u].c[a].re, rv.s[u].c[a].re);
        pv.s[u].c[a].im = fma(beta, pv.s[u].c[a].im, rv.s[u].c[a].im);
      }
    p.store(i, pv);
  }
}

// Start-up of one RHS with x = 0: r = rhs (inner precision), p = 0, x_lo = 0, x_hi = 0 and
// sc->res2 = |rhs|^2 (the residual of the normal equations at x = 0 needs no operator).
template <class HiT, class FieldT, class XFieldT>
__global__ void __launch_bounds__(kBlock) w_start_kernel(int V, HiT rhs, FieldT r, FieldT p, XFieldT x_lo, HiT x_hi,
                                                         CgScalars* sc, double* partials) {
  using T = typename FieldT::T;
  using TH = typename HiT::T;
  double red[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const spinor<TH> b = rhs.load(i);
    spinor<T> rl, z;
    spinor<typename XFieldT::T> zx;
    spinor<TH> zh;
    zero(z);
    zero(zx);
    zero(zh);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int a = 0; a < 3; ++a) rl.s[u].c[a] = {(T)b.s[u].c[a].re, (T)b.s[u].c[a].im};
    r.store(i, rl);
    p.store(i, z);
    x_lo.store(i, zx);
    x_hi.store(i, zh);
    accum(red[0], norm2(b));
  }
  double tot[1];
  if (grid_sum_last_block<1>(red, partials, &sc->counter[4], tot) && threadIdx.x == 0) sc->res2 = tot[0];
}

// canonical complex128[V][4][3] <-> packed
template <class FieldT>
__global__ void w_pack_kernel(int V, FieldT out, const double2* __restrict__ canon) {
  using T = typename FieldT::T;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    spinor<T> v;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const double2 d = canon[(size_t)i * 12 + q];
      v.s[q / 3].c[q % 3] = {(T)d.x, (T)d.y};
    }
    out.store(i, v);
  }
}
template <class FieldT>
__global__ void w_unpack_kernel(int V, double2* __restrict__ canon, FieldT in) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const auto v = in.load(i);
#pragma unroll
    for (int q = 0; q < 12; ++q) canon[(size_t)i * 12 + q] = make_double2((double)v.s[q / 3].c[q % 3].re, (double)v.s[q / 3].c[q % 3].im);
  }
}
// zero a field
template <class FieldT>
__global__ void w_zero_kernel(int V, FieldT f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    spinor<typename FieldT::T> z;
    zero(z);
    f.store(i, z);
  }
}
// x_hi += x_lo, x_lo = 0
template <class HiT, class XFieldT>
__global__ void w_accumulate_kernel(int V, HiT xh, XFieldT xl) {
  using TH = typename HiT::T;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    spinor<TH> a = xh.load(i);
    const auto b = xl.load(i);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a.s[q].c[c].re += (TH)b.s[q].c[c].re;
        a.s[q].c[c].im += (TH)b.s[q].c[c].im;
      }
    xh.store(i, a);
    spinor<typename XFieldT::T> z;
    zero(z);
    xl.store(i, z);
  }
}

template <int PREC>
__global__ void w_pack_links_kernel(Geom g, int V, const double2* __restrict__ canon, void* out) {
  const long long total = 4ll * V;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % V), mu = (int)(t / V);
    int c[4];
    full_site(g, i, c);
    const double z = (mu == 3 && c[3] == g.L3 - 1) ? (double)g.tbc : 1.0;
    const double2* src = canon + ((size_t)i * 4 + mu) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const double2 d = src[e];
      const size_t o = ((size_t)mu * 9 + e) * V + i;
      if constexpr (PREC == QCD_PREC_DOUBLE) {
        ((double2*)out)[o] = make_double2(z * d.x, z * d.y);
      } else if constexpr (PREC == QCD_PREC_DF64) {
        const df64 re(z * d.x), im(z * d.y);
        ((float4*)out)[o] = make_float4(re.hi, re.lo, im.hi, im.lo);
      } else {
        ((float2*)out)[o] = make_float2((float)(z * d.x), (float)(z * d.y));
      }
    }
  }
}

// ---------------------------------------------------------------- host side
// Workspace of an R-RHS CGNR: every per-RHS field is R fields back to back.
struct WWork {
  CgScalars* sc;           // [R]
  double* partials;        // [max(R, 2)][kMaxPartials]
  void *b64, *rhs, *x_hi;  // high precision (FP64 or df64, 16 B per complex), R fields each: b,
                           // M^dagger b, the solution accumulator
  void* t64;               // high-precision scratch, one field (reliable updates run one RHS at a time)
  void *r, *p, *t;         // inner precision, R fields each
  void* x_lo;              // inner precision, R fields (aliases x_hi in FP64)
  size_t total;
};

static WWork w_carve(long long V, int prec, int R, char* base) {
  WWork w{};
  size_t off = 0;
  auto take = [&](size_t n) { void* q = base ? base + off : nullptr; off += align256(n); return q; };
  w.sc = (CgScalars*)take(sizeof(CgScalars) * R);
  w.partials = (double*)take(sizeof(double) * kMaxPartials * (R > 2 ? R : 2));
  const size_t f64 = wfield_bytes(QCD_PREC_DOUBLE, V), fin = wfield_bytes(prec, V);
  w.b64 = take(f64 * R);
  w.rhs = take(f64 * R);
  w.x_hi = take(f64 * R);
  w.t64 = take(f64);
  w.r = take(fin * R);
  w.p = take(fin * R);
  w.t = take(fin * R);
  w.x_lo = prec == QCD_PREC_DOUBLE ? w.x_hi : take(fin * R);
  w.total = off;
  return w;
}

size_t wilson_workspace_bytes(const qcd_lattice* lat, int prec, int nrhs) {
  return w_carve(lat->V, prec, nrhs, nullptr).total;
}

template <int PREC>
static WField<PREC> wf(void* p, int V) {
  return {(typename std::conditional<PREC == QCD_PREC_DOUBLE, double2, float4>::type*)p, V};
}
template <int PREC>
static WLinks<PREC> wl(const void* p, int V) {
  using E = typename std::conditional<PREC == QCD_PREC_DOUBLE, double2,
                                      typename std::conditional<PREC == QCD_PREC_DF64, float4, float2>::type>::type;
  return {(const E*)p, V};
}

int launch_wilson_pack_links(const qcd_lattice* lat, const void* canon, void* out, int prec, cudaStream_t st) {
  const Geom g = make_geom(lat);
  const int V = (int)lat->V;
  const int grid = (int)std::min<long long>((4ll * V + 255) / 256, 152 * 64);
  if (prec == QCD_PREC_DOUBLE) w_pack_links_kernel<QCD_PREC_DOUBLE><<<grid, 256, 0, st>>>(g, V, (const double2*)canon, out);
  else if (prec == QCD_PREC_SINGLE) w_pack_links_kernel<QCD_PREC_SINGLE><<<grid, 256, 0, st>>>(g, V, (const double2*)canon, out);
  else if (prec == QCD_PREC_DF64) w_pack_links_kernel<QCD_PREC_DF64><<<grid, 256, 0, st>>>(g, V, (const double2*)canon, out);
  else return QCD_ERR_UNSUPPORTED;
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

int launch_wilson_pack(const qcd_lattice* lat, void* packed, const void* canon, int prec, bool unpack, cudaStream_t st) {
  const int V = (int)lat->V;
  const int grid = site_grid(V);
  if (prec == QCD_PREC_DOUBLE) {
    if (unpack) w_unpack_kernel<<<grid, kBlock, 0, st>>>(V, (double2*)canon, wf<QCD_PREC_DOUBLE>(packed, V));
    else w_pack_kernel<<<grid, kBlock, 0, st>>>(V, wf<QCD_PREC_DOUBLE>(packed, V), (const double2*)canon);
  } else if (prec == QCD_PREC_SINGLE) {
    if (unpack) w_unpack_kernel<<<grid, kBlock, 0, st>>>(V, (double2*)canon, wf<QCD_PREC_SINGLE>(packed, V));
    else w_pack_kernel<<<grid, kBlock, 0, st>>>(V, wf<QCD_PREC_SINGLE>(packed, V), (const double2*)canon);
  } else if (prec == QCD_PREC_DF64) {
    if (unpack) w_unpack_kernel<<<grid, kBlock, 0, st>>>(V, (double2*)canon, wf<QCD_PREC_DF64>(packed, V));
    else w_pack_kernel<<<grid, kBlock, 0, st>>>(V, wf<QCD_PREC_DF64>(packed, V), (const double2*)canon);
  } else {
    return QCD_ERR_UNSUPPORTED;
  }
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

template <int PREC>
static int wilson_op_typed(const qcd_lattice* lat, void* out, const void* in, double kappa, int mode, cudaStream_t st) {
  const Geom g = make_geom(lat);
  const int V = (int)lat->V;
  auto U = wl<PREC>(lat->wilson_links[PREC], V);
  auto fin = wf<PREC>(const_cast<void*>(in), V);
  auto fout = wf<PREC>(out, V);
  const int grid = site_grid(V);
  using FT = WField<PREC>;
  if (mode == 0) wilson_kernel<WLinks<PREC>, FT, false><<<grid, kBlock, 0, st>>>(g, V, U, fin, WStore<FT>{fout});
  else if (mode == 1) wilson_kernel<WLinks<PREC>, FT, false><<<grid, kBlock, 0, st>>>(g, V, U, fin, WApplyM<FT, false>{fin, fout, kappa});
  else wilson_kernel<WLinks<PREC>, FT, true><<<grid, kBlock, 0, st>>>(g, V, U, fin, WApplyM<FT, true>{fin, fout, kappa});
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

// mode 0: out = D_W in; 1: out = M in; 2: out = M^dagger in
int launch_wilson_op(const qcd_lattice* lat, void* out, const void* in, double kappa, int mode, int prec, cudaStream_t st) {
  if (prec == QCD_PREC_DOUBLE) return wilson_op_typed<QCD_PREC_DOUBLE>(lat, out, in, kappa, mode, st);
  if (prec == QCD_PREC_SINGLE) return wilson_op_typed<QCD_PREC_SINGLE>(lat, out, in, kappa, mode, st);
  if (prec == QCD_PREC_DF64) return wilson_op_typed<QCD_PREC_DF64>(lat, out, in, kappa, mode, st);
  return QCD_ERR_UNSUPPORTED;
}

// (x, y) grid for a multi-RHS kernel: gy rows, x-extent within one wave of resident blocks (each
// block ends in a fence + counter update, so further waves only add that cost).
template <class KernelT>
static dim3 w_grid(KernelT kernel, long long V, int gy) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  const long long need = (V + kBlock - 1) / kBlock;
  long long gx = (long long)sms * per_sm / gy;
  if (gx > need) gx = need;
  if (gx > kMaxPartials) gx = kMaxPartials;
  return dim3((unsigned)(gx > 0 ? gx : 1), (unsigned)gy);
}

// register block of right-hand sides: the opts value if given (1, 2, 4 in FP32; 1, 2 in FP64), else 1
// below kShWarps RHS (measured for 8 RHS on 32^3x64 in FP32 before the shared-link kernel: 177 ms of
// operator time per solve against 207 ms for 2 and 265 ms for 4)
// -1 (kRhsShared) selects the shared-link kernel, the default from kShWarps right-hand sides on
// (fewer leave warps of its blocks idle). Returns 0 for a request this precision does not support.
int wilson_rhs_block(int prec, int R, int requested) {
  const int cap = prec == QCD_PREC_DOUBLE ? 2 : 4;
  if (requested == kRhsShared) return kRhsShared;
  if (requested > 0) return (requested == 1 || requested == 2 || requested == 4) && requested <= cap ? requested : 0;
  return R >= kShWarps ? kRhsShared : 1;
}

template <int PREC, int RB>
static int wilson_op_mrhs_typed(const qcd_lattice* lat, void* out, const void* in, int R, double kappa, int mode,
                                cudaStream_t st) {
  using FT = WField<PREC>;
  const Geom g = make_geom(lat);
  const int V = (int)lat->V;
  auto U = wl<PREC>(lat->wilson_links[PREC], V);
  const FT fin = wf<PREC>(const_cast<void*>(in), V), fout = wf<PREC>(out, V);
  if (mode == 0) {
    auto k = wilson_mrhs_kernel<WLinks<PREC>, FT, false, RB, WOpM<FT, 0>>;
    k<<<w_grid(k, V, 1), kBlock, 0, st>>>(g, V, U, fin, R, WOpM<FT, 0>{fin, fout, kappa, nullptr});
  } else if (mode == 1) {
    auto k = wilson_mrhs_kernel<WLinks<PREC>, FT, false, RB, WOpM<FT, 1>>;
    k<<<w_grid(k, V, 1), kBlock, 0, st>>>(g, V, U, fin, R, WOpM<FT, 1>{fin, fout, kappa, nullptr});
  } else {
    auto k = wilson_mrhs_kernel<WLinks<PREC>, FT, true, RB, WOpM<FT, 2>>;
    k<<<w_grid(k, V, 1), kBlock, 0, st>>>(g, V, U, fin, R, WOpM<FT, 2>{fin, fout, kappa, nullptr});
  }
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

template <int PREC>
static int wilson_op_mrhs_shared(const qcd_lattice* lat, void* out, const void* in, int R, double kappa, int mode,
                                 cudaStream_t st) {
  using FT = WField<PREC>;
  const Geom g = make_geom(lat);
  const int V = (int)lat->V;
  auto U = wl<PREC>(lat->wilson_links[PREC], V);
  const FT fin = wf<PREC>(const_cast<void*>(in), V), fout = wf<PREC>(out, V);
  if (mode == 0) {
    auto k = wilson_mrhs_shared_kernel<WLinks<PREC>, FT, false, WOpM<FT, 0>>;
    k<<<w_shared_grid(k, V), kShThreads, 0, st>>>(g, V, U, fin, R, WOpM<FT, 0>{fin, fout, kappa, nullptr},
                                                   w_sweep_chunk(g));
  } else if (mode == 1) {
    auto k = wilson_mrhs_shared_kernel<WLinks<PREC>, FT, false, WOpM<FT, 1>>;
    k<<<w_shared_grid(k, V), kShThreads, 0, st>>>(g, V, U, fin, R, WOpM<FT, 1>{fin, fout, kappa, nullptr},
                                                   w_sweep_chunk(g));
  } else {
    auto k = wilson_mrhs_shared_kernel<WLinks<PREC>, FT, true, WOpM<FT, 2>>;
    k<<<w_shared_grid(k, V), kShThreads, 0, st>>>(g, V, U, fin, R, WOpM<FT, 2>{fin, fout, kappa, nullptr},
                                                   w_sweep_chunk(g));
  }
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

int launch_wilson_op_mrhs(const qcd_lattice* lat, void* out, const void* in, int R, double kappa, int mode, int prec,
                          cudaStream_t st) {
  // the default kernel for R right-hand sides: shared links from kShWarps on, else register block 1
  const bool shared = wilson_rhs_block(prec, R, 0) == kRhsShared;
  if (prec == QCD_PREC_DOUBLE)
    return shared ? wilson_op_mrhs_shared<QCD_PREC_DOUBLE>(lat, out, in, R, kappa, mode, st)
                  : wilson_op_mrhs_typed<QCD_PREC_DOUBLE, 1>(lat, out, in, R, kappa, mode, st);
  if (prec == QCD_PREC_SINGLE)
    return shared ? wilson_op_mrhs_shared<QCD_PREC_SINGLE>(lat, out, in, R, kappa, mode, st)
                  : wilson_op_mrhs_typed<QCD_PREC_SINGLE, 1>(lat, out, in, R, kappa, mode, st);
  return QCD_ERR_UNSUPPORTED;
}

// CGNR on R right-hand sides: each RHS r has its own scalars sc[r]; one iteration is
//   K3  p_r = r_r + beta_r p_r                          (w_p_kernel, grid.y = RHS)
//   K1  t_r = M p_r, alpha_r = rr_r / |t_r|^2             (multi-RHS operator kernel)
//   K2  r_r -= alpha_r M^dagger t_r, x_r += alpha_r p_r, beta_r, exit tests
// A converged or max-iteration RHS drops out of the kernels. Reliable updates (the true residual
// s = b - M x_hi at the high precision HI, then r_lo = M^dagger s at the inner precision) run per
// RHS between iterations; a RHS whose residual falls below the tolerance is confirmed by the full
// residual of the normal equations at HI, M^dagger b - M^dagger M x_hi, before it stops. HI is FP64,
// or df64 (opts->prec_outer): the same 16 bytes per complex, a 48-bit significand, and the
// high-precision operator on the FP32 pipes, which on GB300 run it about five times faster than
// the FP64 pipe. The host reads the R
// states after every k iterations (k = opts->check_interval for one RHS, 1 for several, so that a
// RHS waiting for its update does not idle while the others iterate).
template <int PREC, int HI, int RB>
static int wilson_cgnr_typed(qcd_lattice* lat, int R, void* x, const void* b, double kappa, double tol, int max_iter,
                             const qcd_solver_opts& o, void* ws, qcd_solve_info* info, cudaStream_t st) {
  using FT = WField<PREC>;
  using FH = WField<HI>;  // the high precision: FP64, or df64 on the FP32 pipes
  const Geom g = make_geom(lat);
  const int V = (int)lat->V;
  const bool mixed = PREC != QCD_PREC_DOUBLE;
  WWork w = w_carve(V, PREC, R, (char*)ws);
  auto U = wl<PREC>(lat->wilson_links[PREC], V);
  auto UH = wl<HI>(lat->wilson_links[HI], V);
  const FT r = wf<PREC>(w.r, V), p = wf<PREC>(w.p, V), t = wf<PREC>(w.t, V), xl = wf<PREC>(w.x_lo, V);
  const FH b64 = wf<HI>(w.b64, V), rhs = wf<HI>(w.rhs, V);
  const FH xh = wf<HI>(w.x_hi, V), t64 = wf<HI>(w.t64, V);
  const int grid = one_wave_grid(V, wilson_kernel<WLinks<HI>, FH, true, WEpiResidual<FH, FT, false>>);
  const int grid_ru = one_wave_grid(V, wilson_kernel<WLinks<PREC>, FT, true, WEpiReliableInner<FT>>);
  // the two operator launches of an iteration: the shared-link kernel (RB == kRhsShared) or the
  // register-blocked one
  constexpr int RBK = RB == kRhsShared ? 1 : RB;
  auto K1 = wilson_mrhs_kernel<WLinks<PREC>, FT, false, RBK, WEpiT<FT>>;
  auto K2 = wilson_mrhs_kernel<WLinks<PREC>, FT, true, RBK, WEpiUpdate<FT, FT>>;
  auto S1 = wilson_mrhs_shared_kernel<WLinks<PREC>, FT, false, WEpiT<FT>>;
  auto S2 = wilson_mrhs_shared_kernel<WLinks<PREC>, FT, true, WEpiUpdate<FT, FT>>;
  const dim3 gp = w_grid(w_p_kernel<FT>, V, R);
  const int zc = w_sweep_chunk(g);
  const dim3 g1 = RB == kRhsShared ? dim3(w_shared_grid(S1, V)) : w_grid(K1, V, 1);
  const dim3 g2 = RB == kRhsShared ? dim3(w_shared_grid(S2, V)) : w_grid(K2, V, 1);
  const size_t cbytes = (size_t)V * 12 * sizeof(double2);  // one canonical spinor field
  long long launches = 0;

  std::vector<CgScalars> h(R);
  for (auto& s : h) {
    s = CgScalars{};
    s.tol2 = tol * tol;
    s.max_iter = max_iter;
    s.ru_interval = o.reliable_interval > 0 ? o.reliable_interval : 100;
    s.delta2 = o.reliable_delta * o.reliable_delta;
    s.mixed = mixed ? 1 : 0;
  }
  auto upload = [&]() -> int {
    QCD_CUDA(cudaMemcpyAsync(w.sc, h.data(), sizeof(CgScalars) * R, cudaMemcpyHostToDevice, st));
    return QCD_OK;
  };
  auto download = [&]() -> int {
    QCD_CUDA(cudaMemcpyAsync(h.data(), w.sc, sizeof(CgScalars) * R, cudaMemcpyDeviceToHost, st));
    QCD_CUDA(cudaStreamSynchronize(st));
    return QCD_OK;
  };
  int rc = upload();
  if (rc) return rc;
  // start-up per RHS: rhs_q = M^dagger b_q (high precision); r_q = rhs_q, p_q = x_q = 0; |rhs_q|^2
  for (int q = 0; q < R; ++q) {
    if ((rc = launch_wilson_pack(lat, b64.at(q).p, (const char*)b + q * cbytes, HI, false, st))) return rc;
    wilson_kernel<WLinks<HI>, FH, true><<<grid, kBlock, 0, st>>>(
        g, V, UH, b64.at(q), WApplyM<FH, true>{b64.at(q), rhs.at(q), kappa});
    w_start_kernel<<<grid, kBlock, 0, st>>>(V, rhs.at(q), r.at(q), p.at(q), xl.at(q), xh.at(q), w.sc + q, w.partials);
    launches += 3;
  }
  QCD_CUDA(cudaGetLastError());
  if ((rc = download())) return rc;
  std::vector<double> rhs2(R);
  for (int q = 0; q < R; ++q) {
    CgScalars& s = h[q];
    rhs2[q] = s.res2;
    s.delit = tol * tol * rhs2[q];
    s.rr = s.rr_prev = s.rmax2 = rhs2[q];
    s.done = !std::isfinite(rhs2[q]) ? kBreakdown : (rhs2[q] == 0.0 ? kTrueConverged : kRunning);
  }
  if ((rc = upload())) return rc;

  // high-precision residual of the normal equations for RHS q: x_hi += x_lo; t64 = M x_hi;
  // res = rhs - M^dagger t64 (-> r_lo unless final_report); sc[q] state from |res|^2
  auto true_residual = [&](int q, bool final_report) -> int {
    if (mixed) w_accumulate_kernel<<<grid, kBlock, 0, st>>>(V, xh.at(q), xl.at(q));
    wilson_kernel<WLinks<HI>, FH, false><<<grid, kBlock, 0, st>>>(
        g, V, UH, xh.at(q), WApplyM<FH, false>{xh.at(q), t64, kappa});
    if (final_report)
      wilson_kernel<WLinks<HI>, FH, true><<<grid, kBlock, 0, st>>>(
          g, V, UH, t64, WEpiResidual<FH, FT, true>{t64, rhs.at(q), r.at(q), kappa, w.sc + q, w.partials});
    else
      wilson_kernel<WLinks<HI>, FH, true><<<grid, kBlock, 0, st>>>(
          g, V, UH, t64, WEpiResidual<FH, FT, false>{t64, rhs.at(q), r.at(q), kappa, w.sc + q, w.partials});
    launches += mixed ? 3 : 2;
    QCD_CUDA(cudaGetLastError());
    return QCD_OK;
  };

  // reliable update of the mixed recursion for RHS q (x_hi += x_lo; s = b - M x_hi at HI;
  // r_lo = M^dagger s at the inner precision)
  auto reliable_update = [&](int q) -> int {
    w_accumulate_kernel<<<grid, kBlock, 0, st>>>(V, xh.at(q), xl.at(q));
    wilson_kernel<WLinks<HI>, FH, false><<<grid, kBlock, 0, st>>>(
        g, V, UH, xh.at(q), WEpiSysResidual<FH, FT>{xh.at(q), b64.at(q), t.at(q), kappa});
    wilson_kernel<WLinks<PREC>, FT, true><<<grid_ru, kBlock, 0, st>>>(
        g, V, U, t.at(q), WEpiReliableInner<FT>{t.at(q), r.at(q), kappa, w.sc + q, w.partials});
    launches += 3;
    QCD_CUDA(cudaGetLastError());
    return QCD_OK;
  };

  const bool profile = o.profile != 0;
  const int k = R > 1 ? 1 : (o.check_interval > 0 ? o.check_interval : 8);
  std::vector<cudaEvent_t> ev(profile ? 2 * k : 0, nullptr);
  auto cleanup = [&]() {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  };
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) { cleanup(); return cuda_fail(cudaGetLastError(), "cudaEventCreate"); }
  double dslash_ms = 0.0;
  long long op_launches = 0;
  while (true) {
    bool running = false, updated = false;
    for (int q = 0; q < R; ++q) {
      const int d = h[q].done;
      if (d == kConverged) {  // confirmed (or refuted) by the full high-precision residual
        if ((rc = true_residual(q, false))) { cleanup(); return rc; }
        updated = true;
      } else if (mixed && d == kReliable) {
        if ((rc = reliable_update(q))) { cleanup(); return rc; }
        updated = true;
      } else if (d == kRunning) {
        running = true;
      }
    }
    if (updated) {
      if ((rc = download())) { cleanup(); return rc; }
      continue;
    }
    if (!running) break;
    for (int i = 0; i < k; ++i) {
      w_p_kernel<<<gp, kBlock, 0, st>>>(V, r, p, w.sc);
      if (profile) cudaEventRecord(ev[2 * i], st);
      if (RB == kRhsShared) {
        S1<<<g1, kShThreads, 0, st>>>(g, V, U, p, R, WEpiT<FT>{p, t, kappa, w.sc, w.partials}, zc);
        S2<<<g2, kShThreads, 0, st>>>(g, V, U, t, R, WEpiUpdate<FT, FT>{t, p, r, xl, kappa, w.sc, w.partials}, zc);
      } else {
        K1<<<g1, kBlock, 0, st>>>(g, V, U, p, R, WEpiT<FT>{p, t, kappa, w.sc, w.partials});
        K2<<<g2, kBlock, 0, st>>>(g, V, U, t, R, WEpiUpdate<FT, FT>{t, p, r, xl, kappa, w.sc, w.partials});
      }
      if (profile) cudaEventRecord(ev[2 * i + 1], st);
      launches += 3;
      op_launches += 2;
    }
    QCD_CUDA(cudaGetLastError());
    if ((rc = download())) { cleanup(); return rc; }
    if (profile) {
      for (int i = 0; i < k; ++i) {
        float ms = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaEventElapsedTime"); }
        dslash_ms += ms;
      }
    }
  }
  cleanup();
  // final report: a RHS that ended on a confirmed high-precision residual (kTrueConverged) already holds it
  // in res2 with x_lo folded into x_hi; the others are recomputed here
  for (int q = 0; q < R; ++q)
    if (h[q].done != kTrueConverged && (rc = true_residual(q, true))) return rc;
  for (int q = 0; q < R; ++q)
    if ((rc = launch_wilson_pack(lat, xh.at(q).p, (char*)x + q * cbytes, HI, true, st))) return rc;
  launches += R;
  if ((rc = download())) return rc;
  int status = QCD_OK;
  for (int q = 0; q < R; ++q) {
    const CgScalars& s = h[q];
    const double true_rel = rhs2[q] > 0 ? std::sqrt(s.res2 / rhs2[q]) : 0.0;
    int st_q = s.done == kBreakdown ? QCD_ERR_BREAKDOWN
                                    : (s.done == kMaxIter ? QCD_ERR_NOT_CONVERGED : QCD_OK);
    if (st_q == QCD_OK && !(true_rel <= tol)) st_q = QCD_ERR_NOT_CONVERGED;
    if (st_q == QCD_ERR_BREAKDOWN || (status == QCD_OK && st_q != QCD_OK)) status = st_q;
    if (info) {
      qcd_solve_info& in = info[q];
      in.iterations = s.iter;
      in.reliable_updates = s.ru_count;
      in.true_rel_residual = true_rel;
      in.iterated_rel_residual = rhs2[q] > 0 ? std::sqrt(s.rr / rhs2[q]) : 0.0;
      in.converged = st_q == QCD_OK;
      in.status = st_q;
    }
  }
  if (info) {
    info[0].kernel_launches = (int)launches;
    info[0].dslash_launches = (int)op_launches;
    info[0].dslash_ms = dslash_ms;
  }
  return status;
}

int run_wilson_cgnr(qcd_lattice* lat, int R, void* x, const void* b, double kappa, double tol, int max_iter,
                    const qcd_solver_opts& o, void* ws, qcd_solve_info* info, cudaStream_t st) {
  const int rb = wilson_rhs_block(o.prec_inner, R, o.rhs_block);
  if (rb == 0) {
    set_error("unsupported RHS block %d for Wilson precision %d", o.rhs_block, o.prec_inner);
    return QCD_ERR_INVALID_ARG;
  }
  constexpr int D = QCD_PREC_DOUBLE, S = QCD_PREC_SINGLE, DF = QCD_PREC_DF64, SH = kRhsShared;
  if (o.prec_inner == D) {
    if (rb == SH) return wilson_cgnr_typed<D, D, SH>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
    if (rb == 1) return wilson_cgnr_typed<D, D, 1>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
    return wilson_cgnr_typed<D, D, 2>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
  }
  if (o.prec_inner == S && o.prec_outer == D) {
    if (rb == SH) return wilson_cgnr_typed<S, D, SH>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
    if (rb == 1) return wilson_cgnr_typed<S, D, 1>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
    if (rb == 2) return wilson_cgnr_typed<S, D, 2>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
    return wilson_cgnr_typed<S, D, 4>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
  }
  if (o.prec_inner == S && o.prec_outer == DF) {
    if (rb == SH) return wilson_cgnr_typed<S, DF, SH>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
    if (rb == 1) return wilson_cgnr_typed<S, DF, 1>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
    if (rb == 2) return wilson_cgnr_typed<S, DF, 2>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
    return wilson_cgnr_typed<S, DF, 4>(lat, R, x, b, kappa, tol, max_iter, o, ws, info, st);
  }
  return QCD_ERR_UNSUPPORTED;
}

}  // namespace qcd
