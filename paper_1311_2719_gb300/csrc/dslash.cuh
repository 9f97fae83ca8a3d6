// The staggered hopping term on one output parity (the paper's matrix-vector routine, §3) and
// the generic site kernel that fuses a caller-chosen epilogue onto it (the CG vector algebra of
// the paper's congrad, §4).
#pragma once

#include <type_traits>

#include "qcd_internal.cuh"

namespace qcd {

// A neighbour vector v and a factor s with in(j) = s v: the FP16 field's per-site scale (its
// load_raw), else s = 1. The unfolded-link hop multiplies U v by (sign / 2) s in one coefficient.
template <class In>
__device__ __forceinline__ auto load_unscaled(const In& in, int j, typename In::T& s, int)
    -> decltype(in.load_raw(j, s)) {
  return in.load_raw(j, s);
}
template <class In>
__device__ __forceinline__ cvec3<typename In::T> load_unscaled(const In& in, int j, typename In::T& s, long) {
  s = typename In::T(1);
  return in.load(j);
}

// out(n) = sum_mu [ s_mu(n) U_mu(n) in(n+mu) - s_mu(n-mu) U_mu(n-mu)^dagger in(n-mu) ] / 2 for the
// even-odd site k of parity out_par; s = eta * zeta. Folded links already carry s/2.
template <class LinksT, class FieldT>
__device__ __forceinline__ cvec3<typename LinksT::T> hop(const Geom& g, const LinksT& U, const FieldT& in,
                                                         int out_par, int k) {
  using T = typename LinksT::T;
  const Site s = site_of(g, k, out_par);
  int fwd[4], bwd[4];
  neighbours(g, s, fwd, bwd);
  cvec3<T> acc;
  zero(acc);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const su3<T> Uf = U.load(out_par, mu, k);
    if constexpr (LinksT::kFolded) {
      mul_add(acc, Uf, in.load(fwd[mu]));
    } else {
      T sc;
      const cvec3<T> xf = load_unscaled(in, fwd[mu], sc, 0);
      axpy(acc, T(0.5f * fwd_sign(g, s, mu)) * sc, mul(Uf, xf));
    }
    const su3<T> Ub = U.load(1 - out_par, mu, bwd[mu]);
    if constexpr (LinksT::kFolded) {
      adj_mul_sub(acc, Ub, in.load(bwd[mu]));
    } else {
      T sc;
      const cvec3<T> xb = load_unscaled(in, bwd[mu], sc, 0);
      axpy(acc, T(-0.5f * bwd_sign(g, s, mu)) * sc, adj_mul(Ub, xb));
    }
  }
  return acc;
}

// The four forward hops (sub = 0) or the four backward hops (sub = 1) of site k, written as ONE
// instruction stream for both lanes of a pair: the link parity and indices are selected, and
// the backward lane multiplies by -U^dagger (or -s/2 U^dagger) built element by element with
// selects, so the two lanes of a warp never diverge.
template <class LinksT, class FieldT>
__device__ __forceinline__ cvec3<typename LinksT::T> hop_half(const Geom& g, const LinksT& U, const FieldT& in,
                                                              int out_par, int k, int sub) {
  using T = typename LinksT::T;
  const Site s = site_of(g, k, out_par);
  int fwd[4], bwd[4];
  neighbours(g, s, fwd, bwd);
  const int lpar = out_par ^ sub;
  cvec3<T> acc;
  zero(acc);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int li = sub ? bwd[mu] : k;
    const int xi = sub ? bwd[mu] : fwd[mu];
    const su3<T> L = U.load(lpar, mu, li);
    T sc = T(1);
    cvec3<T> xv;
    if constexpr (LinksT::kFolded) xv = in.load(xi);
    else xv = load_unscaled(in, xi, sc, 0);
    su3<T> M;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        M.e[a][b].re = sub ? -L.e[b][a].re : L.e[a][b].re;
        M.e[a][b].im = sub ? L.e[b][a].im : L.e[a][b].im;
      }
    if constexpr (LinksT::kFolded) {
      mul_add(acc, M, xv);
    } else {
      const float sg = sub ? bwd_sign(g, s, mu) : fwd_sign(g, s, mu);
      axpy(acc, T(0.5f * sg) * sc, mul(M, xv));
    }
  }
  return acc;
}

__device__ __forceinline__ float shfl_pair(float v) { return __shfl_xor_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_pair(double v) { return __shfl_xor_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ df64 shfl_pair(df64 v) { return df64(shfl_pair(v.hi), shfl_pair(v.lo)); }

template <typename T>
__device__ __forceinline__ void pair_sum(cvec3<T>& acc) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc.c[a].re += shfl_pair(acc.c[a].re);
    acc.c[a].im += shfl_pair(acc.c[a].im);
  }
}

// Epilogue interface:
//   static constexpr int NV;                        number of FP64 sums reduced over the grid
//   static constexpr bool kPrefetch;                true: prefetch(k) / site_pre(k, acc, red, pre)
//                                                   are used on the one-thread-per-site path
//   bool skip() const;                              true -> whole kernel returns at once
//   void site(int k, cvec3<T>& acc, A* red);        consume the hop result of site k (A = Accum<T>)
//   void finish(A* red);                            grid reduction + scalar update (NV > 0)
// TPS = threads per output site: 1, or 2 (forward / backward hops on a lane pair, for lattices
// too small to fill the GPU with one thread per site).
// Resident blocks per SM the operator kernels are compiled for: 8 (<= 64 registers) for the
// FP32-arithmetic operators, which are bound by memory latency and need the warps (measured on
// GB300: the reduction epilogues otherwise take 96 registers and half the occupancy); 5 for FP64
// and 4 for df64, whose 64-bit operands need the registers.
template <class LinksT>
struct MinBlocks {
  static constexpr int value =
      sizeof(typename LinksT::T) == 4 ? 8 : (std::is_same<typename LinksT::T, double>::value ? 5 : 4);
};

// The same budget as a register cap, so that a launch may also use wider blocks (one block per SM
// on lattices smaller than a wave, see cg_launch_shape): 64 / 96 / 128 registers.
template <class LinksT>
struct MaxRegs {
  static constexpr int value = 65536 / (kBlock * MinBlocks<LinksT>::value) / 8 * 8;
};

// The operator's input as the epilogue sees it: an epilogue with a bind(in) member replaces the
// input accessor at kernel start (the CG's K1 reads p = r + beta p_old instead of a stored p).
template <class Epi, class In>
__device__ __forceinline__ auto bind_input(const Epi& epi, const In& in, int) -> decltype(epi.bind(in)) {
  return epi.bind(in);
}
template <class Epi, class In>
__device__ __forceinline__ In bind_input(const Epi&, const In& in, long) {
  return in;
}

template <class LinksT, class FieldT, class Epi, int TPS = 1>
__global__ void __maxnreg__(MaxRegs<LinksT>::value) dslash_kernel(Geom g, LinksT U, FieldT in_arg,
                                                                                 int out_par, Epi epi) {
  if (epi.skip()) return;
  const auto in = bind_input(epi, in_arg, 0);
  using A = typename Accum<typename LinksT::T>::type;
  A red[Epi::NV > 0 ? Epi::NV : 1];
#pragma unroll
  for (int j = 0; j < (Epi::NV > 0 ? Epi::NV : 1); ++j) red[j] = A(0);
  if constexpr (TPS == 1) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
      if constexpr (Epi::kPrefetch) {
        // the epilogue's own-site operands are loaded before the hop so that their latency
        // overlaps the neighbour gathers instead of following them
        const auto pre = epi.prefetch(k);
        auto acc = hop(g, U, in, out_par, k);
        epi.site_pre(k, acc, red, pre);
      } else {
        auto acc = hop(g, U, in, out_par, k);
        epi.site(k, acc, red);
      }
    }
  } else {
    // block-uniform trip count: every lane reaches the pair shuffle in every pass
    const int per_block = blockDim.x >> 1;
    const int sub = threadIdx.x & 1;
    for (int base = blockIdx.x * per_block; base < g.Vh; base += gridDim.x * per_block) {
      const int k = base + (threadIdx.x >> 1);
      const bool valid = k < g.Vh;
      cvec3<typename LinksT::T> acc;
      if (valid) acc = hop_half(g, U, in, out_par, k, sub);
      else zero(acc);
      pair_sum(acc);
      if (valid && sub == 0) epi.site(k, acc, red);
    }
  }
  if constexpr (Epi::NV > 0) epi.finish(red);
}

// Plain store epilogue.
template <class FieldT>
struct EpiStore {
  static constexpr int NV = 0;
  static constexpr bool kPrefetch = false;
  FieldT out;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class T, class A>
  __device__ __forceinline__ void site(int k, cvec3<T>& acc, A*) const {
    out.store(k, acc);
  }
  template <class A>
  __device__ __forceinline__ void finish(A*) const {}
};

template <int PREC>
__host__ __device__ inline Field<PREC> make_field(void* p, int Vh);
template <>
__host__ __device__ inline Field<QCD_PREC_DOUBLE> make_field<QCD_PREC_DOUBLE>(void* p, int Vh) { return {(double2*)p, Vh}; }
template <>
__host__ __device__ inline Field<QCD_PREC_SINGLE> make_field<QCD_PREC_SINGLE>(void* p, int Vh) { return {(float2*)p, Vh}; }
template <>
__host__ __device__ inline Field<QCD_PREC_HALF> make_field<QCD_PREC_HALF>(void* p, int Vh) { return {(uint4*)p, Vh}; }
template <>
__host__ __device__ inline Field<QCD_PREC_DF64> make_field<QCD_PREC_DF64>(void* p, int Vh) { return {(float4*)p, Vh}; }

template <int PREC, int RECON>
__host__ __device__ inline Links<PREC, RECON> make_links(const void* p, int Vh);
template <>
__host__ __device__ inline Links<QCD_PREC_DOUBLE, 18> make_links<QCD_PREC_DOUBLE, 18>(const void* p, int Vh) { return {(const double2*)p, Vh}; }
template <>
__host__ __device__ inline Links<QCD_PREC_SINGLE, 18> make_links<QCD_PREC_SINGLE, 18>(const void* p, int Vh) { return {(const float2*)p, Vh}; }
template <>
__host__ __device__ inline Links<QCD_PREC_SINGLE, 12> make_links<QCD_PREC_SINGLE, 12>(const void* p, int Vh) { return {(const float4*)p, Vh}; }
template <>
__host__ __device__ inline Links<QCD_PREC_DF64, 18> make_links<QCD_PREC_DF64, 18>(const void* p, int Vh) { return {(const float4*)p, Vh}; }
template <>
__host__ __device__ inline Links<QCD_PREC_HALF, 12> make_links<QCD_PREC_HALF, 12>(const void* p, int Vh) {
  return {(const uint4*)p, (const uint2*)((const uint4*)p + 8 * (size_t)Vh), Vh};
}

// Two threads per site when one thread per site leaves most of the GPU idle (below about 2
// blocks of 128 sites per SM, e.g. 16^4 = 32768 sites per parity on 152 SMs) — for the FP32 and
// FP16 operators only: measured on GB300, the FP64 operator is bound by the FP64 pipe and the
// pair split (extra selects and shuffles) makes it slower at every size from 8^4 to 24^4.
inline int threads_per_site(int prec, long long Vh) {
  if (prec == QCD_PREC_DOUBLE) return 1;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return Vh < (long long)sms * kBlock * 2 ? 2 : 1;
}

// Field r of a multi-RHS packed field (nrhs fields back to back).
template <class FieldT>
__device__ __forceinline__ FieldT field_at(const FieldT& f, int r) {
  FieldT o = f;
  o.p = f.p + (size_t)r * FieldT::kElemsPerSite * f.Vh;
  return o;
}

template <typename T>
__device__ __forceinline__ void scale(su3<T>& U, T s) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) { U.e[a][b].re *= s; U.e[a][b].im *= s; }
}

// Grid size for the site kernels: enough blocks to cover V/2 sites, capped so that the
// per-block reduction partials fit (grid-stride loop beyond that).
inline int site_grid(long long Vh) {
  long long b = (Vh + kBlock - 1) / kBlock;
  const long long cap = kMaxPartials;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// Grid for kernels that end in a grid-wide reduction: at most one wave of resident blocks
// (SMs x blocks per SM of `kernel`), each looping over sites. Every block pays the end-of-block
// barrier and partial write once per launch instead of once per wave of blocks.
template <class KernelT>
inline int one_wave_grid(long long Vh, KernelT kernel, int tps = 1) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return site_grid(Vh);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  const long long wave = (long long)sms * per_sm;
  const long long need = (Vh * tps + kBlock - 1) / kBlock;
  long long g = need < wave ? need : wave;
  if (g > kMaxPartials) g = kMaxPartials;
  return (int)(g > 0 ? g : 1);
}

}  // namespace qcd
