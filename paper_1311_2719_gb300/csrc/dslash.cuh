// The staggered hopping term on one output parity (the paper's matrix-vector routine, §3) and
// the generic site kernel that fuses a caller-chosen epilogue onto it (the CG vector algebra of
// the paper's congrad, §4).
#pragma once

#include "qcd_internal.cuh"

namespace qcd {

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
    const cvec3<T> xf = in.load(fwd[mu]);
    if constexpr (LinksT::kFolded) {
      mul_add(acc, Uf, xf);
    } else {
      axpy(acc, T(0.5f * fwd_sign(g, s, mu)), mul(Uf, xf));
    }
    const su3<T> Ub = U.load(1 - out_par, mu, bwd[mu]);
    const cvec3<T> xb = in.load(bwd[mu]);
    if constexpr (LinksT::kFolded) {
      adj_mul_sub(acc, Ub, xb);
    } else {
      axpy(acc, T(-0.5f * bwd_sign(g, s, mu)), adj_mul(Ub, xb));
    }
  }
  return acc;
}

// Epilogue interface:
//   static constexpr int NV;                        number of FP64 sums reduced over the grid
//   bool skip() const;                              true -> whole kernel returns at once
//   void site(int k, cvec3<T>& acc, double* red);   consume the hop result of site k
//   void finish(double* red);                       grid reduction + scalar update (NV > 0)
template <class LinksT, class FieldT, class Epi>
__global__ void __launch_bounds__(kBlock) dslash_kernel(Geom g, LinksT U, FieldT in, int out_par, Epi epi) {
  if (epi.skip()) return;
  double red[Epi::NV > 0 ? Epi::NV : 1];
#pragma unroll
  for (int j = 0; j < (Epi::NV > 0 ? Epi::NV : 1); ++j) red[j] = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
    auto acc = hop(g, U, in, out_par, k);
    epi.site(k, acc, red);
  }
  if constexpr (Epi::NV > 0) epi.finish(red);
}

// Plain store epilogue.
template <class FieldT>
struct EpiStore {
  static constexpr int NV = 0;
  FieldT out;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class T>
  __device__ __forceinline__ void site(int k, cvec3<T>& acc, double*) const {
    out.store(k, acc);
  }
  __device__ __forceinline__ void finish(double*) const {}
};

template <int PREC>
__host__ __device__ inline Field<PREC> make_field(void* p, int Vh);
template <>
__host__ __device__ inline Field<QCD_PREC_DOUBLE> make_field<QCD_PREC_DOUBLE>(void* p, int Vh) { return {(double2*)p, Vh}; }
template <>
__host__ __device__ inline Field<QCD_PREC_SINGLE> make_field<QCD_PREC_SINGLE>(void* p, int Vh) { return {(float2*)p, Vh}; }
template <>
__host__ __device__ inline Field<QCD_PREC_HALF> make_field<QCD_PREC_HALF>(void* p, int Vh) { return {(uint4*)p, Vh}; }

template <int PREC, int RECON>
__host__ __device__ inline Links<PREC, RECON> make_links(const void* p, int Vh);
template <>
__host__ __device__ inline Links<QCD_PREC_DOUBLE, 18> make_links<QCD_PREC_DOUBLE, 18>(const void* p, int Vh) { return {(const double2*)p, Vh}; }
template <>
__host__ __device__ inline Links<QCD_PREC_SINGLE, 18> make_links<QCD_PREC_SINGLE, 18>(const void* p, int Vh) { return {(const float2*)p, Vh}; }
template <>
__host__ __device__ inline Links<QCD_PREC_SINGLE, 12> make_links<QCD_PREC_SINGLE, 12>(const void* p, int Vh) { return {(const float4*)p, Vh}; }
template <>
__host__ __device__ inline Links<QCD_PREC_HALF, 12> make_links<QCD_PREC_HALF, 12>(const void* p, int Vh) {
  return {(const uint4*)p, (const uint2*)((const uint4*)p + 8 * (size_t)Vh), Vh};
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

}  // namespace qcd
