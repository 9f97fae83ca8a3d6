// Stand-alone operator launches: the half-lattice hop, its multi-RHS form, and the even-site
// normal operator m^2 - D_eo D_oe (the paper's fmv / fmtv pair of §4, applied once).
#include "dslash.cuh"

namespace qcd {

// out_e = m^2 in_e - acc  (acc = D_eo tmp_o)
template <class FieldT>
struct EpiMdagm {
  static constexpr int NV = 0;
  FieldT in, out;
  double m2;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class T>
  __device__ __forceinline__ void site(int k, cvec3<T>& acc, double*) const {
    cvec3<T> v = in.load(k);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v.c[a].re = fma(T(m2), v.c[a].re, -acc.c[a].re);
      v.c[a].im = fma(T(m2), v.c[a].im, -acc.c[a].im);
    }
    out.store(k, v);
  }
  __device__ __forceinline__ void finish(double*) const {}
};

template <int PREC, int RECON>
static int dslash_typed(const qcd_lattice* lat, void* out, const void* in, int out_par, cudaStream_t st) {
  const Geom g = make_geom(lat);
  auto U = make_links<PREC, RECON>(lat->links[PREC].ptr, g.Vh);
  auto fin = make_field<PREC>(const_cast<void*>(in), g.Vh);
  EpiStore<Field<PREC>> epi{make_field<PREC>(out, g.Vh)};
  dslash_kernel<<<site_grid(g.Vh), kBlock, 0, st>>>(g, U, fin, out_par, epi);
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

template <int PREC, int RECON>
static int mdagm_typed(const qcd_lattice* lat, void* out, const void* in, double mass, void* tmp, cudaStream_t st) {
  const Geom g = make_geom(lat);
  auto U = make_links<PREC, RECON>(lat->links[PREC].ptr, g.Vh);
  auto fin = make_field<PREC>(const_cast<void*>(in), g.Vh);
  auto ftmp = make_field<PREC>(tmp, g.Vh);
  const int grid = site_grid(g.Vh);
  dslash_kernel<<<grid, kBlock, 0, st>>>(g, U, fin, QCD_ODD, EpiStore<Field<PREC>>{ftmp});
  QCD_CUDA(cudaGetLastError());
  EpiMdagm<Field<PREC>> epi{fin, make_field<PREC>(out, g.Vh), mass * mass};
  dslash_kernel<<<grid, kBlock, 0, st>>>(g, U, ftmp, QCD_EVEN, epi);
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

int launch_dslash(const qcd_lattice* lat, void* out, const void* in, int out_par, int prec, cudaStream_t st) {
  const int recon = lat->links[prec].recon;
#define CALL_DSLASH(P, R) dslash_typed<P, R>(lat, out, in, out_par, st)
  if (prec == QCD_PREC_DOUBLE && recon == 18) return CALL_DSLASH(QCD_PREC_DOUBLE, 18);
  if (prec == QCD_PREC_SINGLE && recon == 18) return CALL_DSLASH(QCD_PREC_SINGLE, 18);
  if (prec == QCD_PREC_SINGLE && recon == 12) return CALL_DSLASH(QCD_PREC_SINGLE, 12);
  if (prec == QCD_PREC_HALF && recon == 12) return CALL_DSLASH(QCD_PREC_HALF, 12);
#undef CALL_DSLASH
  return QCD_ERR_UNSUPPORTED;
}

int launch_mdagm(const qcd_lattice* lat, void* out, const void* in, double mass, int prec, void* tmp, cudaStream_t st) {
  const int recon = lat->links[prec].recon;
#define CALL_MDAGM(P, R) mdagm_typed<P, R>(lat, out, in, mass, tmp, st)
  if (prec == QCD_PREC_DOUBLE && recon == 18) return CALL_MDAGM(QCD_PREC_DOUBLE, 18);
  if (prec == QCD_PREC_SINGLE && recon == 18) return CALL_MDAGM(QCD_PREC_SINGLE, 18);
  if (prec == QCD_PREC_SINGLE && recon == 12) return CALL_MDAGM(QCD_PREC_SINGLE, 12);
  if (prec == QCD_PREC_HALF && recon == 12) return CALL_MDAGM(QCD_PREC_HALF, 12);
#undef CALL_MDAGM
  return QCD_ERR_UNSUPPORTED;
}

// ------------------------------------------------------------------------------------------
// Multi-RHS hop: each thread owns one output site and applies every loaded link to RB
// right-hand sides before moving on, so a link is read once per RB vectors.
// ------------------------------------------------------------------------------------------
template <class LinksT, class FieldT, int RB>
__global__ void __launch_bounds__(kBlock) dslash_mrhs_kernel(Geom g, LinksT U, FieldT in, FieldT out, int nrhs,
                                                             int out_par) {
  using T = typename LinksT::T;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
    const Site s = site_of(g, k, out_par);
    int fwd[4], bwd[4];
    neighbours(g, s, fwd, bwd);
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
      cvec3<T> acc[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) zero(acc[j]);
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        su3<T> Uf = U.load(out_par, mu, k);
        if constexpr (!LinksT::kFolded) scale(Uf, T(0.5f * fwd_sign(g, s, mu)));
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (r0 + j < nrhs) mul_add(acc[j], Uf, field_at(in, r0 + j).load(fwd[mu]));
        su3<T> Ub = U.load(1 - out_par, mu, bwd[mu]);
        if constexpr (!LinksT::kFolded) scale(Ub, T(0.5f * bwd_sign(g, s, mu)));
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (r0 + j < nrhs) adj_mul_sub(acc[j], Ub, field_at(in, r0 + j).load(bwd[mu]));
      }
#pragma unroll
      for (int j = 0; j < RB; ++j)
        if (r0 + j < nrhs) field_at(out, r0 + j).store(k, acc[j]);
    }
  }
}

template <int PREC, int RECON>
static int mrhs_typed(const qcd_lattice* lat, void* out, const void* in, int nrhs, int out_par, int rb,
                      cudaStream_t st) {
  const Geom g = make_geom(lat);
  auto U = make_links<PREC, RECON>(lat->links[PREC].ptr, g.Vh);
  auto fin = make_field<PREC>(const_cast<void*>(in), g.Vh);
  auto fout = make_field<PREC>(out, g.Vh);
  const int grid = site_grid(g.Vh);
  switch (rb) {
    case 1: dslash_mrhs_kernel<decltype(U), Field<PREC>, 1><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break;
    case 2: dslash_mrhs_kernel<decltype(U), Field<PREC>, 2><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break;
    case 4: dslash_mrhs_kernel<decltype(U), Field<PREC>, 4><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break;
    case 8: dslash_mrhs_kernel<decltype(U), Field<PREC>, 8><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break;
    case 16: dslash_mrhs_kernel<decltype(U), Field<PREC>, 16><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break;
    default: return QCD_ERR_INVALID_ARG;
  }
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

int launch_dslash_mrhs(const qcd_lattice* lat, void* out, const void* in, int nrhs, int out_par, int prec, int rb,
                       cudaStream_t st) {
  const int recon = lat->links[prec].recon;
#define CALL_MRHS(P, R) mrhs_typed<P, R>(lat, out, in, nrhs, out_par, rb, st)
  if (prec == QCD_PREC_DOUBLE && recon == 18) return CALL_MRHS(QCD_PREC_DOUBLE, 18);
  if (prec == QCD_PREC_SINGLE && recon == 18) return CALL_MRHS(QCD_PREC_SINGLE, 18);
  if (prec == QCD_PREC_SINGLE && recon == 12) return CALL_MRHS(QCD_PREC_SINGLE, 12);
  if (prec == QCD_PREC_HALF && recon == 12) return CALL_MRHS(QCD_PREC_HALF, 12);
#undef CALL_MRHS
  return QCD_ERR_UNSUPPORTED;
}

}  // namespace qcd
