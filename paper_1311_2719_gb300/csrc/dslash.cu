// Stand-alone operator launches: the half-lattice hop, its multi-RHS form, and the even-site
// normal operator m^2 - D_eo D_oe (the paper's fmv / fmtv pair of §4, applied once).
#include "dslash.cuh"

namespace qcd {

// out_e = m^2 in_e - acc  (acc = D_eo tmp_o)
template <class FieldT>
struct EpiMdagm {
  static constexpr int NV = 0;
  static constexpr bool kPrefetch = false;
  FieldT in, out;
  double m2;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class T, class A>
  __device__ __forceinline__ void site(int k, cvec3<T>& acc, A*) const {
    cvec3<T> v = in.load(k);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v.c[a].re = fma(T(m2), v.c[a].re, -acc.c[a].re);
      v.c[a].im = fma(T(m2), v.c[a].im, -acc.c[a].im);
    }
    out.store(k, v);
  }
  template <class A>
  __device__ __forceinline__ void finish(A*) const {}
};

template <int PREC, int RECON>
static int dslash_typed(const qcd_lattice* lat, void* out, const void* in, int out_par, cudaStream_t st) {
  const Geom g = make_geom(lat);
  auto U = make_links<PREC, RECON>(lat->links[PREC].ptr, g.Vh);
  U.stream = stream_links(PREC, RECON, g.Vh);
  auto fin = make_field<PREC>(const_cast<void*>(in), g.Vh);
  EpiStore<Field<PREC>> epi{make_field<PREC>(out, g.Vh)};
  if (threads_per_site(PREC, g.Vh) == 2)
    dslash_kernel<decltype(U), Field<PREC>, EpiStore<Field<PREC>>, 2><<<site_grid(2ll * g.Vh), kBlock, 0, st>>>(g, U, fin, out_par, epi);
  else
    dslash_kernel<<<site_grid(g.Vh), kBlock, 0, st>>>(g, U, fin, out_par, epi);
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

template <int PREC, int RECON>
static int mdagm_typed(const qcd_lattice* lat, void* out, const void* in, double mass, void* tmp, cudaStream_t st) {
  const Geom g = make_geom(lat);
  auto U = make_links<PREC, RECON>(lat->links[PREC].ptr, g.Vh);
  U.stream = stream_links(PREC, RECON, g.Vh);
  auto fin = make_field<PREC>(const_cast<void*>(in), g.Vh);
  auto ftmp = make_field<PREC>(tmp, g.Vh);
  EpiMdagm<Field<PREC>> epi{fin, make_field<PREC>(out, g.Vh), mass * mass};
  if (threads_per_site(PREC, g.Vh) == 2) {
    const int grid = site_grid(2ll * g.Vh);
    dslash_kernel<decltype(U), Field<PREC>, EpiStore<Field<PREC>>, 2><<<grid, kBlock, 0, st>>>(g, U, fin, QCD_ODD, EpiStore<Field<PREC>>{ftmp});
    dslash_kernel<decltype(U), Field<PREC>, EpiMdagm<Field<PREC>>, 2><<<grid, kBlock, 0, st>>>(g, U, ftmp, QCD_EVEN, epi);
  } else {
    const int grid = site_grid(g.Vh);
    dslash_kernel<<<grid, kBlock, 0, st>>>(g, U, fin, QCD_ODD, EpiStore<Field<PREC>>{ftmp});
    dslash_kernel<<<grid, kBlock, 0, st>>>(g, U, ftmp, QCD_EVEN, epi);
  }
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
  if (prec == QCD_PREC_DF64 && recon == 18) return CALL_DSLASH(QCD_PREC_DF64, 18);
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
  if (prec == QCD_PREC_DF64 && recon == 18) return CALL_MDAGM(QCD_PREC_DF64, 18);
#undef CALL_MDAGM
  return QCD_ERR_UNSUPPORTED;
}

}  // namespace qcd
