// Multi-RHS half-lattice operator (qcd_dslash_mrhs): every loaded link applied to RB vectors.
#include "dslash.cuh"

namespace qcd {

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
  constexpr bool wide = PREC == QCD_PREC_DOUBLE || PREC == QCD_PREC_DF64;  // 64-bit accumulators: RB <= 4
  switch (rb) {
    case 1: dslash_mrhs_kernel<decltype(U), Field<PREC>, 1><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break;
    case 2: dslash_mrhs_kernel<decltype(U), Field<PREC>, 2><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break;
    case 4: dslash_mrhs_kernel<decltype(U), Field<PREC>, 4><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break;
    case 8:
      if constexpr (!wide) { dslash_mrhs_kernel<decltype(U), Field<PREC>, 8><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break; }
      [[fallthrough]];
    case 16:
      if constexpr (!wide) { dslash_mrhs_kernel<decltype(U), Field<PREC>, 16><<<grid, kBlock, 0, st>>>(g, U, fin, fout, nrhs, out_par); break; }
      [[fallthrough]];
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
  if (prec == QCD_PREC_DF64 && recon == 18) return CALL_MRHS(QCD_PREC_DF64, 18);
#undef CALL_MRHS
  return QCD_ERR_UNSUPPORTED;
}

}  // namespace qcd
