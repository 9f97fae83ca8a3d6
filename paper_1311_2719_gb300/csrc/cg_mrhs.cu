// Multi-RHS CG entry: dispatch to the per-precision instantiations (cg_mrhs_*.cu).
#include "cg_mrhs.cuh"

namespace qcd {

extern template int mrhs_typed<QCD_PREC_DOUBLE, 18>(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*, qcd_solve_info*, cudaStream_t);
extern template int mrhs_typed<QCD_PREC_SINGLE, 18>(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*, qcd_solve_info*, cudaStream_t);
extern template int mrhs_typed<QCD_PREC_SINGLE, 12>(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*, qcd_solve_info*, cudaStream_t);
extern template int mrhs_typed<QCD_PREC_HALF, 12>(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*, qcd_solve_info*, cudaStream_t);
extern template int mrhs_typed<QCD_PREC_DF64, 18>(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*, qcd_solve_info*, cudaStream_t);

int run_cg_mrhs(qcd_lattice* lat, int R, void* x, const void* b, double mass, double tol, int max_iter,
                const qcd_solver_opts& o, void* ws, void* y, qcd_solve_info* info, cudaStream_t st) {
  const int prec = o.prec_inner;
  const int recon = lat->links[prec].recon;
  if (prec == QCD_PREC_DOUBLE && recon == 18) return mrhs_typed<QCD_PREC_DOUBLE, 18>(lat, R, x, b, mass, tol, max_iter, o, ws, y, info, st);
  if (prec == QCD_PREC_SINGLE && recon == 18) return mrhs_typed<QCD_PREC_SINGLE, 18>(lat, R, x, b, mass, tol, max_iter, o, ws, y, info, st);
  if (prec == QCD_PREC_SINGLE && recon == 12) return mrhs_typed<QCD_PREC_SINGLE, 12>(lat, R, x, b, mass, tol, max_iter, o, ws, y, info, st);
  if (prec == QCD_PREC_HALF && recon == 12) return mrhs_typed<QCD_PREC_HALF, 12>(lat, R, x, b, mass, tol, max_iter, o, ws, y, info, st);
  if (prec == QCD_PREC_DF64 && recon == 18) return mrhs_typed<QCD_PREC_DF64, 18>(lat, R, x, b, mass, tol, max_iter, o, ws, y, info, st);
  return QCD_ERR_UNSUPPORTED;
}

}  // namespace qcd
