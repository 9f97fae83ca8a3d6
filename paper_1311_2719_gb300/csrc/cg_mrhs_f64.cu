// Multi-RHS CG instantiations for one precision (split for parallel compilation).
#include "cg_mrhs.cuh"

namespace qcd {
template int mrhs_typed<QCD_PREC_DOUBLE, 18>(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*, qcd_solve_info*, cudaStream_t);
}  // namespace qcd
