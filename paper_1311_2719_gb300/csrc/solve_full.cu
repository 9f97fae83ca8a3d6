// Full-system solve M x = b, M = m + D on both parities, by even-odd reduction onto the solver of
// cg.cu: (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o, then x_o = (b_o - D_oe x_e) / m
// (the odd half follows from the even solution and the paper's "solution on the second half
// lattice", y = D_oe x_e). The full FP64 residual |b - M x| / |b| is recomputed at the end.
#include <cmath>

#include "cg_common.cuh"

namespace qcd {

size_t cg_workspace_bytes(const qcd_lattice*, int, int);
int run_cg(qcd_lattice*, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*,
           qcd_solve_info*, cudaStream_t);
int launch_pack_field(const qcd_lattice*, void*, const void*, int, int, cudaStream_t);

// b'_e = m b_e - D_eo b_o, written into a canonical field (even sites); reduces |b'|^2 and |b|^2
// (both parities: the thread of even site k also reads the odd site with the same index).
struct EpiSource {
  static constexpr int NV = 2;
  static constexpr bool kPrefetch = false;
  Geom g;
  const double2* b;
  double2* out;
  double m;
  double* partials;
  unsigned* counter;
  double* sums;  // sums[0] = |b'|^2, sums[1] = |b|^2
  __device__ __forceinline__ bool skip() const { return false; }
  template <class A>
  __device__ __forceinline__ void site(int k, cvec3<double>& acc, A* red) const {
    const Site s = site_of(g, k, QCD_EVEN), so = site_of(g, k, QCD_ODD);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 bv = b[(size_t)s.lex * 3 + a], bo = b[(size_t)so.lex * 3 + a];
      const double re = fma(m, bv.x, -acc.c[a].re), im = fma(m, bv.y, -acc.c[a].im);
      out[(size_t)s.lex * 3 + a] = make_double2(re, im);
      red[0] += re * re + im * im;
      red[1] += bv.x * bv.x + bv.y * bv.y + bo.x * bo.x + bo.y * bo.y;
    }
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    const A v[2] = {red[0], red[1]};
    double tot[2];
    if (grid_sum_last_block<2>(v, partials, counter, tot) && threadIdx.x == 0) {
      sums[0] = tot[0];
      sums[1] = tot[1];
    }
  }
};

// |b - m x - D x|^2 and |b|^2 over the sites of one parity (acc = D x from the other parity).
struct EpiFullResidual {
  static constexpr int NV = 2;
  static constexpr bool kPrefetch = false;
  Geom g;
  int par;
  const double2* b;
  const double2* x;
  double m;
  double* partials;
  unsigned* counter;
  double* out;  // out[0] += residual^2, out[1] += |b|^2 (this parity)
  __device__ __forceinline__ bool skip() const { return false; }
  template <class A>
  __device__ __forceinline__ void site(int k, cvec3<double>& acc, A* red) const {
    const Site s = site_of(g, k, par);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 bv = b[(size_t)s.lex * 3 + a], xv = x[(size_t)s.lex * 3 + a];
      const double re = bv.x - fma(m, xv.x, acc.c[a].re), im = bv.y - fma(m, xv.y, acc.c[a].im);
      red[0] += re * re + im * im;
      red[1] += bv.x * bv.x + bv.y * bv.y;
    }
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    const A v[2] = {red[0], red[1]};
    double tot[2];
    if (grid_sum_last_block<2>(v, partials, counter, tot) && threadIdx.x == 0) {
      out[0] += tot[0];
      out[1] += tot[1];
    }
  }
};

// x_o = (b_o - y_o) / m on the odd sites of the canonical fields.
__global__ void __launch_bounds__(kBlock) full_odd_kernel(Geom g, const double2* __restrict__ b,
                                                          const double2* __restrict__ y, double2* __restrict__ x,
                                                          double inv_m) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
    const Site s = site_of(g, k, QCD_ODD);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 bv = b[(size_t)s.lex * 3 + a], yv = y[(size_t)s.lex * 3 + a];
      x[(size_t)s.lex * 3 + a] = make_double2((bv.x - yv.x) * inv_m, (bv.y - yv.y) * inv_m);
    }
  }
}

struct FullWork {
  char* cg;         // the even-odd CG workspace
  double2* src;     // canonical b' (even sites used)
  double2* y;       // canonical y = D_oe x_e
  void* f_even;     // packed FP64 fields
  void* f_odd;
  double* sums;     // [2] residual^2, |b|^2 + counter + partials
  unsigned* counter;
  double* partials;
  size_t total;
};

static FullWork carve_full(const qcd_lattice* lat, int prec, char* base) {
  FullWork w{};
  size_t off = 0;
  auto take = [&](size_t n) { char* p = base ? base + off : nullptr; off += align256(n); return p; };
  w.cg = take(cg_workspace_bytes(lat, prec, 1));
  const size_t canon = (size_t)lat->V * 3 * sizeof(double2);
  w.src = (double2*)take(canon);
  w.y = (double2*)take(canon);
  w.f_even = take(field_bytes(QCD_PREC_DOUBLE, lat->Vh));
  w.f_odd = take(field_bytes(QCD_PREC_DOUBLE, lat->Vh));
  w.sums = (double*)take(4 * sizeof(double));
  w.counter = (unsigned*)take(sizeof(unsigned));
  w.partials = (double*)take(sizeof(double) * kMaxPartials * 2);
  w.total = off;
  return w;
}

size_t full_workspace_bytes(const qcd_lattice* lat, int prec) { return carve_full(lat, prec, nullptr).total; }

int run_solve_full(qcd_lattice* lat, void* x, const void* b, double mass, double tol, int max_iter,
                   const qcd_solver_opts& o, void* ws, qcd_solve_info* info, cudaStream_t st) {
  FullWork w = carve_full(lat, o.prec_inner, (char*)ws);
  const Geom g = make_geom(lat);
  auto U64 = make_links<QCD_PREC_DOUBLE, 18>(lat->links[QCD_PREC_DOUBLE].ptr, g.Vh);
  auto fe = make_field<QCD_PREC_DOUBLE>(w.f_even, g.Vh);
  auto fo = make_field<QCD_PREC_DOUBLE>(w.f_odd, g.Vh);
  const int grid = site_grid(g.Vh);
  // b' = m b_e - D_eo b_o, with |b'| and |b|
  int rc = launch_pack_field(lat, w.f_odd, b, QCD_ODD, QCD_PREC_DOUBLE, st);
  if (rc) return rc;
  QCD_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned), st));
  const int rgrid = one_wave_grid(g.Vh, dslash_kernel<Links<QCD_PREC_DOUBLE, 18>, Field<QCD_PREC_DOUBLE>, EpiFullResidual>);
  dslash_kernel<<<rgrid, kBlock, 0, st>>>(
      g, U64, fo, QCD_EVEN, EpiSource{g, (const double2*)b, w.src, mass, w.partials, w.counter, w.sums + 2});
  QCD_CUDA(cudaGetLastError());
  double nb[2] = {0.0, 0.0};
  QCD_CUDA(cudaMemcpyAsync(nb, w.sums + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  QCD_CUDA(cudaStreamSynchronize(st));
  // The full residual is r_e = (Schur residual) / m, r_o = 0: solve the even system to
  // tol * m |b| / |b'| so that |b - M x| / |b| meets tol.
  double tol_s = tol;
  if (nb[0] > 0.0 && nb[1] > 0.0) tol_s = tol * mass * std::sqrt(nb[1] / nb[0]);
  if (!(tol_s < 1.0)) tol_s = 0.5;
  // even solve (writes x on the even sites, zero on the odd ones) and y = D_oe x_e
  rc = nb[0] > 0.0 ? run_cg(lat, x, w.src, mass, tol_s, max_iter, o, w.cg, w.y, info, st)
                   : run_cg(lat, x, w.src, mass, tol, max_iter, o, w.cg, w.y, info, st);
  if (rc != QCD_OK && rc != QCD_ERR_NOT_CONVERGED) return rc;
  const int cg_status = rc;
  full_odd_kernel<<<grid, kBlock, 0, st>>>(g, (const double2*)b, w.y, (double2*)x, 1.0 / mass);
  // full FP64 residual |b - M x| / |b|
  QCD_CUDA(cudaMemsetAsync(w.sums, 0, 2 * sizeof(double), st));
  if ((rc = launch_pack_field(lat, w.f_even, x, QCD_EVEN, QCD_PREC_DOUBLE, st))) return rc;
  if ((rc = launch_pack_field(lat, w.f_odd, x, QCD_ODD, QCD_PREC_DOUBLE, st))) return rc;
  dslash_kernel<<<rgrid, kBlock, 0, st>>>(
      g, U64, fo, QCD_EVEN,
      EpiFullResidual{g, QCD_EVEN, (const double2*)b, (const double2*)x, mass, w.partials, w.counter, w.sums});
  dslash_kernel<<<rgrid, kBlock, 0, st>>>(
      g, U64, fe, QCD_ODD,
      EpiFullResidual{g, QCD_ODD, (const double2*)b, (const double2*)x, mass, w.partials, w.counter, w.sums});
  QCD_CUDA(cudaGetLastError());
  double h[2] = {0.0, 0.0};
  QCD_CUDA(cudaMemcpyAsync(h, w.sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  QCD_CUDA(cudaStreamSynchronize(st));
  const double rel = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
  int status = cg_status;
  if (!std::isfinite(rel)) status = QCD_ERR_BREAKDOWN;
  else if (status == QCD_OK && !(rel <= tol)) status = QCD_ERR_NOT_CONVERGED;
  if (info) {
    info->true_rel_residual = rel;
    info->kernel_launches += 8;
    info->status = status;
    info->converged = status == QCD_OK;
  }
  return status;
}

}  // namespace qcd
