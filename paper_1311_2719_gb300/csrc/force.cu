// Staggered fermion force: the derivative of the even-site pseudofermion action
// S = phi^dagger (m^2 - D_eo D_oe)^-1 phi with respect to the gauge links, computed from the two
// fields the CG returns (the paper's congrad, §4: x on the even sites and "the solution on the
// second half lattice" y = D_oe x on the odd sites), for the molecular-dynamics program (§2) that
// calls it.
//
// G_mu(n) is the traceless Hermitian matrix with dS = eps tr(H G_mu(n)) under
// U_mu(n) -> exp(i eps H) U_mu(n). With c = eta_mu(n) zeta_mu(n) / 2 (the link's coefficient in D),
//   n even:  W = c a b^dagger,  a = U_mu(n) y(n+mu),  b = x(n)
//   n odd :  W = c a b^dagger,  a = y(n),             b = U_mu(n) x(n+mu)
//   G_mu(n) = i (W - W^dagger) minus its trace / 3
// (dS = 2 Re x^dagger dD_eo y; link U_mu(n) enters D_eo through the forward hop of an even n or the
// backward hop of n + mu for an odd n).
//
// Layout: canonical links and force complex128[V][4][3][3], x and y complex128[V][3]. One thread
// per link, mu fastest, so that a warp reads and writes 32 consecutive 144-byte link matrices.
#include "qcd_internal.cuh"

namespace qcd {

__global__ void __launch_bounds__(kBlock) force_kernel(Geom g, const double2* __restrict__ U,
                                                      const double2* __restrict__ x, const double2* __restrict__ y,
                                                      double2* __restrict__ G) {
  const long long nlinks = 8ll * g.Vh;  // 4 V
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nlinks;
       t += (long long)gridDim.x * blockDim.x) {
    const int lex = (int)(t >> 2), mu = (int)(t & 3);
    int c[4];
    {
      int r = lex;
      const int r0 = fdiv(r, g.d0);
      c[0] = r - r0 * g.L0;
      const int r1 = fdiv(r0, g.d1);
      c[1] = r0 - r1 * g.L1;
      c[3] = fdiv(r1, g.d2);
      c[2] = r1 - c[3] * g.L2;
    }
    const int L[4] = {g.L0, g.L1, g.L2, g.L3};
    const int st[4] = {1, g.L0, g.L0 * g.L1, g.L0 * g.L1 * g.L2};
    const int up = c[mu] == L[mu] - 1 ? lex - (L[mu] - 1) * st[mu] : lex + st[mu];
    int e = 0;
    for (int nu = 0; nu < mu; ++nu) e += c[nu];
    double coef = (e & 1) ? -0.5 : 0.5;
    if (mu == 3 && c[3] == g.L3 - 1) coef *= (double)g.tbc;
    const bool even = ((c[0] + c[1] + c[2] + c[3]) & 1) == 0;

    su3<double> Ul;
    const double2* ub = U + (size_t)t * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double2 d = ub[k];
      Ul.e[k / 3][k % 3] = {d.x, d.y};
    }
    // a b^dagger with (a, b) = (U y(n+mu), x(n)) on even sites, (y(n), U x(n+mu)) on odd sites
    const double2* own = (even ? x : y) + (size_t)lex * 3;
    const double2* nbr = (even ? y : x) + (size_t)up * 3;
    cvec3<double> vo, vn;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 o = own[a], n = nbr[a];
      vo.c[a] = {o.x, o.y};
      vn.c[a] = {n.x, n.y};
    }
    const cvec3<double> un = mul(Ul, vn);
    const cvec3<double>& av = even ? un : vo;
    cvec3<double> bv = even ? vo : un;
#pragma unroll
    for (int b = 0; b < 3; ++b) {  // the real coefficient goes on b (3 entries instead of 9)
      bv.c[b].re *= coef;
      bv.c[b].im *= coef;
    }
    cplx<double> W[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {  // a_a conj(b_b)
        W[a][b].re = fma(av.c[a].re, bv.c[b].re, av.c[a].im * bv.c[b].im);
        W[a][b].im = fma(av.c[a].im, bv.c[b].re, -av.c[a].re * bv.c[b].im);
      }
    // G = i (W - W^dagger): G_ab = i (W_ab - conj(W_ba)); the diagonal is real, -2 Im W_aa
    double diag[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) diag[a] = -2.0 * W[a][a].im;
    const double tr3 = (diag[0] + diag[1] + diag[2]) / 3.0;
    double2* gb = G + (size_t)t * 9;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (a == b) {
          gb[3 * a + b] = make_double2(diag[a] - tr3, 0.0);
        } else {
          // i (W_ab - conj(W_ba)) = i ((W_ab.re - W_ba.re) + i (W_ab.im + W_ba.im))
          gb[3 * a + b] = make_double2(-(W[a][b].im + W[b][a].im), W[a][b].re - W[b][a].re);
        }
      }
  }
}

int launch_fermion_force(const qcd_lattice* lat, void* force, const void* links, const void* x, const void* y,
                         cudaStream_t st) {
  const Geom g = make_geom(lat);
  const long long nlinks = 4ll * lat->V;
  long long blocks = (nlinks + kBlock - 1) / kBlock;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_kernel, kBlock, 0) == cudaSuccess && sms > 0 &&
      per_sm > 0 && blocks > (long long)sms * per_sm)
    blocks = (long long)sms * per_sm;
  force_kernel<<<(unsigned)blocks, kBlock, 0, st>>>(g, (const double2*)links, (const double2*)x, (const double2*)y,
                                                   (double2*)force);
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

}  // namespace qcd
