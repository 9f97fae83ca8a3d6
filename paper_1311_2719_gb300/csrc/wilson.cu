// Wilson fermions (the paper's second program, §2/§6): the hopping term D_W on the full lattice,
// M = 1 - kappa D_W, M^dagger = gamma5 M gamma5, and CGNR (CG on M^dagger M x = M^dagger b) with
// FP64 reliable updates when the recursion runs in FP32.
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

size_t wfield_bytes(int prec, long long V) {
  return prec == QCD_PREC_DOUBLE ? WField<QCD_PREC_DOUBLE>::bytes(V)
                                 : (prec == QCD_PREC_SINGLE ? WField<QCD_PREC_SINGLE>::bytes(V) : 0);
}
size_t wlinks_bytes(int prec, long long V) {
  return prec == QCD_PREC_DOUBLE ? WLinks<QCD_PREC_DOUBLE>::bytes(V)
                                 : (prec == QCD_PREC_SINGLE ? WLinks<QCD_PREC_SINGLE>::bytes(V) : 0);
}

// ---------------------------------------------------------------- geometry (full lattice)
__device__ __forceinline__ void full_site(const Geom& g, int i, int c[4]) {
  int t = i;
  c[0] = t % g.L0; t /= g.L0;
  c[1] = t % g.L1; t /= g.L1;
  c[2] = t % g.L2;
  c[3] = t / g.L2;
}

// ---------------------------------------------------------------- the hopping term at site i
// G5IN: the input field is read as gamma5 psi (spins 2, 3 negated) — used for M^dagger.
template <class LinksT, class FieldT, bool G5IN>
__device__ __forceinline__ spinor<typename LinksT::T> wilson_hop(const Geom& g, const LinksT& U, const FieldT& in, int i) {
  using T = typename LinksT::T;
  int c[4];
  full_site(g, i, c);
  const int L[4] = {g.L0, g.L1, g.L2, g.L3};
  const int st[4] = {1, g.L0, g.L0 * g.L1, g.L0 * g.L1 * g.L2};
  spinor<T> acc;
  zero(acc);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {  // dir 0: forward, (1 - gamma); dir 1: backward, (1 + gamma)
      const int sgn = dir == 0 ? 2 : 0;   // phase code of s: -1 -> 2, +1 -> 0
      const int nb = dir == 0 ? (c[mu] == L[mu] - 1 ? i - (L[mu] - 1) * st[mu] : i + st[mu])
                              : (c[mu] == 0 ? i + (L[mu] - 1) * st[mu] : i - st[mu]);
      spinor<T> psi = in.load(nb);
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
      const su3<T> Ul = U.load(mu, dir == 0 ? i : nb);
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
  }
  return acc;
}

template <class LinksT, class FieldT, bool G5IN, class Epi>
__global__ void __launch_bounds__(kBlock) wilson_kernel(Geom g, int V, LinksT U, FieldT in, Epi epi) {
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

// CGNR K1: t = M p, |t|^2 -> alpha = rr / |t|^2
template <class FieldT>
struct WEpiT {
  static constexpr int NV = 1;
  FieldT p, t;
  double kappa;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return sc->done != kRunning; }
  template <class T, class A>
  __device__ __forceinline__ void site(int i, spinor<T>& acc, A* red) const {
    const spinor<T> v = m_combine<FieldT, false>(p, i, acc, (T)kappa);
    t.store(i, v);
    accum(red[0], norm2(v));
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    double v[1] = {(double)red[0]}, tot[1];
    if (grid_sum_last_block<1>(v, partials, &sc->counter[2], tot) && threadIdx.x == 0) {
      const double alpha = sc->rr / tot[0];
      if (!(tot[0] > 0.0) || !isfinite(alpha)) sc->done = kBreakdown;
      else sc->alpha = alpha;
    }
  }
};

// CGNR K2: s = M^dagger t; x += alpha p; r -= alpha s; |r|^2 -> beta and the exit tests
template <class FieldT, class XFieldT>
struct WEpiUpdate {
  static constexpr int NV = 1;
  FieldT t, p, r;
  XFieldT x;
  double kappa;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return sc->done != kRunning; }
  template <class T, class A>
  __device__ __forceinline__ void site(int i, spinor<T>& acc, A* red) const {
    using TX = typename XFieldT::T;
    const spinor<T> s = m_combine<FieldT, true>(t, i, acc, (T)kappa);
    const T alpha = (T)sc->alpha;
    const spinor<T> pv = p.load(i);
    spinor<T> rv = r.load(i);
    spinor<TX> xv = x.load(i);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        rv.s[q].c[a].re = fma(-alpha, s.s[q].c[a].re, rv.s[q].c[a].re);
        rv.s[q].c[a].im = fma(-alpha, s.s[q].c[a].im, rv.s[q].c[a].im);
        xv.s[q].c[a].re = fma((TX)alpha, (TX)pv.s[q].c[a].re, xv.s[q].c[a].re);
        xv.s[q].c[a].im = fma((TX)alpha, (TX)pv.s[q].c[a].im, xv.s[q].c[a].im);
      }
    r.store(i, rv);
    x.store(i, xv);
    accum(red[0], norm2(rv));
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    double v[1] = {(double)red[0]}, tot[1];
    if (grid_sum_last_block<1>(v, partials, &sc->counter[3], tot) && threadIdx.x == 0) {
      const double rr = tot[0];
      sc->iter += 1;
      sc->since_ru += 1;
      sc->rr_prev = sc->rr;
      sc->rr = rr;
      if (!isfinite(rr)) { sc->done = kBreakdown; return; }
      sc->beta = rr / sc->rr_prev;
      if (rr > sc->rmax2) sc->rmax2 = rr;
      if (rr < sc->delit) sc->done = kConverged;
      else if (sc->iter >= sc->max_iter) sc->done = kMaxIter;
      else if (sc->mixed && (sc->since_ru >= sc->ru_interval || rr < sc->delta2 * sc->rmax2)) sc->done = kReliable;
    }
  }
};

// FP64 residual of the normal equations: res = rhs - M^dagger t (t = M x); r_lo <- res; |res|^2.
// Used at start-up (x = 0: res = rhs), for reliable updates and for the final report.
template <class FieldT, bool FINAL>
struct WEpiResidual {
  static constexpr int NV = 1;
  WField<QCD_PREC_DOUBLE> t, rhs;
  FieldT r_lo;
  double kappa;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return false; }
  template <class A>
  __device__ __forceinline__ void site(int i, spinor<double>& acc, A* red) const {
    using T = typename FieldT::T;
    const spinor<double> s = m_combine<WField<QCD_PREC_DOUBLE>, true>(t, i, acc, kappa);
    const spinor<double> b = rhs.load(i);
    spinor<double> res;
    spinor<T> rl;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        res.s[q].c[a] = {b.s[q].c[a].re - s.s[q].c[a].re, b.s[q].c[a].im - s.s[q].c[a].im};
        rl.s[q].c[a] = {(T)res.s[q].c[a].re, (T)res.s[q].c[a].im};
      }
    if (!FINAL) r_lo.store(i, rl);
    red[0] += norm2(res);
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    double v[1] = {(double)red[0]}, tot[1];
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

// ---------------------------------------------------------------- small streaming kernels
template <class FieldT>
__global__ void __launch_bounds__(kBlock) w_p_kernel(int V, FieldT r, FieldT p, CgScalars* sc, double* partials) {
  using T = typename FieldT::T;
  if (sc->done != kRunning) return;
  const T beta = (T)sc->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const spinor<T> rv = r.load(i);
    spinor<T> pv = p.load(i);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pv.s[q].c[a].re = fma(beta, pv.s[q].c[a].re, rv.s[q].c[a].re);
        pv.s[q].c[a].im = fma(beta, pv.s[q].c[a].im, rv.s[q].c[a].im);
      }
    p.store(i, pv);
  }
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
template <class XFieldT>
__global__ void w_accumulate_kernel(int V, WField<QCD_PREC_DOUBLE> xh, XFieldT xl) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    spinor<double> a = xh.load(i);
    const auto b = xl.load(i);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a.s[q].c[c].re += (double)b.s[q].c[c].re;
        a.s[q].c[c].im += (double)b.s[q].c[c].im;
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
      if constexpr (PREC == QCD_PREC_DOUBLE) ((double2*)out)[((size_t)mu * 9 + e) * V + i] = make_double2(z * d.x, z * d.y);
      else ((float2*)out)[((size_t)mu * 9 + e) * V + i] = make_float2((float)(z * d.x), (float)(z * d.y));
    }
  }
}

// ---------------------------------------------------------------- host side
struct WWork {
  CgScalars* sc;
  double* partials;
  void *rhs, *x_hi, *t64;  // FP64
  void *r, *p, *t;         // inner precision
  void* x_lo;              // inner precision (aliases x_hi in FP64)
  size_t total;
};

static WWork w_carve(long long V, int prec, char* base) {
  WWork w{};
  size_t off = 0;
  auto take = [&](size_t n) { void* q = base ? base + off : nullptr; off += align256(n); return q; };
  w.sc = (CgScalars*)take(sizeof(CgScalars));
  w.partials = (double*)take(sizeof(double) * kMaxPartials * 2);
  const size_t f64 = wfield_bytes(QCD_PREC_DOUBLE, V), fin = wfield_bytes(prec, V);
  w.rhs = take(f64);
  w.x_hi = take(f64);
  w.t64 = take(f64);
  w.r = take(fin);
  w.p = take(fin);
  w.t = take(fin);
  w.x_lo = prec == QCD_PREC_DOUBLE ? w.x_hi : take(fin);
  w.total = off;
  return w;
}

size_t wilson_workspace_bytes(const qcd_lattice* lat, int prec) { return w_carve(lat->V, prec, nullptr).total; }

template <int PREC>
static WField<PREC> wf(void* p, int V) {
  return {(typename std::conditional<PREC == QCD_PREC_DOUBLE, double2, float4>::type*)p, V};
}
template <int PREC>
static WLinks<PREC> wl(const void* p, int V) {
  return {(const typename std::conditional<PREC == QCD_PREC_DOUBLE, double2, float2>::type*)p, V};
}

int launch_wilson_pack_links(const qcd_lattice* lat, const void* canon, void* out, int prec, cudaStream_t st) {
  const Geom g = make_geom(lat);
  const int V = (int)lat->V;
  const int grid = (int)std::min<long long>((4ll * V + 255) / 256, 152 * 64);
  if (prec == QCD_PREC_DOUBLE) w_pack_links_kernel<QCD_PREC_DOUBLE><<<grid, 256, 0, st>>>(g, V, (const double2*)canon, out);
  else if (prec == QCD_PREC_SINGLE) w_pack_links_kernel<QCD_PREC_SINGLE><<<grid, 256, 0, st>>>(g, V, (const double2*)canon, out);
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
  return QCD_ERR_UNSUPPORTED;
}

template <int PREC>
static int wilson_cgnr_typed(qcd_lattice* lat, void* x, const void* b, double kappa, double tol, int max_iter,
                             const qcd_solver_opts& o, void* ws, qcd_solve_info* info, cudaStream_t st) {
  using FT = WField<PREC>;
  using F64 = WField<QCD_PREC_DOUBLE>;
  const Geom g = make_geom(lat);
  const int V = (int)lat->V;
  const bool mixed = PREC != QCD_PREC_DOUBLE;
  WWork w = w_carve(V, PREC, (char*)ws);
  auto U = wl<PREC>(lat->wilson_links[PREC], V);
  auto U64 = wl<QCD_PREC_DOUBLE>(lat->wilson_links[QCD_PREC_DOUBLE], V);
  FT r = wf<PREC>(w.r, V), p = wf<PREC>(w.p, V), t = wf<PREC>(w.t, V), xl = wf<PREC>(w.x_lo, V);
  F64 rhs = wf<QCD_PREC_DOUBLE>(w.rhs, V), xh = wf<QCD_PREC_DOUBLE>(w.x_hi, V), t64 = wf<QCD_PREC_DOUBLE>(w.t64, V);
  const int grid = one_wave_grid(V, wilson_kernel<WLinks<PREC>, FT, true, WEpiUpdate<FT, FT>>);
  long long launches = 0;

  CgScalars h{};
  h.tol2 = tol * tol;
  h.max_iter = max_iter;
  h.ru_interval = o.reliable_interval > 0 ? o.reliable_interval : 100;
  h.delta2 = o.reliable_delta * o.reliable_delta;
  h.mixed = mixed ? 1 : 0;
  QCD_CUDA(cudaMemcpyAsync(w.sc, &h, sizeof(CgScalars), cudaMemcpyHostToDevice, st));
  // rhs = M^dagger b (FP64), x = 0, p = 0, r = rhs (the residual epilogue with t = b: rhs - M^dagger(0))
  int rc = launch_wilson_pack(lat, w.t64, b, QCD_PREC_DOUBLE, false, st);
  if (rc) return rc;
  wilson_kernel<WLinks<QCD_PREC_DOUBLE>, F64, true><<<grid, kBlock, 0, st>>>(g, V, U64, t64, WApplyM<F64, true>{t64, rhs, kappa});
  w_zero_kernel<<<grid, kBlock, 0, st>>>(V, xh);
  if (mixed) w_zero_kernel<<<grid, kBlock, 0, st>>>(V, xl);
  w_zero_kernel<<<grid, kBlock, 0, st>>>(V, p);
  w_zero_kernel<<<grid, kBlock, 0, st>>>(V, t64);
  // r = rhs - M^dagger M x with x = 0: the residual kernel on t64 = 0 gives rhs; sets rr, delit
  wilson_kernel<WLinks<QCD_PREC_DOUBLE>, F64, true><<<grid, kBlock, 0, st>>>(
      g, V, U64, t64, WEpiResidual<FT, false>{t64, rhs, r, kappa, w.sc, w.partials});
  QCD_CUDA(cudaGetLastError());
  launches += 6 + (mixed ? 1 : 0);
  QCD_CUDA(cudaMemcpyAsync(&h, w.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
  QCD_CUDA(cudaStreamSynchronize(st));
  const double rhs2 = h.res2;
  h.delit = tol * tol * rhs2;
  h.rr = h.rr_prev = h.rmax2 = rhs2;
  h.beta = 0.0;
  h.iter = 0;
  h.ru_count = 0;
  h.done = !std::isfinite(rhs2) ? kBreakdown : (rhs2 == 0.0 ? kTrueConverged : kRunning);
  QCD_CUDA(cudaMemcpyAsync(w.sc, &h, sizeof(CgScalars), cudaMemcpyHostToDevice, st));

  auto true_residual = [&](bool final_report) -> int {
    // x_hi += x_lo; t64 = M x_hi; res = rhs - M^dagger t64
    if (mixed) w_accumulate_kernel<<<grid, kBlock, 0, st>>>(V, xh, xl);
    wilson_kernel<WLinks<QCD_PREC_DOUBLE>, F64, false><<<grid, kBlock, 0, st>>>(g, V, U64, xh, WApplyM<F64, false>{xh, t64, kappa});
    if (final_report)
      wilson_kernel<WLinks<QCD_PREC_DOUBLE>, F64, true><<<grid, kBlock, 0, st>>>(
          g, V, U64, t64, WEpiResidual<FT, true>{t64, rhs, r, kappa, w.sc, w.partials});
    else
      wilson_kernel<WLinks<QCD_PREC_DOUBLE>, F64, true><<<grid, kBlock, 0, st>>>(
          g, V, U64, t64, WEpiResidual<FT, false>{t64, rhs, r, kappa, w.sc, w.partials});
    launches += mixed ? 3 : 2;
    QCD_CUDA(cudaGetLastError());
    return QCD_OK;
  };

  const int k = o.check_interval > 0 ? o.check_interval : 8;
  int status = QCD_OK;
  while (true) {
    if (h.done == kBreakdown) { status = QCD_ERR_BREAKDOWN; break; }
    if (h.done == kMaxIter) { status = QCD_ERR_NOT_CONVERGED; break; }
    if (h.done == kTrueConverged) break;
    if (h.done == kConverged || (mixed && h.done == kReliable)) {
      if ((rc = true_residual(false))) return rc;
    } else {
      for (int i = 0; i < k; ++i) {
        w_p_kernel<<<grid, kBlock, 0, st>>>(V, r, p, w.sc, w.partials);
        wilson_kernel<WLinks<PREC>, FT, false><<<grid, kBlock, 0, st>>>(g, V, U, p, WEpiT<FT>{p, t, kappa, w.sc, w.partials});
        wilson_kernel<WLinks<PREC>, FT, true><<<grid, kBlock, 0, st>>>(
            g, V, U, t, WEpiUpdate<FT, FT>{t, p, r, xl, kappa, w.sc, w.partials});
        launches += 3;
      }
      QCD_CUDA(cudaGetLastError());
    }
    QCD_CUDA(cudaMemcpyAsync(&h, w.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    QCD_CUDA(cudaStreamSynchronize(st));
  }
  // final: FP64 residual of the normal equations, and x out
  if ((rc = true_residual(true))) return rc;
  if ((rc = launch_wilson_pack(lat, w.x_hi, x, QCD_PREC_DOUBLE, true, st))) return rc;
  QCD_CUDA(cudaMemcpyAsync(&h, w.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
  QCD_CUDA(cudaStreamSynchronize(st));
  const double true_rel = rhs2 > 0 ? std::sqrt(h.res2 / rhs2) : 0.0;
  if (status == QCD_OK && !(true_rel <= tol)) status = QCD_ERR_NOT_CONVERGED;
  if (info) {
    info->iterations = h.iter;
    info->reliable_updates = h.ru_count;
    info->true_rel_residual = true_rel;
    info->iterated_rel_residual = rhs2 > 0 ? std::sqrt(h.rr / rhs2) : 0.0;
    info->converged = status == QCD_OK;
    info->status = status;
    info->kernel_launches = (int)launches;
    info->dslash_launches = 2 * h.iter;
  }
  return status;
}

int run_wilson_cgnr(qcd_lattice* lat, void* x, const void* b, double kappa, double tol, int max_iter,
                    const qcd_solver_opts& o, void* ws, qcd_solve_info* info, cudaStream_t st) {
  if (o.prec_inner == QCD_PREC_DOUBLE) return wilson_cgnr_typed<QCD_PREC_DOUBLE>(lat, x, b, kappa, tol, max_iter, o, ws, info, st);
  if (o.prec_inner == QCD_PREC_SINGLE) return wilson_cgnr_typed<QCD_PREC_SINGLE>(lat, x, b, kappa, tol, max_iter, o, ws, info, st);
  return QCD_ERR_UNSUPPORTED;
}

}  // namespace qcd
