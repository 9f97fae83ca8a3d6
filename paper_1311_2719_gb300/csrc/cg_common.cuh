// Conjugate-gradient building blocks shared by the single-RHS, multi-RHS and batched solvers:
// device scalars, the fused epilogues, the reliable-update and output kernels, the workspace
// layout and the single-RHS launch sequences.
#pragma once

#include <type_traits>

#include "dslash.cuh"
#include "dslash_staged.cuh"


namespace qcd {

struct __align__(256) CgScalars {
  double rr, rr_prev, pp, alpha, beta, delit, bb, m2, res2, rmax2, delta2, tol2;
  int iter, max_iter, done, since_ru, ru_count, ru_interval, mixed, loops;
  int fault;  // set by a kernel whose bounded device-side wait gave up: 1, or 2 when its drain of the
              // copies in flight gave up as well
  unsigned counter[16];
};
static_assert(sizeof(CgScalars) <= 256, "scalars block");

// kConverged: the recursion met tol; the solver confirms it by replacing r with the true FP64
// residual (a reliable update), which ends in kTrueConverged or back in kRunning.
enum { kRunning = 0, kConverged = 1, kMaxIter = 2, kBreakdown = 3, kReliable = 4, kTrueConverged = 5 };

__device__ __forceinline__ bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// ---------------------------------------------------------------- init: r = b_e, x = 0, p = 0
template <class FieldT, class XFieldT>
__global__ void __launch_bounds__(kSpreadBlockMax) cg_init_kernel(Geom g, const double2* __restrict__ b_canon,
                                                         Field<QCD_PREC_DOUBLE> b_hi, Field<QCD_PREC_DOUBLE> x_hi,
                                                         FieldT r, FieldT p, XFieldT x_lo, int mixed, CgScalars* sc,
                                                         double* partials) {
  using T = typename FieldT::T;
  using TX = typename XFieldT::T;
  double red[1] = {0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
    const Site s = site_of(g, k, QCD_EVEN);
    cvec3<double> b;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double2 d = b_canon[(size_t)s.lex * 3 + a];
      b.c[a].re = d.x; b.c[a].im = d.y;
    }
    b_hi.store(k, b);
    cvec3<T> bl, z;
    zero(z);
#pragma unroll
    for (int a = 0; a < 3; ++a) { bl.c[a].re = (T)b.c[a].re; bl.c[a].im = (T)b.c[a].im; }
    r.store(k, bl);
    p.store(k, z);
    cvec3<TX> zx;
    zero(zx);
    x_lo.store(k, zx);
    if (mixed) {
      cvec3<double> zd;
      zero(zd);
      x_hi.store(k, zd);
    }
    red[0] += norm2(b);
  }
  double tot[1];
  if (grid_sum_last_block<1>(red, partials, &sc->counter[0], tot) && threadIdx.x == 0) {
    const double bb = tot[0];
    sc->bb = bb;
    sc->rr = bb;
    sc->rr_prev = bb;
    sc->rmax2 = bb;
    sc->pp = 0.0;
    sc->beta = 0.0;
    sc->alpha = 0.0;
    sc->delit = sc->tol2 * bb;
    sc->iter = 0;
    sc->since_ru = 0;
    sc->ru_count = 0;
    sc->loops = 0;
    sc->done = !isfinite(bb) ? kBreakdown : (bb == 0.0 ? kTrueConverged : kRunning);
  }
}

// ---------------------------------------------------------------- K3: p = r + beta p
// A plain axpy: |p|^2 is summed by the next K1 (which reads p anyway), so K3 needs no grid reduction.
template <class FieldT>
__global__ void __launch_bounds__(kSpreadBlockMax) cg_p_kernel(int Vh, FieldT r, FieldT p, CgScalars* sc) {
  using T = typename FieldT::T;
  if (sc->done != kRunning) return;
  const T beta = (T)sc->beta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Vh; k += gridDim.x * blockDim.x) {
    cvec3<T> rv = r.load(k), pv = p.load(k);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      pv.c[a].re = fma(beta, pv.c[a].re, rv.c[a].re);
      pv.c[a].im = fma(beta, pv.c[a].im, rv.c[a].im);
    }
    p.store(k, pv);
  }
}

// ---------------------------------------------------------------- K1 epilogue: ap = D_oe p
// Besides |ap|^2 (odd sites) it sums |p|^2 over the even site with the same index k, so that every
// even site is counted once: alpha = rr / (|D_oe p|^2 + m^2 |p|^2) from one launch.
template <class FieldT>
struct EpiAp {
  static constexpr int NV = 2;
  static constexpr bool kPrefetch = false;
  FieldT ap;
  FieldT p;  // the even field the operator reads
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return sc->done != kRunning; }
  template <class T, class A>
  __device__ __forceinline__ void site(int k, cvec3<T>& acc, A* red) const {
    ap.store(k, acc);
    accum(red[0], norm2(acc));
    accum(red[1], norm2(p.load(k)));
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    const A v[2] = {red[0], red[1]};
    double tot[2];
    if (grid_sum_last_block<2>(v, partials, &sc->counter[2], tot) && threadIdx.x == 0) {
      sc->pp = tot[1];
      const double d = tot[0] + sc->m2 * tot[1];  // <p, A p> = |D_oe p|^2 + m^2 |p|^2
      const double alpha = sc->rr / d;
      if (!finite_pos(d) || !isfinite(alpha)) {
        sc->done = kBreakdown;
      } else {
        sc->alpha = alpha;
      }
    }
  }
};

// ---------------------------------------------------------------- K1 with the p update folded in
// p_next = r + beta p at a site, from the stored r and p: the CG's "p = r + beta p" step, done by the
// operator that consumes p so that it needs no launch and no pass over memory of its own.
template <class FieldT>
struct PNext {
  using T = typename FieldT::T;
  static constexpr int kElemsPerSite = FieldT::kElemsPerSite;
  FieldT r, p;
  T beta;
  __device__ __forceinline__ cvec3<T> load(int j) const {
    const cvec3<T> rv = r.load(j);
    cvec3<T> pv = p.load(j);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      pv.c[a].re = fma(beta, pv.c[a].re, rv.c[a].re);
      pv.c[a].im = fma(beta, pv.c[a].im, rv.c[a].im);
    }
    return pv;
  }
};

// K1 for the FP32 recursion: iteration i reads p_i from buffer i mod 2 (p0, p1), gathers
// p_{i+1} = r + beta p_i at the neighbours, and writes ap = D_oe p_{i+1}, p_{i+1} at the even site with
// the same index into the other buffer, |ap|^2 and |p_{i+1}|^2. The stored p_{i+1} is bit-identical to
// the one every neighbour formed (the same FP32 multiply-add), so the recursion is the unfolded one.
// Measured on GB300 (32^4, m = 0.01): 334.7 -> 329.6 ms per solve. The other recursions keep the
// separate p kernel: FP16 (issue-bound decoding two packed fields at every neighbour, and the stored p
// rounded to FP16 differs from the gathered one; 318.6 -> 329.7 ms), FP64 and df64 (the extra
// multiply-adds at every neighbour cost more on the FP64 / FP32 pipes than the pass they save).
template <class FieldT>
struct EpiApFold {
  static constexpr int NV = 2;
  static constexpr bool kPrefetch = false;
  using T = typename FieldT::T;
  FieldT ap, r, p0, p1;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return sc->done != kRunning; }
  __device__ __forceinline__ PNext<FieldT> next() const { return {r, (sc->iter & 1) ? p1 : p0, (T)sc->beta}; }
  template <class In>
  __device__ __forceinline__ PNext<FieldT> bind(const In&) const { return next(); }
  template <class A>
  __device__ __forceinline__ void site(int k, cvec3<T>& acc, A* red) const {
    ap.store(k, acc);
    const cvec3<T> pv = next().load(k);
    ((sc->iter & 1) ? p0 : p1).store(k, pv);
    accum(red[0], norm2(acc));
    accum(red[1], norm2(pv));
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const { EpiAp<FieldT>{ap, p0, sc, partials}.finish(red); }
};

// ---------------------------------------------------------------- K2 epilogue: update x, r
template <class FieldT, class XFieldT>
struct EpiUpdate {
  static constexpr int NV = 1;
  static constexpr bool kPrefetch = true;
  FieldT p, r;
  XFieldT x;
  CgScalars* sc;
  double* partials;
  // With the p update folded into K1 (EpiApFold), p of iteration i + 1 sits in p_odd when i is even
  // and in p when i is odd.
  FieldT p_odd = {};
  int pingpong = 0;
  struct Pre {
    cvec3<typename FieldT::T> p, r;
    cvec3<typename XFieldT::T> x;
  };
  __device__ __forceinline__ bool skip() const { return sc->done != kRunning; }
  __device__ __forceinline__ const FieldT& cur_p() const { return (pingpong && !(sc->iter & 1)) ? p_odd : p; }
  __device__ __forceinline__ Pre prefetch(int k) const { return Pre{cur_p().load(k), r.load(k), x.load(k)}; }
  template <class T, class A>
  __device__ __forceinline__ void site(int k, cvec3<T>& acc, A* red) const { site_pre(k, acc, red, prefetch(k)); }
  template <class T, class A>
  __device__ __forceinline__ void site_pre(int k, cvec3<T>& acc, A* red, const Pre& pre) const {
    using TX = typename XFieldT::T;
    const T alpha = (T)sc->alpha, m2 = (T)sc->m2;
    const cvec3<T>& pv = pre.p;
    cvec3<T> rv = pre.r;
    cvec3<TX> xv = pre.x;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T at_re = fma(m2, pv.c[a].re, -acc.c[a].re);  // (A p)_a = m^2 p - D_eo D_oe p
      const T at_im = fma(m2, pv.c[a].im, -acc.c[a].im);
      rv.c[a].re = fma(-alpha, at_re, rv.c[a].re);
      rv.c[a].im = fma(-alpha, at_im, rv.c[a].im);
      xv.c[a].re = fma((TX)alpha, (TX)pv.c[a].re, xv.c[a].re);
      xv.c[a].im = fma((TX)alpha, (TX)pv.c[a].im, xv.c[a].im);
    }
    r.store(k, rv);
    x.store(k, xv);
    accum(red[0], norm2(rv));
  }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const {
    const A v[1] = {red[0]};
    double tot[1];
    if (grid_sum_last_block<1>(v, partials, &sc->counter[3], tot) && threadIdx.x == 0) {
      const double rr = tot[0];
      sc->iter += 1;
      sc->since_ru += 1;
      sc->rr_prev = sc->rr;
      sc->rr = rr;
      if (!isfinite(rr)) {
        sc->done = kBreakdown;
        return;
      }
      sc->beta = rr / sc->rr_prev;
      if (rr > sc->rmax2) sc->rmax2 = rr;
      if (rr < sc->delit) {
        sc->done = kConverged;  // mixed: confirmed by a reliable update on the host's next check
      } else if (sc->iter >= sc->max_iter) {
        sc->done = kMaxIter;
      } else if (sc->mixed && (sc->since_ru >= sc->ru_interval || rr < sc->delta2 * sc->rmax2)) {
        sc->done = kReliable;
      }
    }
  }
};

// ---------------------------------------------------------------- reliable update (FP64)
// True when the recursion asks for a reliable update: it met tol (confirm on the true residual)
// or, mixed only, the periodic / delta test fired.
__device__ __forceinline__ bool ru_wanted(const CgScalars* sc) {
  const int d = sc->done;
  return d == kConverged || (sc->mixed && d == kReliable);
}

// x_hi += x_lo, x_lo = 0. With `gate`, the kernel returns at once unless ru_wanted(gate).
template <class XFieldT>
__global__ void __launch_bounds__(kSpreadBlockMax) ru_accumulate_kernel(int Vh, Field<QCD_PREC_DOUBLE> x_hi, XFieldT x_lo,
                                                               const CgScalars* gate = nullptr) {
  using TX = typename XFieldT::T;
  if (gate && !ru_wanted(gate)) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Vh; k += gridDim.x * blockDim.x) {
    cvec3<double> xh = x_hi.load(k);
    const cvec3<TX> xl = x_lo.load(k);
#pragma unroll
    for (int a = 0; a < 3; ++a) { xh.c[a].re += (double)xl.c[a].re; xh.c[a].im += (double)xl.c[a].im; }
    x_hi.store(k, xh);
    cvec3<TX> z;
    zero(z);
    x_lo.store(k, z);
  }
}

// r_hi = b - (m^2 x_hi - D_eo tmp) with tmp = D_oe x_hi; the low-precision r takes r_hi.
template <class FieldT>
struct EpiReliable {
  static constexpr int NV = 1;
  static constexpr bool kPrefetch = false;
  Field<QCD_PREC_DOUBLE> b, x;
  FieldT r_lo;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void site(int k, cvec3<double>& acc, double* red) const {
    using T = typename FieldT::T;
    const cvec3<double> bv = b.load(k), xv = x.load(k);
    cvec3<double> rv;
    cvec3<T> rl;
    const double m2 = sc->m2;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      rv.c[a].re = bv.c[a].re - fma(m2, xv.c[a].re, -acc.c[a].re);
      rv.c[a].im = bv.c[a].im - fma(m2, xv.c[a].im, -acc.c[a].im);
      rl.c[a].re = (T)rv.c[a].re;
      rl.c[a].im = (T)rv.c[a].im;
    }
    r_lo.store(k, rl);
    red[0] += norm2(rv);
  }
  __device__ __forceinline__ void finish(double* red) const {
    double v[1] = {red[0]}, tot[1];
    if (grid_sum_last_block<1>(v, partials, &sc->counter[4], tot) && threadIdx.x == 0) {
      const double rr = tot[0];
      if (!isfinite(rr)) {
        sc->done = kBreakdown;
        return;
      }
      sc->beta = sc->iter > 0 ? rr / sc->rr_prev : 0.0;
      sc->rr = rr;
      sc->rmax2 = rr;
      sc->since_ru = 0;
      sc->ru_count += 1;
      sc->res2 = rr;
      if (rr < sc->delit) sc->done = kTrueConverged;
      else if (sc->iter >= sc->max_iter) sc->done = kMaxIter;
      else sc->done = kRunning;
    }
  }
};

// An epilogue that runs only when a reliable update is wanted (for the device-side solve loop,
// where the update kernels sit in every pass of the loop body and return at once otherwise).
template <class Epi>
struct Gated {
  static constexpr int NV = Epi::NV;
  static constexpr bool kPrefetch = false;
  Epi epi;
  const CgScalars* gate;
  __device__ __forceinline__ bool skip() const { return !ru_wanted(gate) || epi.skip(); }
  template <class T, class A>
  __device__ __forceinline__ void site(int k, cvec3<T>& acc, A* red) const { epi.site(k, acc, red); }
  template <class A>
  __device__ __forceinline__ void finish(A* red) const { epi.finish(red); }
};

// Last node of the device-side solve loop: keep looping while the recursion runs (bounded by
// `max_loops` passes as a guard).
static __global__ void cg_loop_control_kernel(CgScalars* sc, cudaGraphConditionalHandle handle, int max_loops) {
  const int loops = ++sc->loops;
  cudaGraphSetConditional(handle, (sc->done == kRunning && sc->fault == 0 && loops < max_loops) ? 1u : 0u);
}

// Final true residual: res = b - (m^2 x - D_eo y), y = D_oe x.
struct EpiResidual {
  static constexpr int NV = 1;
  static constexpr bool kPrefetch = false;
  Field<QCD_PREC_DOUBLE> b, x;
  CgScalars* sc;
  double* partials;
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void site(int k, cvec3<double>& acc, double* red) const {
    const cvec3<double> bv = b.load(k), xv = x.load(k);
    const double m2 = sc->m2;
    cvec3<double> rv;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      rv.c[a].re = bv.c[a].re - fma(m2, xv.c[a].re, -acc.c[a].re);
      rv.c[a].im = bv.c[a].im - fma(m2, xv.c[a].im, -acc.c[a].im);
    }
    red[0] += norm2(rv);
  }
  __device__ __forceinline__ void finish(double* red) const {
    double v[1] = {red[0]}, tot[1];
    if (grid_sum_last_block<1>(v, partials, &sc->counter[5], tot) && threadIdx.x == 0) sc->res2 = tot[0];
  }
};

// Write x (even sites) and y (odd sites) into canonical fields, zeroing the other halves.
static __global__ void __launch_bounds__(kSpreadBlockMax) cg_output_kernel(Geom g, double2* __restrict__ x_canon,
                                                           double2* __restrict__ y_canon, Field<QCD_PREC_DOUBLE> x_e,
                                                           Field<QCD_PREC_DOUBLE> y_o) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
    const Site se = site_of(g, k, QCD_EVEN), so = site_of(g, k, QCD_ODD);
    const cvec3<double> xv = x_e.load(k);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x_canon[(size_t)se.lex * 3 + a] = make_double2(xv.c[a].re, xv.c[a].im);
      x_canon[(size_t)so.lex * 3 + a] = make_double2(0.0, 0.0);
    }
    if (y_canon) {
      const cvec3<double> yv = y_o.load(k);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        y_canon[(size_t)so.lex * 3 + a] = make_double2(yv.c[a].re, yv.c[a].im);
        y_canon[(size_t)se.lex * 3 + a] = make_double2(0.0, 0.0);
      }
    }
  }
}

// ---------------------------------------------------------------- workspace layout
// R right-hand sides: every field kind is R packed fields back to back, R scalar blocks.
struct CgWork {
  CgScalars* sc;
  double* partials;
  void* b_hi;
  void* x_hi;
  void* tmp_o;  // FP64 odd: reliable-update D_oe x and the final y
  void* r;
  void* p;
  void* p2;  // second p buffer of the folded K1 (FP32 recursion), else nullptr
  void* ap;
  void* x_lo;
  size_t total;
  int R;
  size_t f64, fin, fx;  // bytes of one field: FP64, inner precision, x accumulator
};

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

inline CgWork carve(const qcd_lattice* lat, int prec_inner, int R, char* base) {
  CgWork w{};
  size_t off = 0;
  auto take = [&](size_t n) { void* p = base ? base + off : nullptr; off += align256(n); return p; };
  w.R = R;
  w.sc = (CgScalars*)take(sizeof(CgScalars) * R);
  w.partials = (double*)take(sizeof(double) * kMaxPartials * (R > 2 ? R : 2));
  const long long Vh = lat->Vh;
  w.f64 = field_bytes(QCD_PREC_DOUBLE, Vh);
  w.fin = field_bytes(prec_inner, Vh);
  w.fx = field_bytes(x_prec(prec_inner), Vh);
  w.b_hi = take(w.f64 * R);
  w.x_hi = take(w.f64 * R);
  w.tmp_o = take(w.f64 * R);
  w.r = take(w.fin * R);
  w.p = take(w.fin * R);
  w.ap = take(w.fin * R);
  // the FP32 recursion alternates p between two buffers (EpiApFold)
  w.p2 = prec_inner == QCD_PREC_SINGLE ? take(w.fin * R) : nullptr;
  // plain FP64: x accumulates directly in the FP64 field
  w.x_lo = prec_inner == QCD_PREC_DOUBLE ? w.x_hi : take(w.fx * R);
  w.total = off;
  return w;
}

// The single-RHS view of right-hand side r.
inline CgWork view(const CgWork& w, int r) {
  CgWork v = w;
  auto at = [&](void* p, size_t stride) { return p ? (void*)((char*)p + stride * r) : nullptr; };
  v.sc = w.sc + r;
  v.b_hi = at(w.b_hi, w.f64);
  v.x_hi = at(w.x_hi, w.f64);
  v.tmp_o = at(w.tmp_o, w.f64);
  v.r = at(w.r, w.fin);
  v.p = at(w.p, w.fin);
  v.p2 = at(w.p2, w.fin);
  v.ap = at(w.ap, w.fin);
  v.x_lo = at(w.x_lo, w.fx);
  v.R = 1;
  return v;
}

// ---------------------------------------------------------------- single-RHS launch sequences
template <int PREC, int RECON>
struct CgRunner {
  using FieldT = Field<PREC>;
  using XPREC = std::integral_constant<int, x_prec(PREC)>;
  using XFieldT = Field<XPREC::value>;
  const qcd_lattice* lat;
  Geom g;
  CgWork w;
  cudaStream_t st;
  int grid;
  int block = kBlock;  // threads per block of every kernel of the runner (<= kBlock)
  int tps = 1;         // threads per site of the operator kernels
  long long launches = 0;

  int stream_in = 0;    // stream the inner-precision links with the L2 evict-first policy
  int stream64 = 0;     // the same for the FP64 links of the reliable updates and the output
  int staged_grid = 0;  // > 0: FP32 recon-12 operator launches use the staged kernel with this grid
  long long wait_cycles = kWaitCycles;

  // Enable the staged operator (FP32 recon-12, 16-byte aligned links; it maps one thread to one site
  // of a tile whatever `tps` says) and size its persistent grid: all resident blocks, at most one
  // per tile.
  void setup_staged(bool want) {
    staged_grid = 0;
    if constexpr (PREC == QCD_PREC_SINGLE && RECON == 12) {
      const void* lp = lat->links[PREC].ptr;
      if (!want || ((uintptr_t)lp & 15u) != 0) return;
      const int smem = 2 * (int)sizeof(StageFp32R12);
      auto k1 = dslash_staged_fp32r12_kernel<EpiAp<FieldT>>;
      auto k2 = dslash_staged_fp32r12_kernel<EpiUpdate<FieldT, XFieldT>>;
      if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
          cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
      int dev = 0, sms = 0, per1 = 0, per2 = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k1, kStageSites, smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k2, kStageSites, smem) != cudaSuccess || per1 < 1 || per2 < 1) {
        cudaGetLastError();
        return;
      }
      const long long tiles = (g.Vh + kStageSites - 1) / kStageSites;
      long long gr = (long long)sms * (per1 < per2 ? per1 : per2);
      if (gr > tiles) gr = tiles;
      if (gr > kMaxPartials) gr = kMaxPartials;
      staged_grid = (int)gr;
    }
  }

  // One operator launch with epilogue `epi` at the runner's threads-per-site.
  template <class LinksT, class InT, class Epi>
  void op(const LinksT& U, const InT& in, int out_par, const Epi& epi) {
    if constexpr (std::is_same<LinksT, Links<QCD_PREC_SINGLE, 12>>::value && std::is_same<InT, Field<QCD_PREC_SINGLE>>::value) {
      if (staged_grid > 0) {
        dslash_staged_fp32r12_kernel<Epi><<<staged_grid, kStageSites, 2 * sizeof(StageFp32R12), st>>>(
            g, U, in, out_par, epi, &w.sc->fault, wait_cycles);
        return;
      }
    }
    if (tps == 2) dslash_kernel<LinksT, InT, Epi, 2><<<grid, block, 0, st>>>(g, U, in, out_par, epi);
    else dslash_kernel<LinksT, InT, Epi, 1><<<grid, block, 0, st>>>(g, U, in, out_par, epi);
  }

  // One CG iteration (K3 p = r + beta p; K1 ap = D_oe p with |ap|^2 and |p|^2; K2 D_eo ap and the
  // x, r update with |r|^2). With `ev` (4 events) the two operator launches are bracketed.
  // The FP32 recursion runs the p update inside K1 (two launches per iteration), except with the
  // staged operator, which stages one stored input field.
  bool folded() const { return PREC == QCD_PREC_SINGLE && staged_grid == 0 && w.p2; }
  int launches_per_iteration() const { return folded() ? 2 : 3; }

  int iteration(cudaEvent_t* ev = nullptr) {
    auto U = make_links<PREC, RECON>(lat->links[PREC].ptr, g.Vh);
    U.stream = stream_in;
    FieldT r = make_field<PREC>(w.r, g.Vh), p = make_field<PREC>(w.p, g.Vh), ap = make_field<PREC>(w.ap, g.Vh);
    XFieldT x = make_field<XPREC::value>(w.x_lo, g.Vh);
    if (folded()) {
      FieldT p2 = make_field<PREC>(w.p2, g.Vh);
      if (ev) QCD_CUDA(cudaEventRecord(ev[0], st));
      op(U, p, QCD_ODD, EpiApFold<FieldT>{ap, r, p, p2, w.sc, w.partials});
      if (ev) QCD_CUDA(cudaEventRecord(ev[1], st));
      if (ev) QCD_CUDA(cudaEventRecord(ev[2], st));
      op(U, ap, QCD_EVEN, EpiUpdate<FieldT, XFieldT>{p, r, x, w.sc, w.partials, p2, 1});
      if (ev) QCD_CUDA(cudaEventRecord(ev[3], st));
      QCD_CUDA(cudaGetLastError());
      launches += 2;
      return QCD_OK;
    }
    cg_p_kernel<<<grid, block, 0, st>>>(g.Vh, r, p, w.sc);
    if (ev) QCD_CUDA(cudaEventRecord(ev[0], st));
    op(U, p, QCD_ODD, EpiAp<FieldT>{ap, p, w.sc, w.partials});
    if (ev) QCD_CUDA(cudaEventRecord(ev[1], st));
    if (ev) QCD_CUDA(cudaEventRecord(ev[2], st));
    op(U, ap, QCD_EVEN, EpiUpdate<FieldT, XFieldT>{p, r, x, w.sc, w.partials});
    if (ev) QCD_CUDA(cudaEventRecord(ev[3], st));
    QCD_CUDA(cudaGetLastError());
    launches += 3;
    return QCD_OK;
  }

  int init(const void* b_canon) {
    FieldT r = make_field<PREC>(w.r, g.Vh), p = make_field<PREC>(w.p, g.Vh);
    XFieldT x = make_field<XPREC::value>(w.x_lo, g.Vh);
    launches += 1;
    cg_init_kernel<<<grid, block, 0, st>>>(g, (const double2*)b_canon, make_field<QCD_PREC_DOUBLE>(w.b_hi, g.Vh),
                                            make_field<QCD_PREC_DOUBLE>(w.x_hi, g.Vh), r, p, x,
                                            PREC != QCD_PREC_DOUBLE, w.sc, w.partials);
    QCD_CUDA(cudaGetLastError());
    return QCD_OK;
  }

  // Replace the iterated residual by the true one, r = b - A x_hi in FP64 (mixed: after folding
  // x_lo into x_hi). Plain FP64 runs it once the recursion meets tol, to confirm on the true
  // residual; the mixed solver also every reliable_interval iterations / on the delta test.
  // `gated`: every kernel checks the device flag first (for the device-side loop body).
  int reliable_update(bool gated = false) {
    auto U64 = make_links<QCD_PREC_DOUBLE, 18>(lat->links[QCD_PREC_DOUBLE].ptr, g.Vh);
    U64.stream = stream64;
    auto xh = make_field<QCD_PREC_DOUBLE>(w.x_hi, g.Vh);
    auto tmp = make_field<QCD_PREC_DOUBLE>(w.tmp_o, g.Vh);
    launches += PREC != QCD_PREC_DOUBLE ? 3 : 2;
    if (PREC != QCD_PREC_DOUBLE)  // plain FP64: x_lo is x_hi itself
      ru_accumulate_kernel<<<grid, block, 0, st>>>(g.Vh, xh, make_field<XPREC::value>(w.x_lo, g.Vh),
                                                    gated ? w.sc : nullptr);
    EpiStore<Field<QCD_PREC_DOUBLE>> store{tmp};
    EpiReliable<FieldT> rel{make_field<QCD_PREC_DOUBLE>(w.b_hi, g.Vh), xh, make_field<PREC>(w.r, g.Vh), w.sc,
                            w.partials};
    if (gated) {
      op(U64, xh, QCD_ODD, Gated<decltype(store)>{store, w.sc});
      op(U64, tmp, QCD_EVEN, Gated<decltype(rel)>{rel, w.sc});
    } else {
      op(U64, xh, QCD_ODD, store);
      op(U64, tmp, QCD_EVEN, rel);
    }
    QCD_CUDA(cudaGetLastError());
    return QCD_OK;
  }

  int finish(void* x_canon, void* y_canon) {
    auto U64 = make_links<QCD_PREC_DOUBLE, 18>(lat->links[QCD_PREC_DOUBLE].ptr, g.Vh);
    U64.stream = stream64;
    auto xh = make_field<QCD_PREC_DOUBLE>(w.x_hi, g.Vh);
    auto tmp = make_field<QCD_PREC_DOUBLE>(w.tmp_o, g.Vh);
    launches += PREC != QCD_PREC_DOUBLE ? 4 : 3;
    if (PREC != QCD_PREC_DOUBLE)
      ru_accumulate_kernel<<<grid, block, 0, st>>>(g.Vh, xh, make_field<XPREC::value>(w.x_lo, g.Vh));
    op(U64, xh, QCD_ODD, EpiStore<Field<QCD_PREC_DOUBLE>>{tmp});
    op(U64, tmp, QCD_EVEN, EpiResidual{make_field<QCD_PREC_DOUBLE>(w.b_hi, g.Vh), xh, w.sc, w.partials});
    cg_output_kernel<<<grid, block, 0, st>>>(g, (double2*)x_canon, (double2*)y_canon, xh, tmp);
    QCD_CUDA(cudaGetLastError());
    return QCD_OK;
  }
};

// One-wave grid of the CG kernels of (PREC, RECON), sized on the heaviest of them (K2). The same
// value serves every RHS count so that multi-RHS and single-RHS reductions sum identically.
template <int PREC, int RECON>
inline int cg_grid(long long Vh, int tps) {
  using FieldT = Field<PREC>;
  using XFieldT = Field<x_prec(PREC)>;
  if (tps == 2) return one_wave_grid(Vh, dslash_kernel<Links<PREC, RECON>, FieldT, EpiUpdate<FieldT, XFieldT>, 2>, 2);
  return one_wave_grid(Vh, dslash_kernel<Links<PREC, RECON>, FieldT, EpiUpdate<FieldT, XFieldT>, 1>, 1);
}

// Launch shape of the single-RHS CG kernels: the one-wave grid of 128-thread blocks; when the
// lattice needs less than one wave, one block per SM with the sites spread evenly (blocks of
// ceil(threads / SMs), rounded up to whole warps). The busiest SM sets the time of the pipe-bound
// operator: 16^4 = 32768 sites per parity in 128-thread blocks puts 256 sites on some SMs against
// 216 on average; 147 blocks of 224 put at most 224 on one.
inline void cg_launch_shape(long long threads, int wave_grid, int* grid, int* block) {
  *grid = wave_grid;
  *block = kBlock;
  if ((threads + kBlock - 1) / kBlock > wave_grid) return;  // at least a full wave
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    return;
  long long b = (threads + sms - 1) / sms;
  b = (b + 31) / 32 * 32;
  if (b <= kBlock || b > kSpreadBlockMax) return;
  *block = (int)b;
  *grid = (int)((threads + b - 1) / b);
}

inline int read_scalars(const CgWork& w, CgScalars* h, cudaStream_t st, int count = 1) {
  QCD_CUDA(cudaMemcpyAsync(h, w.sc, sizeof(CgScalars) * count, cudaMemcpyDeviceToHost, st));
  QCD_CUDA(cudaStreamSynchronize(st));
  return QCD_OK;
}

// ---------------------------------------------------------------- multi-RHS grid reductions
// (grid.y enumerates blocks of RB right-hand sides; partials are [rhs][kMaxPartials])
// Write this block's RB partial sums for RHS r0..r0+RB-1; true in the block that finishes last
// over the whole (x, y) grid.
template <int RB, class A>
__device__ __forceinline__ bool mrhs_arrive(const A (&x)[RB], int r0, int nrhs, double* partials, unsigned* counter) {
  __shared__ bool am_last;
  double v[RB];
  block_sum<RB>(x, v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < RB; ++j)
      if (r0 + j < nrhs) partials[(size_t)(r0 + j) * kMaxPartials + blockIdx.x] = v[j];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  return am_last;
}

// In the last block: tot[r] = sum over blocks of partials[r][.] in block order (deterministic).
// Four right-hand sides at a time, so that their loads are in flight together; each total is summed
// in the same order as a single-RHS reduction over the same grid.
__device__ __forceinline__ void mrhs_totals(int nrhs, const double* partials, double* tot_smem) {
  __threadfence();
  int r = 0;
  for (; r + 4 <= nrhs; r += 4) {
    double s[4];
    sum_partials<4>(partials + (size_t)r * kMaxPartials, (int)gridDim.x, s);
    if (threadIdx.x == 0)
      for (int q = 0; q < 4; ++q) tot_smem[r + q] = s[q];
  }
  for (; r < nrhs; ++r) {
    double s[1];
    sum_partials<1>(partials + (size_t)r * kMaxPartials, (int)gridDim.x, s);
    if (threadIdx.x == 0) tot_smem[r] = s[0];
  }
  __syncthreads();
}

}  // namespace qcd
