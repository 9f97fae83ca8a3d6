#pragma once
// (Shared by the per-precision translation units cg_mrhs_*.cu.)
// Multi-RHS even-odd CG: R independent CG recursions on one lattice that share every link load.
//
// The iteration is the single-RHS one (K3 p-update, K1 D_oe p, K2 D_eo ap + x/r update) with the
// operator kernels applying each loaded link to a block of RB right-hand sides held in registers
// (grid.y enumerates the RHS blocks; with RB = R every link is read once per half-lattice hop).
// Each RHS keeps its own device scalars and convergence flag; converged RHS are skipped inside
// the kernels. Reliable updates, start-up and the final y / true residual reuse the single-RHS
// launch sequences on per-RHS views of the workspace.
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "cg_common.cuh"

namespace qcd {

std::string mrhs_key(const qcd_lattice* lat, int prec, int recon, int nrhs);
bool tune_lookup(const std::string& key, std::vector<int>* out);

// Counter slots in sc[0] used by the multi-RHS kernels (single-RHS kernels use 0..5 of each sc[r]).
enum { kCtrK3M = 8, kCtrK1M = 9, kCtrK2M = 10 };

// Last node of the device-side multi-RHS loop: loop again while any right-hand side still runs.
static __global__ void mrhs_loop_control_kernel(CgScalars* sc, int nrhs, cudaGraphConditionalHandle handle,
                                                int max_loops) {
  const int lane = threadIdx.x;
  const bool running = lane < nrhs && sc[lane].done == kRunning;
  const unsigned any = __ballot_sync(0xffffffffu, running);
  if (lane == 0) {
    const int loops = ++sc[0].loops;
    cudaGraphSetConditional(handle, (any != 0u && loops < max_loops) ? 1u : 0u);
  }
}

// ---------------------------------------------------------------- K3: p_r = r_r + beta_r p_r
template <class FieldT>
__global__ void __launch_bounds__(kBlock) cg_p_mrhs_kernel(int Vh, FieldT r_all, FieldT p_all, int nrhs, CgScalars* sc,
                                                           double* partials) {
  using T = typename FieldT::T;
  const int r = blockIdx.y;
  typename Accum<T>::type part = 0;
  if (sc[r].done == kRunning) {
    const FieldT rf = field_at(r_all, r), pf = field_at(p_all, r);
    const T beta = (T)sc[r].beta;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Vh; k += gridDim.x * blockDim.x) {
      cvec3<T> rv = rf.load(k), pv = pf.load(k);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pv.c[a].re = fma(beta, pv.c[a].re, rv.c[a].re);
        pv.c[a].im = fma(beta, pv.c[a].im, rv.c[a].im);
      }
      pf.store(k, pv);
      accum(part, norm2(pv));
    }
  }
  const decltype(part) red[1] = {part};
  if (mrhs_arrive<1>(red, r, nrhs, partials, &sc[0].counter[kCtrK3M])) {
    __shared__ double tot[kMaxRhs];
    mrhs_totals(nrhs, partials, tot);
    // one thread per right-hand side (each update is a chain of dependent global loads and stores)
    if (threadIdx.x < nrhs && sc[threadIdx.x].done == kRunning) sc[threadIdx.x].pp = tot[threadIdx.x];
    if (threadIdx.x == 0) sc[0].counter[kCtrK3M] = 0u;
  }
}

// ---------------------------------------------------------------- operator kernel with per-RHS epilogue
// resident blocks per SM of the multi-RHS operator: 4 (at most 128 registers) for the FP32-arithmetic
// register blocks up to 4 RHS, the compiler's own choice otherwise
template <class LinksT, int RB>
struct MrhsMinBlocks {
  static constexpr int value = (sizeof(typename LinksT::T) == 4 && RB <= 4) ? 4 : 0;
};

template <class LinksT, class FieldT, int RB, class Epi>
__global__ void __launch_bounds__(kBlock, MrhsMinBlocks<LinksT, RB>::value) dslash_mrhs_cg_kernel(Geom g, LinksT U, FieldT in, int nrhs, int out_par,
                                                                Epi epi) {
  using T = typename LinksT::T;
  const int r0 = blockIdx.y * RB;
  unsigned active = 0;
#pragma unroll
  for (int j = 0; j < RB; ++j)
    if (r0 + j < nrhs && epi.sc[r0 + j].done == kRunning) active |= 1u << j;
  using A = typename Accum<T>::type;
  A part[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) part[j] = A(0);
  if (active) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
      const Site s = site_of(g, k, out_par);
      int fwd[4], bwd[4];
      neighbours(g, s, fwd, bwd);
      cvec3<T> acc[RB];
#pragma unroll
      for (int j = 0; j < RB; ++j) zero(acc[j]);
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        su3<T> Uf = U.load(out_par, mu, k);
        if constexpr (!LinksT::kFolded) scale(Uf, T(0.5f * fwd_sign(g, s, mu)));
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if ((active >> j) & 1u) mul_add(acc[j], Uf, field_at(in, r0 + j).load(fwd[mu]));
        su3<T> Ub = U.load(1 - out_par, mu, bwd[mu]);
        if constexpr (!LinksT::kFolded) scale(Ub, T(0.5f * bwd_sign(g, s, mu)));
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if ((active >> j) & 1u) adj_mul_sub(acc[j], Ub, field_at(in, r0 + j).load(bwd[mu]));
      }
#pragma unroll
      for (int j = 0; j < RB; ++j)
        if ((active >> j) & 1u) epi.site(k, r0 + j, acc[j], part[j]);
    }
  }
  if (mrhs_arrive<RB>(part, r0, nrhs, epi.partials, &epi.sc[0].counter[Epi::kCounter])) {
    __shared__ double tot[kMaxRhs];
    mrhs_totals(nrhs, epi.partials, tot);
    // one thread per right-hand side: a serial loop over sixteen updates (dependent global loads and
    // stores, an FP64 division each) kept the summing block's SM busy ~70k cycles after the others
    if (threadIdx.x < nrhs && epi.sc[threadIdx.x].done == kRunning) epi.update(threadIdx.x, tot[threadIdx.x]);
    if (threadIdx.x == 0) epi.sc[0].counter[Epi::kCounter] = 0u;
  }
}

// ---------------------------------------------------------------- operator kernel with shared links
// For many right-hand sides: a block of kShWarps warps takes a tile of kShTile consecutive output
// sites. In the load phase warp w fetches link slot w of the tile's sites (direction w / 2, forward or
// backward; one lane per site, coalesced), rebuilds the third row of a compressed link, applies
// 1/2 eta zeta where the format does not fold it in, turns a backward link into -U^dagger, and stores
// the result in shared memory. After a barrier, warp w applies the eight stored links of each site
// to right-hand sides w and w + kShWarps. Every link is read from memory once per launch; the grid
// rows of dslash_mrhs_cg_kernel instead re-read it from L2 once per RHS block (at 24^4 x 16 RHS, 1 GB
// of L2 reads per launch against 64 MB of links).

// resident blocks per SM: 4 (64 registers, 32 warps to hide the neighbour gathers) in FP32 arithmetic;
// 2 for the 64-bit types, which spill below 128 registers
template <class LinksT>
struct ShMinBlocks {
  static constexpr int value = sizeof(typename LinksT::T) == 4 ? 4 : 2;
};

template <class LinksT, class FieldT, class Epi>
__global__ void __launch_bounds__(kShThreads, ShMinBlocks<LinksT>::value) dslash_mrhs_shared_kernel(Geom g, LinksT U, FieldT in, int nrhs,
                                                                          int out_par, Epi epi) {
  using T = typename LinksT::T;
  using A = typename Accum<T>::type;
  __shared__ __align__(16) unsigned char sl_raw[kShWarps * 9 * kShTile * sizeof(cplx<T>)];
  cplx<T>* sl = reinterpret_cast<cplx<T>*>(sl_raw);  // [slot][element][site of the tile]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned run = 0;
  for (int q = 0; q < nrhs; ++q)
    if (epi.sc[q].done == kRunning) run |= 1u << q;
  if (!run) return;  // every block reads the same flags: none of them arrives below
  const int q0 = w, q1 = w + kShWarps;
  const bool act0 = q0 < nrhs && ((run >> q0) & 1u), act1 = q1 < nrhs && ((run >> q1) & 1u);
  A part0 = A(0), part1 = A(0);
  const int mu = w >> 1, back = w & 1;
  const int ntiles = (g.Vh + kShTile - 1) / kShTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int k = tile * kShTile + lane;
    const bool valid = k < g.Vh;
    Site s{};
    int fwd[4] = {0, 0, 0, 0}, bwd[4] = {0, 0, 0, 0};
    if (valid) {
      s = site_of(g, k, out_par);
      neighbours(g, s, fwd, bwd);
      su3<T> L;
      if (!back) {
        L = U.load(out_par, mu, k);
        if constexpr (!LinksT::kFolded) scale(L, T(0.5f * fwd_sign(g, s, mu)));
      } else {
        const su3<T> B = U.load(1 - out_par, mu, bwd[mu]);
        const T c = LinksT::kFolded ? T(-1.0f) : T(-0.5f * bwd_sign(g, s, mu));  // c U^dagger
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            L.e[a][b].re = c * B.e[b][a].re;
            L.e[a][b].im = -(c * B.e[b][a].im);
          }
      }
#pragma unroll
      for (int e = 0; e < 9; ++e) sl[(w * 9 + e) * kShTile + lane] = L.e[e / 3][e % 3];
    }
    __syncthreads();
    if (valid && (act0 || act1)) {
      cvec3<T> acc0, acc1;
      zero(acc0);
      zero(acc1);
      const FieldT in0 = field_at(in, act0 ? q0 : 0), in1 = field_at(in, act1 ? q1 : 0);
#pragma unroll
      for (int slot = 0; slot < kShWarps; ++slot) {
        const int nb = (slot & 1) ? bwd[slot >> 1] : fwd[slot >> 1];
        su3<T> M;
#pragma unroll
        for (int e = 0; e < 9; ++e) M.e[e / 3][e % 3] = sl[(slot * 9 + e) * kShTile + lane];
        if (act0) mul_add(acc0, M, in0.load(nb));
        if (act1) mul_add(acc1, M, in1.load(nb));
      }
      if (act0) epi.site(k, q0, acc0, part0);
      if (act1) epi.site(k, q1, acc1, part1);
    }
    __syncthreads();  // the slots are refilled by the next tile
  }
  // This block's partial for RHS q is warp (q mod kShWarps)'s sum; its writer fences before the
  // barrier, and thread 0 arrives for the block.
  __shared__ bool am_last;
  {
    const double v0 = warp_sum(part0), v1 = warp_sum(part1);
    if (lane == 0) {
      if (q0 < nrhs) epi.partials[(size_t)q0 * kMaxPartials + blockIdx.x] = v0;
      if (q1 < nrhs) epi.partials[(size_t)q1 * kMaxPartials + blockIdx.x] = v1;
      __threadfence();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(&epi.sc[0].counter[Epi::kCounter], 1u) == gridDim.x - 1;
  __syncthreads();
  if (am_last) {
    __shared__ double tot[kMaxRhs];
    mrhs_totals(nrhs, epi.partials, tot);
    // one thread per right-hand side: a serial loop over sixteen updates (dependent global loads and
    // stores, an FP64 division each) kept the summing block's SM busy ~70k cycles after the others
    if (threadIdx.x < nrhs && epi.sc[threadIdx.x].done == kRunning) epi.update(threadIdx.x, tot[threadIdx.x]);
    if (threadIdx.x == 0) epi.sc[0].counter[Epi::kCounter] = 0u;
  }
}

// K1: ap_r = D_oe p_r, alpha_r = rr_r / (|ap_r|^2 + m^2 |p_r|^2)
template <class FieldT>
struct EpiApM {
  static constexpr int kCounter = kCtrK1M;
  FieldT ap;
  CgScalars* sc;
  double* partials;
  template <class T, class A>
  __device__ __forceinline__ void site(int k, int r, const cvec3<T>& acc, A& red) const {
    field_at(ap, r).store(k, acc);
    accum(red, norm2(acc));
  }
  __device__ __forceinline__ void update(int r, double apap) const {
    CgScalars& s = sc[r];
    const double d = apap + s.m2 * s.pp;
    const double alpha = s.rr / d;
    if (!finite_pos(d) || !isfinite(alpha)) s.done = kBreakdown;
    else s.alpha = alpha;
  }
};

// K2: x_r += alpha_r p_r; r_r -= alpha_r (m^2 p_r - D_eo ap_r); beta_r and the exit tests
template <class FieldT, class XFieldT>
struct EpiUpdateM {
  static constexpr int kCounter = kCtrK2M;
  FieldT p, r;
  XFieldT x;
  CgScalars* sc;
  double* partials;
  template <class T, class A>
  __device__ __forceinline__ void site(int k, int q, const cvec3<T>& acc, A& red) const {
    using TX = typename XFieldT::T;
    const T alpha = (T)sc[q].alpha, m2 = (T)sc[q].m2;
    const FieldT pf = field_at(p, q), rf = field_at(r, q);
    const XFieldT xf = field_at(x, q);
    const cvec3<T> pv = pf.load(k);
    cvec3<T> rv = rf.load(k);
    cvec3<TX> xv = xf.load(k);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T at_re = fma(m2, pv.c[a].re, -acc.c[a].re);
      const T at_im = fma(m2, pv.c[a].im, -acc.c[a].im);
      rv.c[a].re = fma(-alpha, at_re, rv.c[a].re);
      rv.c[a].im = fma(-alpha, at_im, rv.c[a].im);
      xv.c[a].re = fma((TX)alpha, (TX)pv.c[a].re, xv.c[a].re);
      xv.c[a].im = fma((TX)alpha, (TX)pv.c[a].im, xv.c[a].im);
    }
    rf.store(k, rv);
    xf.store(k, xv);
    accum(red, norm2(rv));
  }
  __device__ __forceinline__ void update(int q, double rr) const {
    CgScalars& s = sc[q];
    s.iter += 1;
    s.since_ru += 1;
    s.rr_prev = s.rr;
    s.rr = rr;
    if (!isfinite(rr)) {
      s.done = kBreakdown;
      return;
    }
    s.beta = rr / s.rr_prev;
    if (rr > s.rmax2) s.rmax2 = rr;
    if (rr < s.delit) s.done = kConverged;
    else if (s.iter >= s.max_iter) s.done = kMaxIter;
    else if (s.mixed && (s.since_ru >= s.ru_interval || rr < s.delta2 * s.rmax2)) s.done = kReliable;
  }
};

// ---------------------------------------------------------------- driver
template <int PREC, int RECON>
struct MrhsRunner {
  using FieldT = Field<PREC>;
  using XPREC = std::integral_constant<int, x_prec(PREC)>;
  using XFieldT = Field<XPREC::value>;
  const qcd_lattice* lat;
  Geom g;
  CgWork w;
  cudaStream_t st;
  int grid, R, rb;
  long long launches = 0;

  // x-extent of a grid with `gy` rows that stays within one wave of resident blocks of `kernel`
  // (every block ends in a fence + counter update; more waves multiply that cost).
  template <class KernelT>
  int wave_x(KernelT kernel, int gy) const {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    const long long need = (g.Vh + kBlock - 1) / kBlock;
    long long gx = (long long)sms * per_sm / gy;
    if (gx > need) gx = need;
    if (gx > kMaxPartials) gx = kMaxPartials;
    return (int)(gx > 0 ? gx : 1);
  }

  template <int RB>
  void launch_ops(const Links<PREC, RECON>& U, FieldT p, FieldT ap, FieldT r, XFieldT x, cudaEvent_t* ev) {
    const int gy = (R + RB - 1) / RB;
    const dim3 gr(wave_x(dslash_mrhs_cg_kernel<Links<PREC, RECON>, FieldT, RB, EpiUpdateM<FieldT, XFieldT>>, gy), gy);
    if (ev) cudaEventRecord(ev[0], st);
    dslash_mrhs_cg_kernel<Links<PREC, RECON>, FieldT, RB><<<gr, kBlock, 0, st>>>(
        g, U, p, R, QCD_ODD, EpiApM<FieldT>{ap, w.sc, w.partials});
    if (ev) cudaEventRecord(ev[1], st);
    if (ev) cudaEventRecord(ev[2], st);
    dslash_mrhs_cg_kernel<Links<PREC, RECON>, FieldT, RB><<<gr, kBlock, 0, st>>>(
        g, U, ap, R, QCD_EVEN, EpiUpdateM<FieldT, XFieldT>{p, r, x, w.sc, w.partials});
    if (ev) cudaEventRecord(ev[3], st);
  }

  // The shared-link kernel: one wave of its blocks (at most one per tile).
  void launch_shared(const Links<PREC, RECON>& U, FieldT p, FieldT ap, FieldT r, XFieldT x, cudaEvent_t* ev) {
    auto k2 = dslash_mrhs_shared_kernel<Links<PREC, RECON>, FieldT, EpiUpdateM<FieldT, XFieldT>>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2, kShThreads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    long long gx = (long long)sms * per_sm;
    const long long tiles = (g.Vh + kShTile - 1) / kShTile;
    if (gx > tiles) gx = tiles;
    if (gx > kMaxPartials) gx = kMaxPartials;
    if (ev) cudaEventRecord(ev[0], st);
    dslash_mrhs_shared_kernel<Links<PREC, RECON>, FieldT><<<(int)gx, kShThreads, 0, st>>>(
        g, U, p, R, QCD_ODD, EpiApM<FieldT>{ap, w.sc, w.partials});
    if (ev) cudaEventRecord(ev[1], st);
    if (ev) cudaEventRecord(ev[2], st);
    k2<<<(int)gx, kShThreads, 0, st>>>(g, U, ap, R, QCD_EVEN, EpiUpdateM<FieldT, XFieldT>{p, r, x, w.sc, w.partials});
    if (ev) cudaEventRecord(ev[3], st);
  }

  int iteration(cudaEvent_t* ev = nullptr) {
    auto U = make_links<PREC, RECON>(lat->links[PREC].ptr, g.Vh);
    FieldT r = make_field<PREC>(w.r, g.Vh), p = make_field<PREC>(w.p, g.Vh), ap = make_field<PREC>(w.ap, g.Vh);
    XFieldT x = make_field<XPREC::value>(w.x_lo, g.Vh);
    cg_p_mrhs_kernel<<<dim3(wave_x(cg_p_mrhs_kernel<FieldT>, R), R), kBlock, 0, st>>>(g.Vh, r, p, R, w.sc, w.partials);
    constexpr bool wide = PREC == QCD_PREC_DOUBLE || PREC == QCD_PREC_DF64;  // 64-bit accumulators: RB <= 4
    switch (rb) {
      case kRhsShared: launch_shared(U, p, ap, r, x, ev); break;
      case 1: launch_ops<1>(U, p, ap, r, x, ev); break;
      case 2: launch_ops<2>(U, p, ap, r, x, ev); break;
      case 4: launch_ops<4>(U, p, ap, r, x, ev); break;
      case 8: if constexpr (!wide) { launch_ops<8>(U, p, ap, r, x, ev); break; } [[fallthrough]];
      case 16: if constexpr (!wide) { launch_ops<16>(U, p, ap, r, x, ev); break; } [[fallthrough]];
      default: set_error("unsupported RHS block %d for this precision", rb); return QCD_ERR_INVALID_ARG;
    }
    QCD_CUDA(cudaGetLastError());
    launches += 3;
    return QCD_OK;
  }

  CgRunner<PREC, RECON> single(int r) {
    CgRunner<PREC, RECON> c;
    c.lat = lat;
    c.g = g;
    c.w = view(w, r);
    c.st = st;
    c.grid = grid;
    return c;
  }
};

// Default RHS block (when nothing is tuned): the shared-link kernel from kShWarps right-hand sides
// on (fewer leave warps of its blocks idle). Links that fit in half of L2 are read from L2 by
// every grid row, so register blocking buys nothing and costs registers: 1 (measured on GB300 at
// 24^4 x 16 RHS, FP32 recon-12, links 64 MB: 276 ms per solve against 303 ms with 4). Larger link
// fields would be streamed from DRAM once per row: up to 4 RHS per row. (16 RHS in registers take
// 254 registers per thread and run at a tenth of the bandwidth; qcd_tune_mrhs can still choose
// 8 or 16 where they pay.)
inline int default_rhs_block(int prec, int R, size_t links_bytes) {
  (void)prec;
  if (R >= kShWarps) return kRhsShared;
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
      l2 > 0 && links_bytes * 2 <= (size_t)l2)
    return 1;
  const int cap = 4;
  int rb = 1;
  while (rb * 2 <= R && rb * 2 <= cap) rb *= 2;
  if (rb < R && rb * 2 <= cap) rb *= 2;  // one partially filled block beats two passes
  return rb;
}

template <int PREC, int RECON>
int mrhs_typed(qcd_lattice* lat, int R, void* x, const void* b, double mass, double tol, int max_iter,
                      const qcd_solver_opts& o, void* ws, void* y, qcd_solve_info* info, cudaStream_t st) {
  MrhsRunner<PREC, RECON> M;
  M.lat = lat;
  M.g = make_geom(lat);
  M.w = carve(lat, PREC, R, (char*)ws);
  M.st = st;
  M.grid = cg_grid<PREC, RECON>(lat->Vh, 1);
  M.R = R;
  constexpr bool wide = PREC == QCD_PREC_DOUBLE || PREC == QCD_PREC_DF64;  // 64-bit accumulators: RB <= 4
  M.rb = o.rhs_block;  // -1: the shared-link kernel; 0: tuned or default
  if (wide && M.rb > 4) M.rb = 4;
  if (M.rb == 0) {
    // a tuned value read from a cache file is used only if this precision supports it
    std::vector<int> tuned;
    const bool have = tune_lookup(mrhs_key(lat, PREC, RECON, R), &tuned) && !tuned.empty() &&
                      (tuned[0] == kRhsShared || tuned[0] == 1 || tuned[0] == 2 || tuned[0] == 4 ||
                       (!wide && (tuned[0] == 8 || tuned[0] == 16)));
    M.rb = have ? tuned[0] : default_rhs_block(PREC, R, links_bytes(PREC, RECON, lat->Vh));
  }
  const bool mixed = PREC != QCD_PREC_DOUBLE;
  const size_t canon_bytes = (size_t)lat->V * 3 * sizeof(double2);

  std::vector<CgScalars> h(R);
  for (int r = 0; r < R; ++r) {
    CgScalars s{};
    s.m2 = mass * mass;
    s.tol2 = tol * tol;
    s.max_iter = max_iter;
    s.ru_interval = o.reliable_interval > 0 ? o.reliable_interval : 100;
    s.delta2 = o.reliable_delta * o.reliable_delta;
    s.mixed = mixed ? 1 : 0;
    h[r] = s;
  }
  QCD_CUDA(cudaMemcpyAsync(M.w.sc, h.data(), sizeof(CgScalars) * R, cudaMemcpyHostToDevice, st));
  int rc = QCD_OK;
  for (int r = 0; r < R && rc == QCD_OK; ++r) {
    auto c = M.single(r);
    rc = c.init((const char*)b + canon_bytes * r);
    M.launches += c.launches;
  }
  if (rc) return rc;

  const int k = o.check_interval > 0 ? o.check_interval : 8;
  const bool profile = o.profile != 0;
  std::vector<cudaEvent_t> ev(profile ? 4 * k : 0, nullptr);
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  };
  for (auto& e : ev) {
    cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) { cleanup(); return cuda_fail(ce, "cudaEventCreate"); }
  }
  auto ev_at = [&](int i) -> cudaEvent_t* { return profile ? &ev[4 * i] : nullptr; };
  // With a stream the whole loop is one graph launch: a conditional WHILE node whose body is k
  // iterations, every RHS's flag-gated reliable update and a control kernel (as in cg.cu).
  const bool use_graph = o.use_graph && st != nullptr && !profile;
  if (use_graph) {
    QCD_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    QCD_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams params = {};
    params.type = cudaGraphNodeTypeConditional;
    params.conditional.handle = handle;
    params.conditional.type = cudaGraphCondTypeWhile;
    params.conditional.size = 1;
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &params);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaGraphAddNode"); }
    cudaGraph_t body = params.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaStreamBeginCaptureToGraph"); }
    const long long before = M.launches;
    for (int i = 0; i < k && rc == QCD_OK; ++i) rc = M.iteration();
    for (int r = 0; r < R && rc == QCD_OK; ++r) {
      auto c = M.single(r);
      rc = c.reliable_update(true);
    }
    const int max_loops = max_iter / k + 2 * (max_iter / 100 + 1) + 16;
    if (rc == QCD_OK) mrhs_loop_control_kernel<<<1, 32, 0, st>>>(M.w.sc, R, handle, max_loops);
    M.launches = before;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(st, &captured);
    if (rc) { cleanup(); return rc; }
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaStreamEndCapture"); }
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaGraphInstantiate"); }
    e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaGraphLaunch"); }
  }

  int dslash_launches = 0;
  double dslash_ms = 0.0;
  if ((rc = read_scalars(M.w, h.data(), st, R))) { cleanup(); return rc; }
  if (use_graph) {
    int it_max = 0;
    for (int r = 0; r < R; ++r) it_max = std::max(it_max, h[r].iter);
    dslash_launches = 2 * it_max;
    M.launches += (long long)h[0].loops * (3ll * k + (mixed ? 3 : 2) * R + 1);
  }
  while (!use_graph) {
    bool any_running = false, any_ru = false;
    for (int r = 0; r < R; ++r) {
      const int d = h[r].done;
      if (d == kConverged || (mixed && d == kReliable)) {
        auto c = M.single(r);
        if ((rc = c.reliable_update())) { cleanup(); return rc; }
        M.launches += c.launches;
        any_ru = true;
      }
    }
    if (any_ru && (rc = read_scalars(M.w, h.data(), st, R))) { cleanup(); return rc; }
    for (int r = 0; r < R; ++r) any_running |= h[r].done == kRunning;
    if (!any_running) break;
    int iters_before = 0;
    for (int r = 0; r < R; ++r) iters_before = std::max(iters_before, h[r].iter);
    if (use_graph) {
      cudaError_t e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaGraphLaunch"); }
      M.launches += 3ll * k;
    } else {
      for (int i = 0; i < k; ++i)
        if ((rc = M.iteration(ev_at(i)))) { cleanup(); return rc; }
    }
    if ((rc = read_scalars(M.w, h.data(), st, R))) { cleanup(); return rc; }
    int iters_after = 0;
    for (int r = 0; r < R; ++r) iters_after = std::max(iters_after, h[r].iter);
    const int ran = iters_after - iters_before;  // iterations in which some RHS was still active
    dslash_launches += 2 * ran;
    if (profile) {
      for (int i = 0; i < ran && i < k; ++i) {
        float a = 0.f, c2 = 0.f;
        cudaError_t e1 = cudaEventElapsedTime(&a, ev[4 * i], ev[4 * i + 1]);
        cudaError_t e2 = cudaEventElapsedTime(&c2, ev[4 * i + 2], ev[4 * i + 3]);
        if (e1 != cudaSuccess || e2 != cudaSuccess) { cleanup(); return cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaEventElapsedTime"); }
        dslash_ms += (double)a + (double)c2;
      }
    }
  }
  cleanup();
  for (int r = 0; r < R; ++r) {
    auto c = M.single(r);
    void* yr = y ? (char*)y + canon_bytes * r : nullptr;
    if ((rc = c.finish((char*)x + canon_bytes * r, yr))) return rc;
    M.launches += c.launches;
  }
  if ((rc = read_scalars(M.w, h.data(), st, R))) return rc;
  int status = QCD_OK;
  for (int r = 0; r < R; ++r) {
    const CgScalars& s = h[r];
    const double true_rel = s.bb > 0 ? std::sqrt(s.res2 / s.bb) : 0.0;
    int st_r = QCD_OK;
    if (s.done == kBreakdown) st_r = QCD_ERR_BREAKDOWN;
    else if (s.done == kMaxIter || !(true_rel <= tol)) st_r = QCD_ERR_NOT_CONVERGED;
    if (st_r == QCD_ERR_BREAKDOWN || (st_r != QCD_OK && status == QCD_OK)) status = st_r;
    if (info) {
      qcd_solve_info& I = info[r];
      I.iterations = s.iter;
      I.reliable_updates = s.ru_count;
      I.true_rel_residual = true_rel;
      I.iterated_rel_residual = s.bb > 0 ? std::sqrt(s.rr / s.bb) : 0.0;
      I.converged = st_r == QCD_OK;
      I.status = st_r;
      I.kernel_launches = r == 0 ? (int)M.launches : 0;
      I.dslash_launches = r == 0 ? dslash_launches : 0;
      I.dslash_ms = r == 0 ? dslash_ms : 0.0;
    }
  }
  return status;
}

}  // namespace qcd
