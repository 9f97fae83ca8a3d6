#pragma once
// The half-lattice hop with its inputs staged in shared memory by bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier) — for the FP32 recon-12 operator of the mixed CG, which
// is bound by memory latency when every thread gathers its own links and neighbours.
//
// The output sites are cut into tiles of kStageSites consecutive even-odd indices. In the even-odd
// layout the neighbours of a tile in direction mu are (up to the lattice wrap) again a contiguous
// run: for mu >= 1 the tile shifted by +-h_mu = +-(L0 ... L_{mu-1}) / 2, for mu = 0 the tile widened by
// one site. So one warp of the block issues, per tile, bulk copies of
//   the forward links of the tile (own sites), and per mu and direction
//   the backward links and the neighbour colour vectors of the shifted run,
// into one of two shared-memory stages, while the block computes the previous tile from the other.
// A neighbour outside its staged run (the wrap at a lattice boundary, or a run clamped at the ends
// of the index range) is read from global memory instead. Bulk copies need 16-byte aligned sources
// and sizes: the 8-byte vector planes are staged from an even index to an even index.
//
// Every wait on an mbarrier is bounded (clock64); on expiry the kernel waits (bounded again) for the
// copies it issued, records a fault in the CG scalars (2 when that drain gave up as well), and
// returns. Once a fault is set the launch's outputs are undefined.
//
// Measured on GB300 (32^4, FP32 recon-12): 123 us per operator launch against 52 us for the
// direct-load kernel. Each site needs ~600 staged bytes (every neighbour vector is staged once per
// direction run), so two stages of 64 sites fill the shared memory of two blocks per SM: 4 warps per
// SM compute where the direct kernel keeps ~29 in flight, and the per-tile copy latency shows. It is
// therefore opt-in (qcd_solver_opts.staged); four-dimensional tiles with halos would be needed to
// cut the staged bytes per site.
#include <cstdint>

#include "dslash.cuh"

namespace qcd {

constexpr int kStageSites = 64;                  // sites per tile = threads per block
constexpr int kStageRun = kStageSites + 4;       // room for a shifted, widened and aligned run
constexpr long long kWaitCycles = 4000000000ll;  // default wait limit: about 2 s at 2 GHz

// shared-memory layout of one stage (FP32 recon-12 links: 3 float4 planes; FP32 vectors: 3 float2)
struct StageFp32R12 {
  float4 lf[4][3][kStageSites];  // forward links of the tile's own sites
  float4 lb[4][3][kStageRun];    // backward links (at the backward neighbours)
  float2 vf[4][3][kStageRun];    // forward neighbour vectors
  float2 vb[4][3][kStageRun];    // backward neighbour vectors
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// non-suspending test of the phase with the given parity (the caller polls against a clock limit)
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// bounded wait (limit in SM clock cycles); false when it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_test_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// The index runs of one tile [k0, k1): forward (f) and backward (b) neighbours per mu, clamped to
// [0, Vh). Links are 16-byte elements (any start); vectors are 8-byte elements staged from even to
// even indices. Every thread derives the same runs from the tile, so no run table is shared.
struct TileRuns {
  int flo[4], fhi[4], blo[4], bhi[4];      // neighbour runs (link elements)
  int vflo[4], vfhi[4], vblo[4], vbhi[4];  // the same runs widened to even bounds (vector elements)
};

__device__ __forceinline__ TileRuns tile_runs(const Geom& g, int k0, int k1) {
  TileRuns r;
  const int h[4] = {0, g.L0 / 2, g.L0 * g.L1 / 2, g.L0 * g.L1 * g.L2 / 2};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int flo = min(max(mu == 0 ? k0 : k0 + h[mu], 0), g.Vh);
    const int blo = min(max(mu == 0 ? k0 - 1 : k0 - h[mu], 0), g.Vh);
    const int fhi = min(max(mu == 0 ? k1 + 1 : k1 + h[mu], flo), g.Vh);  // flo <= fhi <= Vh
    const int bhi = min(max(mu == 0 ? k1 : k1 - h[mu], blo), g.Vh);
    r.flo[mu] = flo; r.fhi[mu] = fhi;
    r.blo[mu] = blo; r.bhi[mu] = bhi;
    // even bounds for the 8-byte vector planes; Vh is even, so vlo <= lo <= hi <= vhi <= Vh
    r.vflo[mu] = flo & ~1; r.vfhi[mu] = min((fhi + 1) & ~1, g.Vh);
    r.vblo[mu] = blo & ~1; r.vbhi[mu] = min((bhi + 1) & ~1, g.Vh);
  }
  return r;
}

// Issue the bulk copies of tile [k0, k1) into stage `st` (called by one full warp).
__device__ __forceinline__ void issue_tile_fp32r12(const Geom& g, const Links<QCD_PREC_SINGLE, 12>& U,
                                                  const Field<QCD_PREC_SINGLE>& in, int out_par, int k0, int k1,
                                                  StageFp32R12* st, uint64_t* bar) {
  const int lane = threadIdx.x & 31;
  const TileRuns r = tile_runs(g, k0, k1);
  const int in_par = 1 - out_par;
  unsigned bytes = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
    bytes += 3u * (16u * (unsigned)(k1 - k0) + 16u * (unsigned)(r.bhi[mu] - r.blo[mu]) +
                   8u * (unsigned)(r.vfhi[mu] - r.vflo[mu]) + 8u * (unsigned)(r.vbhi[mu] - r.vblo[mu]));
  if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
  __syncwarp();
  // 48 copies: (mu, plane, kind) spread over the 32 lanes
  for (int j = lane; j < 48; j += 32) {
    const int mu = j / 12, c = (j / 4) % 3, kind = j % 4;
    if (kind == 0) {
      const float4* src = U.p + ((size_t)(out_par * 4 + mu) * 3 + c) * U.Vh + k0;
      bulk_g2s(st->lf[mu][c], src, 16u * (unsigned)(k1 - k0), bar);
    } else if (kind == 1) {
      if (r.bhi[mu] > r.blo[mu]) {
        const float4* src = U.p + ((size_t)(in_par * 4 + mu) * 3 + c) * U.Vh + r.blo[mu];
        bulk_g2s(st->lb[mu][c], src, 16u * (unsigned)(r.bhi[mu] - r.blo[mu]), bar);
      }
    } else if (kind == 2) {
      if (r.vfhi[mu] > r.vflo[mu])
        bulk_g2s(st->vf[mu][c], in.p + (size_t)c * in.Vh + r.vflo[mu], 8u * (unsigned)(r.vfhi[mu] - r.vflo[mu]), bar);
    } else {
      if (r.vbhi[mu] > r.vblo[mu])
        bulk_g2s(st->vb[mu][c], in.p + (size_t)c * in.Vh + r.vblo[mu], 8u * (unsigned)(r.vbhi[mu] - r.vblo[mu]), bar);
    }
  }
}

__device__ __forceinline__ su3<float> link_from_planes(float4 q0, float4 q1, float4 q2) {
  su3<float> U;
  U.e[0][0] = {q0.x, q0.y}; U.e[0][1] = {q0.z, q0.w};
  U.e[0][2] = {q1.x, q1.y}; U.e[1][0] = {q1.z, q1.w};
  U.e[1][1] = {q2.x, q2.y}; U.e[1][2] = {q2.z, q2.w};
  reconstruct_row2(U);
  return U;
}

// The hop of site k (tile-local j) from the staged stage, falling back to global memory outside the runs.
__device__ __forceinline__ cvec3<float> hop_staged_fp32r12(const Geom& g, const Links<QCD_PREC_SINGLE, 12>& U,
                                                           const Field<QCD_PREC_SINGLE>& in, int out_par, int k, int j,
                                                           const TileRuns& r, const StageFp32R12* st) {
  const Site s = site_of(g, k, out_par);
  int fwd[4], bwd[4];
  neighbours(g, s, fwd, bwd);
  cvec3<float> acc;
  zero(acc);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const su3<float> Uf = link_from_planes(st->lf[mu][0][j], st->lf[mu][1][j], st->lf[mu][2][j]);
    cvec3<float> xf;
    if (fwd[mu] >= r.vflo[mu] && fwd[mu] < r.vfhi[mu]) {
      const int o = fwd[mu] - r.vflo[mu];
#pragma unroll
      for (int a = 0; a < 3; ++a) xf.c[a] = {st->vf[mu][a][o].x, st->vf[mu][a][o].y};
    } else {
      xf = in.load(fwd[mu]);
    }
    axpy(acc, 0.5f * fwd_sign(g, s, mu), mul(Uf, xf));
    su3<float> Ub;
    if (bwd[mu] >= r.blo[mu] && bwd[mu] < r.bhi[mu]) {
      const int o = bwd[mu] - r.blo[mu];
      Ub = link_from_planes(st->lb[mu][0][o], st->lb[mu][1][o], st->lb[mu][2][o]);
    } else {
      Ub = U.load(1 - out_par, mu, bwd[mu]);
    }
    cvec3<float> xb;
    if (bwd[mu] >= r.vblo[mu] && bwd[mu] < r.vbhi[mu]) {
      const int o = bwd[mu] - r.vblo[mu];
#pragma unroll
      for (int a = 0; a < 3; ++a) xb.c[a] = {st->vb[mu][a][o].x, st->vb[mu][a][o].y};
    } else {
      xb = in.load(bwd[mu]);
    }
    axpy(acc, -0.5f * bwd_sign(g, s, mu), adj_mul(Ub, xb));
  }
  return acc;
}

// the epilogue's prefetched own-site operands (an empty stand-in when it prefetches nothing)
template <class Epi, bool P = Epi::kPrefetch>
struct PreOf {
  using type = int;
};
template <class Epi>
struct PreOf<Epi, true> {
  using type = typename Epi::Pre;
};

// Persistent staged operator kernel: block b takes tiles b, b + grid, ...; stage i & 1 holds tile i.
// `fault` (nullable) receives 1 if a wait on the copies of a tile exceeds `wait_cycles`.
template <class Epi>
__global__ void __launch_bounds__(kStageSites) dslash_staged_fp32r12_kernel(Geom g, Links<QCD_PREC_SINGLE, 12> U,
                                                                           Field<QCD_PREC_SINGLE> in, int out_par, Epi epi,
                                                                           int* fault, long long wait_cycles) {
  if (epi.skip() || (fault && *(volatile int*)fault)) return;  // an earlier launch already gave up
  extern __shared__ __align__(128) unsigned char stage_mem[];
  StageFp32R12* stages = reinterpret_cast<StageFp32R12*>(stage_mem);
  __shared__ __align__(8) uint64_t bar[2];
  using A = typename Accum<float>::type;
  A red[Epi::NV > 0 ? Epi::NV : 1];
#pragma unroll
  for (int q = 0; q < (Epi::NV > 0 ? Epi::NV : 1); ++q) red[q] = A(0);
  const int ntiles = (g.Vh + kStageSites - 1) / kStageSites;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool producer = threadIdx.x < 32;
  int tile = blockIdx.x;
  if (tile < ntiles && producer)
    issue_tile_fp32r12(g, U, in, out_par, tile * kStageSites, min(tile * kStageSites + kStageSites, g.Vh), &stages[0],
                       &bar[0]);
  unsigned phase[2] = {0u, 0u};
  bool in_flight[2] = {tile < ntiles, false};  // stages whose copies were issued and not yet waited for
  bool ok = true;
  for (int i = 0; tile < ntiles; ++i, tile += gridDim.x) {
    const int sidx = i & 1;
    const int next = tile + gridDim.x;
    if (next < ntiles) {
      if (producer)
        issue_tile_fp32r12(g, U, in, out_par, next * kStageSites, min(next * kStageSites + kStageSites, g.Vh),
                           &stages[sidx ^ 1], &bar[sidx ^ 1]);
      in_flight[sidx ^ 1] = true;
    }
    const int k0 = tile * kStageSites, k1 = min(k0 + kStageSites, g.Vh);
    const int k = k0 + (int)threadIdx.x;
    const bool valid = k < k1;
    typename PreOf<Epi>::type pre{};
    if constexpr (Epi::kPrefetch) {
      if (valid) pre = epi.prefetch(k);  // own-site epilogue operands: their latency overlaps the wait
    }
    const bool waited = mbar_wait_bounded(&bar[sidx], phase[sidx], wait_cycles);
    if (__syncthreads_or(!waited)) { ok = false; break; }  // block-uniform: every thread leaves together
    in_flight[sidx] = false;
    phase[sidx] ^= 1u;
    if (valid) {
      const TileRuns r = tile_runs(g, k0, k1);
      auto acc = hop_staged_fp32r12(g, U, in, out_par, k, (int)threadIdx.x, r, &stages[sidx]);
      if constexpr (Epi::kPrefetch) epi.site_pre(k, acc, red, pre);
      else epi.site(k, acc, red);
    }
    __syncthreads();  // stage sidx is refilled by the next iteration's copies
  }
  if (!ok) {
    // let the copies this block issued land before its shared memory is released (bounded again, by
    // the default limit whatever the caller's)
    bool drained = true;
    for (int q = 0; q < 2; ++q)
      if (in_flight[q] && !mbar_wait_bounded(&bar[q], phase[q], kWaitCycles)) drained = false;
    // 1: a wait gave up and the block's copies landed; 2: the drain gave up too, so copies may still
    // be landing in shared memory that a later block of this launch owns. Either way the launch's
    // outputs are undefined and the solve stops with QCD_ERR_TIMEOUT.
    if (fault && threadIdx.x == 0) atomicMax(fault, drained ? 1 : 2);
    return;
  }
  if constexpr (Epi::NV > 0) epi.finish(red);
}

}  // namespace qcd
