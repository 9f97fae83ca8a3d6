// Many independent even-odd CG solves (lattices of uneven sizes, each with its own mass) in ONE
// persistent launch.
//
// The grid is a set of thread-block clusters. Each cluster takes the next lattice from a work
// queue (longest expected solve first) and runs that lattice's entire CG — start-up, the three
// phases of every iteration, FP64 reliable updates, the final y = D_oe x and true residual —
// before taking the next one. There is no grid-wide synchronisation and no host round trip:
// the phases of one lattice are separated by cluster barriers, and the CG scalars are reduced
// over the cluster through distributed shared memory (each CTA writes its block sum into its own
// shared memory; after the barrier every thread adds the C slots in rank order, so every thread
// of the cluster holds bit-identical scalars and takes identical branches).
//
// Fields that are written during the launch are read through L2 (Coherent<>); only the links
// use the read-only path. Every loop is bounded by the lattice's max_iter.
#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "cg_common.cuh"

namespace cg = cooperative_groups;

namespace qcd {

std::string batched_key(int n, qcd_lattice* const* lats, int prec, int recon);
bool tune_lookup(const std::string& key, std::vector<int>* out);

constexpr int kBatchMaxBlock = 256;
constexpr int kMaxCluster = 16;

struct BatchItem {
  Geom g;
  double m2, tol2;
  int max_iter;
  int orig;  // index in the caller's arrays
  const void* U_in;
  const void* U64;
  const double2* b;
  double2* x;
  double2* y;
  void *b_hi, *x_hi, *tmp, *r, *p, *ap, *x_lo;
};

struct BatchResult {
  int iterations, ru_count, status, pad;
  double bb, rr, res2;
};

enum { kBatchOk = 0, kBatchMaxIter = 1, kBatchBreakdown = 2 };

// Cluster-wide deterministic sum (see the file comment). Every thread passes its partial; the
// total is returned in thread 0 of each CTA only (each CTA's thread 0 adds the same C block
// sums in rank order, so all of them hold the same bits). `slots` is double-buffered: a slot is
// rewritten two reductions later, after every CTA has passed the barrier of the one between.
template <class A>
__device__ __forceinline__ double cluster_total(A part, double* slots, int& buf, const cg::cluster_group& cluster) {
  const A x[1] = {part};
  double v[1];
  block_sum<1>(x, v);
  if (threadIdx.x == 0) slots[buf] = v[0];
  // make this phase's global writes visible to the cluster before its barrier
  asm volatile("fence.acq_rel.cluster;" ::: "memory");
  cluster.sync();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int C = (int)cluster.num_blocks();
    for (int r = 0; r < C; ++r) t += *cluster.map_shared_rank(&slots[buf], r);
  }
  buf ^= 1;
  return t;
}

__device__ __forceinline__ void cluster_barrier(const cg::cluster_group& cluster) {
  asm volatile("fence.acq_rel.cluster;" ::: "memory");
  cluster.sync();
}

// CG state of the lattice a cluster is solving: updated by thread 0 of each CTA (identically in
// every CTA of the cluster), read by the other threads after a __syncthreads.
struct BatchState {
  double rr, rr_prev, rmax2, pp, alpha, beta, bb, delit, res2;
  int iter, since_ru, ru_count, status, action;
};
enum { kActRun = 0, kActReliable = 1, kActStop = 2 };

template <int PREC, int RECON>
__global__ void __launch_bounds__(kBatchMaxBlock) batched_cg_kernel(const BatchItem* __restrict__ items,
                                                                    BatchResult* __restrict__ results, int n_items,
                                                                    unsigned* queue, int ru_interval, double delta2) {
  using FieldT = Field<PREC>;
  using T = typename FieldT::T;
  constexpr int XP = x_prec(PREC);
  using XFieldT = Field<XP>;
  using TX = typename XFieldT::T;
  using A = typename Accum<T>::type;
  constexpr bool mixed = PREC != QCD_PREC_DOUBLE;

  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int nthreads = (int)cluster.num_blocks() * blockDim.x;
  const int tid = crank * blockDim.x + threadIdx.x;
  const bool lead = threadIdx.x == 0;
  __shared__ double slots[2];
  __shared__ int item_slot;
  __shared__ BatchState S;
  int buf = 0;

  while (true) {
    if (crank == 0 && lead) item_slot = (int)atomicAdd(queue, 1u);
    cluster.sync();
    const int it = *cluster.map_shared_rank(&item_slot, 0);
    cluster.sync();  // rank 0 may overwrite item_slot only after everyone has read it
    if (it >= n_items) break;
    const BatchItem& I = items[it];
    const Geom g = I.g;
    const int Vh = g.Vh;
    const double m2 = I.m2;
    auto U = make_links<PREC, RECON>(I.U_in, Vh);
    auto U64 = make_links<QCD_PREC_DOUBLE, 18>(I.U64, Vh);
    const Coherent<FieldT> r{make_field<PREC>(I.r, Vh)}, p{make_field<PREC>(I.p, Vh)}, ap{make_field<PREC>(I.ap, Vh)};
    const Coherent<XFieldT> x{make_field<XP>(I.x_lo, Vh)};
    const Coherent<Field<QCD_PREC_DOUBLE>> b_hi{make_field<QCD_PREC_DOUBLE>(I.b_hi, Vh)},
        x_hi{make_field<QCD_PREC_DOUBLE>(I.x_hi, Vh)}, tmp{make_field<QCD_PREC_DOUBLE>(I.tmp, Vh)};

    // ---- start-up: b_hi = b_e, r = b_e, p = 0, x = 0
    double part64 = 0.0;
    for (int k = tid; k < Vh; k += nthreads) {
      const Site s = site_of(g, k, QCD_EVEN);
      cvec3<double> bv;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double2 d = I.b[(size_t)s.lex * 3 + a];
        bv.c[a].re = d.x; bv.c[a].im = d.y;
      }
      b_hi.store(k, bv);
      cvec3<T> bl, z;
      zero(z);
#pragma unroll
      for (int a = 0; a < 3; ++a) { bl.c[a].re = (T)bv.c[a].re; bl.c[a].im = (T)bv.c[a].im; }
      r.store(k, bl);
      p.store(k, z);
      cvec3<TX> zx;
      zero(zx);
      x.store(k, zx);
      if (mixed) {
        cvec3<double> zd;
        zero(zd);
        x_hi.store(k, zd);
      }
      part64 += norm2(bv);
    }
    {
      const double bb = cluster_total(part64, slots, buf, cluster);
      if (lead) {
        S.bb = S.rr = S.rr_prev = S.rmax2 = bb;
        S.pp = S.alpha = S.beta = 0.0;
        S.delit = I.tol2 * bb;
        S.iter = S.since_ru = S.ru_count = 0;
        S.status = isfinite(bb) ? kBatchOk : kBatchBreakdown;
        S.action = (S.status == kBatchOk && bb > 0.0) ? kActRun : kActStop;
      }
      __syncthreads();
    }

    while (S.action != kActStop) {
      if (S.action == kActRun) {
        // K3: p = r + beta p
        const T beta = (T)S.beta;
        A part = 0;
        for (int k = tid; k < Vh; k += nthreads) {
          cvec3<T> rv = r.load(k), pv = p.load(k);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            pv.c[a].re = fma(beta, pv.c[a].re, rv.c[a].re);
            pv.c[a].im = fma(beta, pv.c[a].im, rv.c[a].im);
          }
          p.store(k, pv);
          accum(part, norm2(pv));
        }
        const double pp = cluster_total(part, slots, buf, cluster);
        // K1: ap = D_oe p
        part = 0;
        for (int k = tid; k < Vh; k += nthreads) {
          const auto acc = hop(g, U, p, QCD_ODD, k);
          ap.store(k, acc);
          accum(part, norm2(acc));
        }
        const double apap = cluster_total(part, slots, buf, cluster);
        if (lead) {
          const double d = apap + m2 * pp;
          const double alpha = S.rr / d;
          if (!(isfinite(d) && d > 0.0) || !isfinite(alpha)) {
            S.status = kBatchBreakdown;
            S.action = kActStop;
          } else {
            S.alpha = alpha;
          }
        }
        __syncthreads();
        if (S.action == kActStop) break;
        // K2: x += alpha p; r -= alpha (m^2 p - D_eo ap)
        const T alpha = (T)S.alpha;
        part = 0;
        for (int k = tid; k < Vh; k += nthreads) {
          const auto acc = hop(g, U, ap, QCD_EVEN, k);
          const cvec3<T> pv = p.load(k);
          cvec3<T> rv = r.load(k);
          cvec3<TX> xv = x.load(k);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const T at_re = fma((T)m2, pv.c[a].re, -acc.c[a].re);
            const T at_im = fma((T)m2, pv.c[a].im, -acc.c[a].im);
            rv.c[a].re = fma(-alpha, at_re, rv.c[a].re);
            rv.c[a].im = fma(-alpha, at_im, rv.c[a].im);
            xv.c[a].re = fma((TX)alpha, (TX)pv.c[a].re, xv.c[a].re);
            xv.c[a].im = fma((TX)alpha, (TX)pv.c[a].im, xv.c[a].im);
          }
          r.store(k, rv);
          x.store(k, xv);
          accum(part, norm2(rv));
        }
        const double rr = cluster_total(part, slots, buf, cluster);
        if (lead) {
          S.iter += 1;
          S.since_ru += 1;
          S.rr_prev = S.rr;
          S.rr = rr;
          if (!isfinite(rr)) {
            S.status = kBatchBreakdown;
            S.action = kActStop;
          } else {
            S.beta = rr / S.rr_prev;
            S.rmax2 = fmax(S.rmax2, rr);
            // reliable update (mixed: periodic / delta test; both: to confirm convergence on the
            // true residual)
            if (rr < S.delit || (mixed && (S.since_ru >= ru_interval || rr < delta2 * S.rmax2)))
              S.action = kActReliable;
            else if (S.iter >= I.max_iter) {
              S.status = kBatchMaxIter;
              S.action = kActStop;
            }
          }
        }
        __syncthreads();
      } else {
        // reliable update: x_hi += x_lo, x_lo = 0; r = b - A x_hi in FP64; r_lo <- r
        if (mixed) {
          for (int k = tid; k < Vh; k += nthreads) {
            cvec3<double> xh = x_hi.load(k);
            const cvec3<TX> xl = x.load(k);
#pragma unroll
            for (int a = 0; a < 3; ++a) { xh.c[a].re += (double)xl.c[a].re; xh.c[a].im += (double)xl.c[a].im; }
            x_hi.store(k, xh);
            cvec3<TX> zx;
            zero(zx);
            x.store(k, zx);
          }
        }
        cluster_barrier(cluster);
        for (int k = tid; k < Vh; k += nthreads) tmp.store(k, hop(g, U64, x_hi, QCD_ODD, k));
        cluster_barrier(cluster);
        part64 = 0.0;
        for (int k = tid; k < Vh; k += nthreads) {
          const auto acc = hop(g, U64, tmp, QCD_EVEN, k);
          const cvec3<double> bv = b_hi.load(k), xv = x_hi.load(k);
          cvec3<double> rv;
          cvec3<T> rl;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            rv.c[a].re = bv.c[a].re - fma(m2, xv.c[a].re, -acc.c[a].re);
            rv.c[a].im = bv.c[a].im - fma(m2, xv.c[a].im, -acc.c[a].im);
            rl.c[a].re = (T)rv.c[a].re;
            rl.c[a].im = (T)rv.c[a].im;
          }
          r.store(k, rl);
          part64 += norm2(rv);
        }
        const double rt = cluster_total(part64, slots, buf, cluster);
        if (lead) {
          if (!isfinite(rt)) {
            S.status = kBatchBreakdown;
            S.action = kActStop;
          } else {
            S.beta = rt / S.rr_prev;
            S.rr = rt;
            S.rmax2 = rt;
            S.since_ru = 0;
            S.ru_count += 1;
            if (rt < S.delit) {
              S.action = kActStop;
            } else if (S.iter >= I.max_iter) {
              S.status = kBatchMaxIter;
              S.action = kActStop;
            } else {
              S.action = kActRun;
            }
          }
        }
        __syncthreads();
      }
    }

    // ---- finish: fold x_lo into x_hi, y = D_oe x, true residual, canonical outputs
    if (mixed) {
      for (int k = tid; k < Vh; k += nthreads) {
        cvec3<double> xh = x_hi.load(k);
        const cvec3<TX> xl = x.load(k);
#pragma unroll
        for (int a = 0; a < 3; ++a) { xh.c[a].re += (double)xl.c[a].re; xh.c[a].im += (double)xl.c[a].im; }
        x_hi.store(k, xh);
        cvec3<TX> zx;
        zero(zx);
        x.store(k, zx);
      }
    }
    cluster_barrier(cluster);
    for (int k = tid; k < Vh; k += nthreads) tmp.store(k, hop(g, U64, x_hi, QCD_ODD, k));
    cluster_barrier(cluster);
    part64 = 0.0;
    for (int k = tid; k < Vh; k += nthreads) {
      const auto acc = hop(g, U64, tmp, QCD_EVEN, k);
      const cvec3<double> bv = b_hi.load(k), xv = x_hi.load(k), yv = tmp.load(k);
      cvec3<double> rv;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        rv.c[a].re = bv.c[a].re - fma(m2, xv.c[a].re, -acc.c[a].re);
        rv.c[a].im = bv.c[a].im - fma(m2, xv.c[a].im, -acc.c[a].im);
      }
      part64 += norm2(rv);
      const Site se = site_of(g, k, QCD_EVEN), so = site_of(g, k, QCD_ODD);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        I.x[(size_t)se.lex * 3 + a] = make_double2(xv.c[a].re, xv.c[a].im);
        I.x[(size_t)so.lex * 3 + a] = make_double2(0.0, 0.0);
        if (I.y) {
          I.y[(size_t)so.lex * 3 + a] = make_double2(yv.c[a].re, yv.c[a].im);
          I.y[(size_t)se.lex * 3 + a] = make_double2(0.0, 0.0);
        }
      }
    }
    const double res2 = cluster_total(part64, slots, buf, cluster);
    if (crank == 0 && lead) {
      BatchResult res;
      res.iterations = S.iter;
      res.ru_count = S.ru_count;
      res.status = S.status;
      res.pad = 0;
      res.bb = S.bb;
      res.rr = S.rr;
      res.res2 = res2;
      results[it] = res;
    }
    __syncthreads();  // S is rewritten for the next lattice only after every thread is past it
  }
}

// ---------------------------------------------------------------- host side
struct BatchLayout {
  BatchItem* items;
  BatchResult* results;
  unsigned* queue;
  std::vector<size_t> field_off;  // per lattice: offset of its first field
  size_t total;
};

static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// Per lattice: b_hi, x_hi, tmp (FP64), r, p, ap (inner), x_lo (FP32, mixed only).
static size_t lattice_fields_bytes(const qcd_lattice* lat, int prec) {
  const size_t f64 = a256(field_bytes(QCD_PREC_DOUBLE, lat->Vh));
  const size_t fin = a256(field_bytes(prec, lat->Vh));
  const size_t fx = prec == QCD_PREC_DOUBLE ? 0 : a256(field_bytes(x_prec(prec), lat->Vh));
  return 3 * f64 + 3 * fin + fx;
}

static BatchLayout batch_layout(int n, const qcd_lattice* const* lats, int prec, char* base) {
  BatchLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += a256(bytes); return o; };
  const size_t o_items = take(sizeof(BatchItem) * n);
  const size_t o_res = take(sizeof(BatchResult) * n);
  const size_t o_q = take(sizeof(unsigned));
  L.field_off.resize(n);
  for (int i = 0; i < n; ++i) L.field_off[i] = take(lattice_fields_bytes(lats[i], prec));
  L.total = off;
  L.items = base ? (BatchItem*)(base + o_items) : nullptr;
  L.results = base ? (BatchResult*)(base + o_res) : nullptr;
  L.queue = base ? (unsigned*)(base + o_q) : nullptr;
  return L;
}

size_t batch_workspace_bytes(int n, const qcd_lattice* const* lats, int prec) {
  return batch_layout(n, lats, prec, nullptr).total;
}

template <int PREC, int RECON>
static int batched_typed(int n, qcd_lattice* const* lats, void* const* x, const void* const* b, void* const* y,
                         const double* mass, double tol, int max_iter, const qcd_solver_opts& o, void* ws,
                         qcd_solve_info* info, cudaStream_t st) {
  char* base = (char*)ws;
  BatchLayout L = batch_layout(n, lats, PREC, base);
  std::vector<BatchItem> items(n);
  for (int i = 0; i < n; ++i) {
    const qcd_lattice* lat = lats[i];
    BatchItem& I = items[i];
    I.g = make_geom(lat);
    I.m2 = mass[i] * mass[i];
    I.tol2 = tol * tol;
    I.max_iter = max_iter;
    I.orig = i;
    I.U_in = lat->links[PREC].ptr;
    I.U64 = lat->links[QCD_PREC_DOUBLE].ptr;
    I.b = (const double2*)b[i];
    I.x = (double2*)x[i];
    I.y = y ? (double2*)y[i] : nullptr;
    char* f = base + L.field_off[i];
    const size_t f64 = a256(field_bytes(QCD_PREC_DOUBLE, lat->Vh));
    const size_t fin = a256(field_bytes(PREC, lat->Vh));
    I.b_hi = f; f += f64;
    I.x_hi = f; f += f64;
    I.tmp = f; f += f64;
    I.r = f; f += fin;
    I.p = f; f += fin;
    I.ap = f; f += fin;
    I.x_lo = PREC == QCD_PREC_DOUBLE ? I.x_hi : (void*)f;
  }
  // longest expected solve first: cost ~ sites / mass (CG iterations grow like 1/m)
  std::stable_sort(items.begin(), items.end(), [](const BatchItem& a, const BatchItem& c) {
    return (double)a.g.Vh / std::sqrt(a.m2) > (double)c.g.Vh / std::sqrt(c.m2);
  });

  int C = o.cluster_size, block = o.block_size;
  if (C <= 0 || block <= 0) {
    std::vector<int> tuned;
    const bool have = tune_lookup(batched_key(n, lats, PREC, RECON), &tuned) && tuned.size() >= 2;
    if (C <= 0) C = have ? tuned[0] : 4;
    if (block <= 0) block = have ? tuned[1] : 256;
  }
  if (C > kMaxCluster || (C & (C - 1))) { set_error("cluster_size must be a power of two <= %d", kMaxCluster); return QCD_ERR_INVALID_ARG; }
  if (block > kBatchMaxBlock || block < 32 || (block & 31)) { set_error("block_size must be a multiple of 32 in [32, %d]", kBatchMaxBlock); return QCD_ERR_INVALID_ARG; }
  auto kern = batched_cg_kernel<PREC, RECON>;
  if (C > 8) QCD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));

  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_clusters = 0;
  cfg.gridDim = dim3(C);
  QCD_CUDA(cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg));
  if (max_clusters < 1) { set_error("a cluster of %d blocks of %d threads does not fit on this GPU", C, block); return QCD_ERR_UNSUPPORTED; }
  const int nclusters = std::min(n, max_clusters);
  cfg.gridDim = dim3(nclusters * C);
  const int ru_interval = o.reliable_interval > 0 ? o.reliable_interval : 100;
  const double delta2 = o.reliable_delta * o.reliable_delta;

  auto enqueue = [&]() -> int {
    QCD_CUDA(cudaMemcpyAsync(L.items, items.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice, st));
    QCD_CUDA(cudaMemsetAsync(L.queue, 0, sizeof(unsigned), st));
    QCD_CUDA(cudaLaunchKernelEx(&cfg, kern, (const BatchItem*)L.items, L.results, n, L.queue, ru_interval, delta2));
    return QCD_OK;
  };
  int rc = QCD_OK;
  if (o.use_graph && st != nullptr) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    QCD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    rc = enqueue();
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    QCD_CUDA(e);
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    QCD_CUDA(e);
    QCD_CUDA(e2);
  } else {
    if ((rc = enqueue())) return rc;
  }
  std::vector<BatchResult> res(n);
  QCD_CUDA(cudaMemcpyAsync(res.data(), L.results, sizeof(BatchResult) * n, cudaMemcpyDeviceToHost, st));
  QCD_CUDA(cudaStreamSynchronize(st));
  int status = QCD_OK;
  for (int j = 0; j < n; ++j) {
    const int i = items[j].orig;
    const BatchResult& R = res[j];
    const double true_rel = R.bb > 0 ? std::sqrt(R.res2 / R.bb) : 0.0;
    int s = QCD_OK;
    if (R.status == kBatchBreakdown) s = QCD_ERR_BREAKDOWN;
    else if (R.status == kBatchMaxIter || !(true_rel <= tol)) s = QCD_ERR_NOT_CONVERGED;
    if (s == QCD_ERR_BREAKDOWN || (s != QCD_OK && status == QCD_OK)) status = s;
    if (info) {
      qcd_solve_info& I = info[i];
      I.iterations = R.iterations;
      I.reliable_updates = R.ru_count;
      I.true_rel_residual = true_rel;
      I.iterated_rel_residual = R.bb > 0 ? std::sqrt(R.rr / R.bb) : 0.0;
      I.converged = s == QCD_OK;
      I.status = s;
      I.kernel_launches = i == 0 ? 1 : 0;
    }
  }
  return status;
}

int run_cg_batched(int n, qcd_lattice* const* lats, void* const* x, const void* const* b, void* const* y,
                   const double* mass, double tol, int max_iter, const qcd_solver_opts& o, void* ws,
                   qcd_solve_info* info, cudaStream_t st) {
  const int prec = o.prec_inner;
  const int recon = lats[0]->links[prec].recon;
  if (prec == QCD_PREC_DOUBLE && recon == 18) return batched_typed<QCD_PREC_DOUBLE, 18>(n, lats, x, b, y, mass, tol, max_iter, o, ws, info, st);
  if (prec == QCD_PREC_SINGLE && recon == 18) return batched_typed<QCD_PREC_SINGLE, 18>(n, lats, x, b, y, mass, tol, max_iter, o, ws, info, st);
  if (prec == QCD_PREC_SINGLE && recon == 12) return batched_typed<QCD_PREC_SINGLE, 12>(n, lats, x, b, y, mass, tol, max_iter, o, ws, info, st);
  if (prec == QCD_PREC_HALF && recon == 12) return batched_typed<QCD_PREC_HALF, 12>(n, lats, x, b, y, mass, tol, max_iter, o, ws, info, st);
  if (prec == QCD_PREC_DF64 && recon == 18) return batched_typed<QCD_PREC_DF64, 18>(n, lats, x, b, y, mass, tol, max_iter, o, ws, info, st);
  return QCD_ERR_UNSUPPORTED;
}

}  // namespace qcd
