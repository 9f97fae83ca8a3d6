// Conjugate gradient on the even-site normal operator A = m^2 - D_eo D_oe (the paper's congrad, §4).
//
// One iteration is three kernels, with every CG scalar kept on the device:
//   K3  p = r + beta p (a plain axpy)
//   K1  ap = D_oe p            (fused store), partials <ap,ap>, <p,p> -> alpha = rr / (<ap,ap> + m^2 <p,p>)
//   K2  t = D_eo ap; x += alpha p; r -= alpha (m^2 p - t), partial <r,r> -> beta, exit test
// (the paper's order with its final "p = r + beta p" moved to the start of the next iteration;
// the first K3 runs with beta = 0 and p = 0, giving p = r = b).
// The grid reductions are deterministic: each block writes an FP64 partial, the block that
// finishes last sums them in index order and updates the scalars.
//
// The host reads the device-side status every `check_interval` iterations (the paper copies
// betan to the host on every iteration); the k-iteration chunk is replayed as a CUDA graph.
//
// Mixed precision (prec_inner = SINGLE or HALF): the recursion runs on low-precision fields with
// FP32 arithmetic and FP64 reductions; x accumulates in FP32 since the last reliable update,
// and a reliable update (x_hi += x_lo; r = b - A x_hi in FP64) replaces the iterated residual
// every `reliable_interval` iterations, when |r| drops below reliable_delta * max|r| since the
// previous update, and whenever the iterated residual meets the tolerance.
#include <chrono>
#include <cmath>
#include <vector>

#include "cg_common.cuh"

namespace qcd {

// Build the device-side solve loop: graph = { WHILE(cond) { k x (K3, K1, K2); gated reliable
// update; control } }. The condition starts at 1 on every launch; the control kernel clears it
// when the recursion stops (converged on the true residual, max_iter, breakdown) or after a
// guard number of passes.
template <int PREC, int RECON>
static int device_loop(CgRunner<PREC, RECON>& R, int k, int max_iter, cudaGraphExec_t& exec, cudaGraph_t& graph) {
  QCD_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  QCD_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams params = {};
  params.type = cudaGraphNodeTypeConditional;
  params.conditional.handle = handle;
  params.conditional.type = cudaGraphCondTypeWhile;
  params.conditional.size = 1;
  cudaGraphNode_t node;
  QCD_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &params));
  cudaGraph_t body = params.conditional.phGraph_out[0];
  QCD_CUDA(cudaStreamBeginCaptureToGraph(R.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = QCD_OK;
  for (int i = 0; i < k && rc == QCD_OK; ++i) rc = R.iteration();
  if (rc == QCD_OK) rc = R.reliable_update(true);
  const int max_loops = max_iter / k + 2 * (max_iter / 100 + 1) + 16;
  if (rc == QCD_OK) {
    cg_loop_control_kernel<<<1, 1, 0, R.st>>>(R.w.sc, handle, max_loops);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) rc = cuda_fail(le, "cg_loop_control_kernel");
  }
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(R.st, &captured);
  if (rc) return rc;
  QCD_CUDA(e);
  QCD_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  return QCD_OK;
}

template <int PREC, int RECON>
static int cg_typed(qcd_lattice* lat, void* x, const void* b, double mass, double tol, int max_iter,
                    const qcd_solver_opts& o, void* ws, void* y, qcd_solve_info* info, cudaStream_t st) {
  CgRunner<PREC, RECON> R;
  R.lat = lat;
  R.g = make_geom(lat);
  R.w = carve(lat, PREC, 1, (char*)ws);
  R.st = st;
  R.tps = threads_per_site(PREC, lat->Vh);
  const int wave = cg_grid<PREC, RECON>(lat->Vh, R.tps);
  cg_launch_shape((long long)lat->Vh * R.tps, wave, &R.grid, &R.block);
  // The FP64 and df64 operators are bound by the FP64 / FP32 pipes: on lattices of more than one
  // wave, a grid of several waves lets the block scheduler even out SMs that run at different
  // speeds (measured on GB300: FP64 32^4 1830 -> 1757 ms and 24^4 139 -> 127 ms with two waves;
  // df64 32^4 907 -> 880 ms with four). Below one wave the spread shape above stays.
  constexpr int kWaves = PREC == QCD_PREC_DOUBLE ? 2 : (PREC == QCD_PREC_DF64 ? 4 : 1);
  if (kWaves > 1 && R.block == kBlock && R.grid == wave) {
    const long long need = ((long long)lat->Vh * R.tps + kBlock - 1) / kBlock;
    long long gg = (long long)wave * kWaves;
    if (gg > need) gg = need;
    if (gg > kMaxPartials) gg = kMaxPartials;
    R.grid = (int)gg;
  }
  R.setup_staged(o.staged != 0);
  R.stream_in = stream_links(PREC, RECON, lat->Vh);
  R.stream64 = stream_links(QCD_PREC_DOUBLE, 18, lat->Vh);
  R.wait_cycles = o.wait_cycles > 0 ? o.wait_cycles : kWaitCycles;
  const bool mixed = PREC != QCD_PREC_DOUBLE;

  CgScalars h{};
  h.m2 = mass * mass;
  h.tol2 = tol * tol;
  h.max_iter = max_iter;
  h.ru_interval = o.reliable_interval > 0 ? o.reliable_interval : 100;
  h.delta2 = o.reliable_delta * o.reliable_delta;
  h.mixed = mixed ? 1 : 0;
  QCD_CUDA(cudaMemcpyAsync(R.w.sc, &h, sizeof(CgScalars), cudaMemcpyHostToDevice, st));
  int rc = R.init(b);
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
  // Events recorded inside a graph cannot be timed, so profiling runs the chunk as direct launches.
  const bool use_graph = o.use_graph && st != nullptr && !profile;
  int status = QCD_OK;
  int dslash_launches = 0;
  double dslash_ms = 0.0;
  if (use_graph) {
    // The whole solve loop is ONE graph launch: a conditional WHILE node whose body runs k
    // iterations, the (flag-gated) reliable update and the control kernel that decides whether
    // to loop again. The host waits once, at the end.
    if ((rc = device_loop(R, k, max_iter, exec, graph))) { cleanup(); return rc; }
    cudaError_t e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaGraphLaunch"); }
    if ((rc = read_scalars(R.w, &h, st))) { cleanup(); return rc; }
    if (h.done == kBreakdown) status = QCD_ERR_BREAKDOWN;
    else if (h.done != kTrueConverged) status = QCD_ERR_NOT_CONVERGED;
    R.launches += (long long)h.loops * ((long long)R.launches_per_iteration() * k + (mixed ? 3 : 2) + 1);
    dslash_launches = 2 * h.iter;
  } else {
    if ((rc = read_scalars(R.w, &h, st))) { cleanup(); return rc; }
  }
  while (!use_graph) {
    if (h.fault) break;  // reported below as QCD_ERR_TIMEOUT
    if (h.done == kBreakdown) { status = QCD_ERR_BREAKDOWN; break; }
    if (h.done == kMaxIter) { status = QCD_ERR_NOT_CONVERGED; break; }
    if (h.done == kTrueConverged) break;
    if (h.done == kConverged || (mixed && h.done == kReliable)) {
      rc = R.reliable_update();
      if (rc) { cleanup(); return rc; }
      if ((rc = read_scalars(R.w, &h, st))) { cleanup(); return rc; }
      continue;
    }
    if (h.iter >= max_iter) { status = QCD_ERR_NOT_CONVERGED; break; }
    const int iter_before = h.iter;
    for (int i = 0; i < k; ++i) {
      if ((rc = R.iteration(ev_at(i)))) { cleanup(); return rc; }
    }
    if ((rc = read_scalars(R.w, &h, st))) { cleanup(); return rc; }
    // the iterations that did work in this chunk: the rest returned at once on the done flag
    const int ran = h.iter - iter_before;
    dslash_launches += 2 * ran;
    if (profile) {
      for (int i = 0; i < ran && i < k; ++i) {
        float a = 0.f, b = 0.f;
        cudaError_t e1 = cudaEventElapsedTime(&a, ev[4 * i], ev[4 * i + 1]);
        cudaError_t e2 = cudaEventElapsedTime(&b, ev[4 * i + 2], ev[4 * i + 3]);
        if (e1 != cudaSuccess || e2 != cudaSuccess) { cleanup(); return cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaEventElapsedTime"); }
        dslash_ms += (double)a + (double)b;
      }
    }
  }
  cleanup();
  if ((rc = R.finish(x, y))) return rc;
  if ((rc = read_scalars(R.w, &h, st))) return rc;
  const double true_rel = h.bb > 0 ? std::sqrt(h.res2 / h.bb) : 0.0;
  if (h.fault) {
    set_error(h.fault == 1 ? "a bounded device-side wait in the staged operator gave up"
                           : "a bounded device-side wait in the staged operator gave up, and so did the wait for "
                             "its bulk copies in flight (the launch's outputs are undefined)");
    status = QCD_ERR_TIMEOUT;
  } else if (status == QCD_OK && !(true_rel <= tol)) {
    // The recursion met the tolerance but the FP64 residual did not (possible in plain FP64 CG
    // for very small tol); report it rather than claim convergence.
    status = QCD_ERR_NOT_CONVERGED;
  }
  if (info) {
    info->iterations = h.iter;
    info->reliable_updates = h.ru_count;
    info->true_rel_residual = true_rel;
    info->iterated_rel_residual = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
    info->converged = status == QCD_OK;
    info->status = status;
    info->kernel_launches = (int)R.launches;
    info->dslash_launches = dslash_launches;
    info->dslash_ms = dslash_ms;
  }
  return status;
}

size_t cg_workspace_bytes(const qcd_lattice* lat, int prec_inner, int nrhs) {
  return carve(lat, prec_inner, nrhs, nullptr).total;
}

int run_cg(qcd_lattice* lat, void* x, const void* b, double mass, double tol, int max_iter, const qcd_solver_opts& o,
           void* ws, void* y, qcd_solve_info* info, cudaStream_t st) {
  const int prec = o.prec_inner;
  const int recon = lat->links[prec].recon;
  if (prec == QCD_PREC_DOUBLE && recon == 18) return cg_typed<QCD_PREC_DOUBLE, 18>(lat, x, b, mass, tol, max_iter, o, ws, y, info, st);
  if (prec == QCD_PREC_SINGLE && recon == 18) return cg_typed<QCD_PREC_SINGLE, 18>(lat, x, b, mass, tol, max_iter, o, ws, y, info, st);
  if (prec == QCD_PREC_SINGLE && recon == 12) return cg_typed<QCD_PREC_SINGLE, 12>(lat, x, b, mass, tol, max_iter, o, ws, y, info, st);
  if (prec == QCD_PREC_HALF && recon == 12) return cg_typed<QCD_PREC_HALF, 12>(lat, x, b, mass, tol, max_iter, o, ws, y, info, st);
  if (prec == QCD_PREC_DF64 && recon == 18) return cg_typed<QCD_PREC_DF64, 18>(lat, x, b, mass, tol, max_iter, o, ws, y, info, st);
  return QCD_ERR_UNSUPPORTED;
}

}  // namespace qcd
