// Autotuner for the launch shapes of the batched solvers.
//
// qcd_tune_mrhs times the multi-RHS solver's operator launches (CUDA events, a short run of the
// real solve) for the shared-link kernel and every register block of right-hand sides;
// qcd_tune_batched times the whole
// persistent batched solve for every (cluster size, block size) pair. The winner is kept in an
// in-process table that the solvers consult when the corresponding option is 0, and appended to
// an optional text cache (one "key value..." line per entry) that qcd_tune_load reads back.
// Keys carry the GPU name, so a cache shared between machines does not mix GPUs.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qcd_internal.cuh"

namespace qcd {

static std::mutex g_tune_mutex;
static std::map<std::string, std::vector<int>> g_tune;

static std::string gpu_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (auto& c : s)
    if (c == ' ') c = '_';
  return s;
}

std::string mrhs_key(const qcd_lattice* lat, int prec, int recon, int nrhs) {
  char buf[256];
  snprintf(buf, sizeof(buf), "mrhs|%s|%dx%dx%dx%d|p%d|r%d|n%d", gpu_name().c_str(), lat->L[0], lat->L[1], lat->L[2],
           lat->L[3], prec, recon, nrhs);
  return buf;
}

std::string batched_key(int n, qcd_lattice* const* lats, int prec, int recon) {
  long long sites = 0;
  for (int i = 0; i < n; ++i) sites += lats[i]->V;
  char buf[256];
  snprintf(buf, sizeof(buf), "batched|%s|n%d|v%lld|p%d|r%d", gpu_name().c_str(), n, sites, prec, recon);
  return buf;
}

bool tune_lookup(const std::string& key, std::vector<int>* out) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

static void tune_store(const std::string& key, const std::vector<int>& v, const char* cache_path) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune[key] = v;
  if (cache_path && *cache_path) {
    if (FILE* f = fopen(cache_path, "a")) {
      fprintf(f, "%s", key.c_str());
      for (int x : v) fprintf(f, " %d", x);
      fprintf(f, "\n");
      fclose(f);
    }
  }
}

int run_cg_mrhs(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*,
                qcd_solve_info*, cudaStream_t);
int run_cg_batched(int, qcd_lattice* const*, void* const*, const void* const*, void* const*, const double*, double, int,
                   const qcd_solver_opts&, void*, qcd_solve_info*, cudaStream_t);
int check_mrhs_args(const qcd_lattice*, int, void*, const void*, void*, double, double, int, const qcd_solver_opts*,
                    void*, qcd_solver_opts&);
int check_batched_args(int, qcd_lattice* const[], void* const[], const void* const[], void* const[], const double[],
                       double, int, const qcd_solver_opts*, void*, qcd_solver_opts&);

}  // namespace qcd

using namespace qcd;

extern "C" {

// A cached entry is loaded only if its values are launch shapes the solvers accept: a multi-RHS
// block of -1 (shared-link kernel), 1, 2, 4, 8 or 16; a cluster of 1-16 blocks (a power of two) of
// 32-256 threads (a multiple of 32). A hand-edited or truncated line is skipped, not launched.
static bool valid_entry(const std::string& key, const std::vector<int>& v) {
  if (key.compare(0, 5, "mrhs|") == 0)
    return v[0] == -1 || v[0] == 1 || v[0] == 2 || v[0] == 4 || v[0] == 8 || v[0] == 16;
  if (key.compare(0, 8, "batched|") == 0)
    return v.size() >= 2 && v[0] >= 1 && v[0] <= 16 && (v[0] & (v[0] - 1)) == 0 && v[1] >= 32 && v[1] <= 256 &&
           v[1] % 32 == 0;
  return false;
}

int qcd_tune_load(const char* cache_path) {
  if (!cache_path) {
    set_error("cache_path is NULL");
    return QCD_ERR_INVALID_ARG;
  }
  FILE* f = fopen(cache_path, "r");
  if (!f) return QCD_OK;  // nothing cached yet
  char line[512];
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  while (fgets(line, sizeof(line), f)) {
    char* save = nullptr;
    char* tok = strtok_r(line, " \n", &save);
    if (!tok) continue;
    std::string key = tok;
    std::vector<int> v;
    while ((tok = strtok_r(nullptr, " \n", &save))) v.push_back(atoi(tok));
    if (!v.empty() && valid_entry(key, v)) g_tune[key] = v;  // later lines win
  }
  fclose(f);
  return QCD_OK;
}

int qcd_tune_mrhs(qcd_lattice* lat, int nrhs, void* x_dev, const void* b_dev, double mass,
                  const qcd_solver_opts* opts, void* workspace_dev, const char* cache_path, int* best_rhs_block,
                  void* stream) {
  if (!best_rhs_block) {
    set_error("best_rhs_block is NULL");
    return QCD_ERR_INVALID_ARG;
  }
  qcd_solver_opts o;
  if (int rc = check_mrhs_args(lat, nrhs, x_dev, b_dev, nullptr, mass, 1e-14, 24, opts, workspace_dev, o)) return rc;
  o.profile = 1;
  const int cands[] = {-1, 1, 2, 4, 8, 16};  // -1: the shared-link kernel
  double best_us = 1e300;
  int best = 0;
  std::vector<qcd_solve_info> info(nrhs);
  for (int rb : cands) {
    if (rb > 2 * nrhs && rb > 1) break;
    if (rb == -1 && nrhs < 2) continue;
    if ((o.prec_inner == QCD_PREC_DOUBLE || o.prec_inner == QCD_PREC_DF64) && rb > 4) break;  // 64-bit accumulators
    o.rhs_block = rb;
    // a short run of the real solve (it stops at max_iter; only the launch timings matter)
    const int rc = run_cg_mrhs(lat, nrhs, x_dev, b_dev, mass, 1e-14, 24, o, workspace_dev, nullptr, info.data(),
                               (cudaStream_t)stream);
    if (rc != QCD_OK && rc != QCD_ERR_NOT_CONVERGED) return rc;
    if (info[0].dslash_launches <= 0) continue;
    const double us = 1e3 * info[0].dslash_ms / info[0].dslash_launches;
    if (us < best_us) {
      best_us = us;
      best = rb;
    }
  }
  if (!best) {
    set_error("qcd_tune_mrhs: no candidate ran");
    return QCD_ERR_UNSUPPORTED;
  }
  tune_store(mrhs_key(lat, o.prec_inner, lat->links[o.prec_inner].recon, nrhs), {best, (int)(best_us * 1000)},
             cache_path);
  *best_rhs_block = best;
  return QCD_OK;
}

int qcd_tune_batched(int n, qcd_lattice* const lats[], void* const x[], const void* const b[], const double mass[],
                     double tol, int max_iter, const qcd_solver_opts* opts, void* workspace_dev,
                     const char* cache_path, int* best_cluster, int* best_block, void* stream) {
  if (!best_cluster || !best_block) {
    set_error("best_cluster and best_block must not be NULL");
    return QCD_ERR_INVALID_ARG;
  }
  qcd_solver_opts o;
  if (int rc = check_batched_args(n, lats, x, b, nullptr, mass, tol, max_iter, opts, workspace_dev, o)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  QCD_CUDA(cudaEventCreate(&e0));
  QCD_CUDA(cudaEventCreate(&e1));
  const int clusters[] = {1, 2, 4, 8, 16};
  const int blocks[] = {128, 256};
  float best_ms = 1e30f;
  int bc = 0, bb = 0;
  std::vector<qcd_solve_info> info(n);
  for (int C : clusters) {
    for (int B : blocks) {
      o.cluster_size = C;
      o.block_size = B;
      cudaEventRecord(e0, st);
      const int rc = run_cg_batched(n, lats, x, b, nullptr, mass, tol, max_iter, o, workspace_dev, info.data(), st);
      cudaEventRecord(e1, st);
      if (rc == QCD_ERR_UNSUPPORTED) continue;  // this cluster shape does not fit
      if (rc != QCD_OK && rc != QCD_ERR_NOT_CONVERGED) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
      }
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        bc = C;
        bb = B;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!bc) {
    set_error("qcd_tune_batched: no cluster shape ran");
    return QCD_ERR_UNSUPPORTED;
  }
  tune_store(batched_key(n, lats, o.prec_inner, lats[0]->links[o.prec_inner].recon), {bc, bb, (int)(best_ms * 1000)},
             cache_path);
  *best_cluster = bc;
  *best_block = bb;
  return QCD_OK;
}

}  // extern "C"
