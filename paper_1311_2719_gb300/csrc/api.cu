// C-ABI entry points: argument validation, handle bookkeeping and error reporting around the
// kernels of pack.cu, dslash.cu and cg.cu.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <new>

#include <cuda.h>  // driver-API types only; the one driver call is fetched at run time

#include "qcd_internal.cuh"

namespace qcd {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return QCD_ERR_CUDA;
}

int launch_pack_links(const qcd_lattice*, const void*, void*, int, int, cudaStream_t);
int launch_pack_field(const qcd_lattice*, void*, const void*, int, int, cudaStream_t);
int launch_unpack_field(const qcd_lattice*, void*, const void*, int, int, cudaStream_t);
int launch_dslash(const qcd_lattice*, void*, const void*, int, int, cudaStream_t);
int launch_dslash_mrhs(const qcd_lattice*, void*, const void*, int, int, int, int, cudaStream_t);
int launch_mdagm(const qcd_lattice*, void*, const void*, double, int, void*, cudaStream_t);
size_t cg_workspace_bytes(const qcd_lattice*, int, int);
int run_cg(qcd_lattice*, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*,
           qcd_solve_info*, cudaStream_t);
size_t batch_workspace_bytes(int, const qcd_lattice* const*, int);
size_t wfield_bytes(int, long long);
size_t wlinks_bytes(int, long long);
size_t wilson_workspace_bytes(const qcd_lattice*, int, int);
int wilson_rhs_block(int, int, int);
int launch_wilson_op_mrhs(const qcd_lattice*, void*, const void*, int, double, int, int, cudaStream_t);
int launch_wilson_pack_links(const qcd_lattice*, const void*, void*, int, cudaStream_t);
int launch_wilson_pack(const qcd_lattice*, void*, const void*, int, bool, cudaStream_t);
int launch_wilson_op(const qcd_lattice*, void*, const void*, double, int, int, cudaStream_t);
int run_wilson_cgnr(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*,
                    qcd_solve_info*, cudaStream_t);
size_t full_workspace_bytes(const qcd_lattice*, int);
int launch_fermion_force(const qcd_lattice*, void*, const void*, const void*, const void*, cudaStream_t);
int run_solve_full(qcd_lattice*, void*, const void*, double, double, int, const qcd_solver_opts&, void*,
                   qcd_solve_info*, cudaStream_t);
int run_cg_batched(int, qcd_lattice* const*, void* const*, const void* const*, void* const*, const double*, double, int,
                   const qcd_solver_opts&, void*, qcd_solve_info*, cudaStream_t);
int run_cg_mrhs(qcd_lattice*, int, void*, const void*, double, double, int, const qcd_solver_opts&, void*, void*,
                qcd_solve_info*, cudaStream_t);

static int invalid(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return QCD_ERR_INVALID_ARG;
}

static bool aligned(const void* p) { return ((uintptr_t)p & 255u) == 0; }
static bool valid_prec(int p) {
  return p == QCD_PREC_DOUBLE || p == QCD_PREC_SINGLE || p == QCD_PREC_HALF || p == QCD_PREC_DF64;
}
static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

static int check_dev_ptr(const void* p, const char* name) {
  if (!p) return invalid("%s is NULL", name);
  if (!aligned(p)) return invalid("%s is not 256-byte aligned", name);
  return QCD_OK;
}

// Bytes from p to the end of the cudaMalloc allocation that holds it; 0 when that is unknown (no
// driver, not device memory, or memory from the virtual-memory or stream-ordered allocators, whose
// mapped ranges need not end where the caller's buffer does).
size_t device_span(const void* p) {
  using GetRange = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);
  using GetAttr = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
  struct Fns {
    GetRange range = nullptr;
    GetAttr attr = nullptr;
  };
  static const Fns fns = [] {
    Fns f;
    void* r = nullptr;
    void* a = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &r, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &a, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      f.range = (GetRange)r;
      f.attr = (GetAttr)a;
    }
    cudaGetLastError();
    return f;
  }();
  if (!p || !fns.range || !fns.attr) return 0;
  const CUdeviceptr d = (CUdeviceptr)(uintptr_t)p;
  unsigned long long legacy = 0;  // a boolean of unstated width: a cudaMalloc-type allocation (the
                                  // only kind whose address range is the allocation itself)
  if (fns.attr(&legacy, CU_POINTER_ATTRIBUTE_IS_LEGACY_CUDA_IPC_CAPABLE, d) != CUDA_SUCCESS || !legacy) return 0;
  CUdeviceptr base = 0;
  size_t size = 0;
  if (fns.range(&base, &size, d) != CUDA_SUCCESS || d < base || d - base > size) return 0;
  return (size_t)(base + size - d);
}

// The buffer at p must have `need` bytes before the end of its allocation, where that is known.
static int check_span(const void* p, size_t need, const char* name) {
  const size_t have = device_span(p);
  if (have && have < need)
    return invalid("%s: %zu bytes from the pointer to the end of its device allocation, %zu needed", name, have, need);
  return QCD_OK;
}
struct Span {
  const void* p;
  size_t need;
  const char* name;
};
static int check_spans(std::initializer_list<Span> spans) {
  for (const Span& s : spans)
    if (s.p)
      if (int rc = check_span(s.p, s.need, s.name)) return rc;
  return QCD_OK;
}
// canonical layouts: links complex128[V][4][3][3], staggered field complex128[V][3], Wilson
// spinor field complex128[V][4][3]
static size_t canon_links(const qcd_lattice* lat) { return (size_t)lat->V * 4 * 9 * 16; }
static size_t canon_field(const qcd_lattice* lat) { return (size_t)lat->V * 3 * 16; }
static size_t canon_spinor(const qcd_lattice* lat) { return (size_t)lat->V * 12 * 16; }

static int check_links(const qcd_lattice* lat, int prec) {
  if (!valid_prec(prec)) return invalid("unknown precision %d", prec);
  if (!lat->links[prec].ptr || !lat->links[prec].recon) {
    set_error("no links loaded for precision %d (call qcd_load_links first)", prec);
    return QCD_ERR_NO_LINKS;
  }
  return QCD_OK;
}

}  // namespace qcd

using namespace qcd;

extern "C" {

const char* qcd_status_string(int s) {
  switch (s) {
    case QCD_OK: return "ok";
    case QCD_ERR_INVALID_ARG: return "invalid argument";
    case QCD_ERR_CUDA: return "CUDA error";
    case QCD_ERR_NOT_CONVERGED: return "not converged";
    case QCD_ERR_BREAKDOWN: return "solver breakdown";
    case QCD_ERR_TIMEOUT: return "device wait timed out";
    case QCD_ERR_UNSUPPORTED: return "unsupported";
    case QCD_ERR_NO_LINKS: return "links not loaded";
  }
  return "unknown status";
}

const char* qcd_last_error(void) { return g_err; }

const char* qcd_version(void) { return "qcd-gb300 0.1 (sm_103a)"; }

int qcd_lattice_create(int L0, int L1, int L2, int L3, qcd_lattice** out) {
  if (!out) return invalid("out is NULL");
  *out = nullptr;
  const int L[4] = {L0, L1, L2, L3};
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (L[mu] < 2 || (L[mu] & 1)) return invalid("extent L%d = %d must be even and >= 2", mu, L[mu]);
    V *= L[mu];
  }
  if (V >= (1ll << 31)) return invalid("volume %lld too large", V);
  qcd_lattice* lat = new (std::nothrow) qcd_lattice();
  if (!lat) return invalid("out of host memory");
  for (int mu = 0; mu < 4; ++mu) lat->L[mu] = L[mu];
  lat->V = V;
  lat->Vh = V / 2;
  lat->tbc = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  lat->device = dev;
  *out = lat;
  return QCD_OK;
}

int qcd_lattice_destroy(qcd_lattice* lat) {
  delete lat;
  return QCD_OK;
}

int qcd_lattice_set_tbc(qcd_lattice* lat, int sign) {
  if (!lat) return invalid("lat is NULL");
  if (sign != 1 && sign != -1) return invalid("tbc sign must be +1 or -1, got %d", sign);
  if (sign != lat->tbc) {
    lat->tbc = sign;
    for (auto& l : lat->links) l = LinkSet{};
    for (auto& w : lat->wilson_links) w = nullptr;
  }
  return QCD_OK;
}

int qcd_lattice_device(const qcd_lattice* lat) { return lat ? lat->device : -1; }

size_t qcd_device_span_bytes(const void* ptr) { return device_span(ptr); }

size_t qcd_field_bytes(const qcd_lattice* lat, int prec) {
  if (!lat || !valid_prec(prec)) return 0;
  return field_bytes(prec, lat->Vh);
}

size_t qcd_links_bytes(const qcd_lattice* lat, int prec, int recon) {
  if (!lat) return 0;
  return links_bytes(prec, recon, lat->Vh);
}

void qcd_solver_opts_default(qcd_solver_opts* o) {
  if (!o) return;
  o->prec_inner = QCD_PREC_DOUBLE;
  o->recon_inner = 18;
  o->reliable_delta = 0.1;
  o->reliable_interval = 100;
  o->check_interval = 8;
  o->use_graph = 1;
  o->profile = 0;
  o->rhs_block = 0;
  o->cluster_size = 0;
  o->block_size = 0;
  o->staged = 0;
  o->wait_cycles = 0;
  o->prec_outer = QCD_PREC_DOUBLE;
}

size_t qcd_workspace_bytes(const qcd_lattice* lat, const qcd_solver_opts* opts, int nrhs) {
  if (!lat || nrhs < 1 || nrhs > kMaxRhs) return 0;
  qcd_solver_opts o;
  qcd_solver_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_prec(o.prec_inner)) return 0;
  return cg_workspace_bytes(lat, o.prec_inner, nrhs);
}

int qcd_load_links(qcd_lattice* lat, const void* links_dev, void* packed_dev, int prec, int recon, void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(links_dev, "links_dev")) return rc;
  if (int rc = check_dev_ptr(packed_dev, "packed_dev")) return rc;
  if (!valid_prec(prec)) return invalid("unknown precision %d", prec);
  if (links_bytes(prec, recon, lat->Vh) == 0) {
    set_error("precision %d with reconstruct-%d is not provided", prec, recon);
    return QCD_ERR_UNSUPPORTED;
  }
  if (int rc = check_spans({{links_dev, canon_links(lat), "links_dev"},
                            {packed_dev, links_bytes(prec, recon, lat->Vh), "packed_dev"}}))
    return rc;
  int rc = launch_pack_links(lat, links_dev, packed_dev, prec, recon, as_stream(stream));
  if (rc) return rc;
  lat->links[prec].ptr = packed_dev;
  lat->links[prec].recon = recon;
  return QCD_OK;
}

int qcd_pack_field(const qcd_lattice* lat, void* packed_dev, const void* canonical_dev, int parity, int prec,
                   void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(packed_dev, "packed_dev")) return rc;
  if (int rc = check_dev_ptr(canonical_dev, "canonical_dev")) return rc;
  if (parity != QCD_EVEN && parity != QCD_ODD) return invalid("parity must be 0 or 1, got %d", parity);
  if (!valid_prec(prec)) return invalid("unknown precision %d", prec);
  if (int rc = check_spans({{packed_dev, field_bytes(prec, lat->Vh), "packed_dev"},
                            {canonical_dev, canon_field(lat), "canonical_dev"}}))
    return rc;
  return launch_pack_field(lat, packed_dev, canonical_dev, parity, prec, as_stream(stream));
}

int qcd_unpack_field(const qcd_lattice* lat, void* canonical_dev, const void* packed_dev, int parity, int prec,
                     void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(packed_dev, "packed_dev")) return rc;
  if (int rc = check_dev_ptr(canonical_dev, "canonical_dev")) return rc;
  if (parity != QCD_EVEN && parity != QCD_ODD) return invalid("parity must be 0 or 1, got %d", parity);
  if (!valid_prec(prec)) return invalid("unknown precision %d", prec);
  if (int rc = check_spans({{packed_dev, field_bytes(prec, lat->Vh), "packed_dev"},
                            {canonical_dev, canon_field(lat), "canonical_dev"}}))
    return rc;
  return launch_unpack_field(lat, canonical_dev, packed_dev, parity, prec, as_stream(stream));
}

int qcd_dslash(const qcd_lattice* lat, void* out_dev, const void* in_dev, int out_parity, int prec, void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(out_dev, "out_dev")) return rc;
  if (int rc = check_dev_ptr(in_dev, "in_dev")) return rc;
  if (out_dev == in_dev) return invalid("out_dev must not alias in_dev");
  if (out_parity != QCD_EVEN && out_parity != QCD_ODD) return invalid("out_parity must be 0 or 1");
  if (int rc = check_links(lat, prec)) return rc;
  const size_t fb = field_bytes(prec, lat->Vh);
  if (int rc = check_spans({{out_dev, fb, "out_dev"}, {in_dev, fb, "in_dev"}})) return rc;
  return launch_dslash(lat, out_dev, in_dev, out_parity, prec, as_stream(stream));
}

int qcd_dslash_mrhs(const qcd_lattice* lat, void* out_dev, const void* in_dev, int nrhs, int out_parity, int prec,
                    void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(out_dev, "out_dev")) return rc;
  if (int rc = check_dev_ptr(in_dev, "in_dev")) return rc;
  if (out_dev == in_dev) return invalid("out_dev must not alias in_dev");
  if (nrhs < 1 || nrhs > kMaxRhs) return invalid("nrhs must be in [1, %d], got %d", kMaxRhs, nrhs);
  if (out_parity != QCD_EVEN && out_parity != QCD_ODD) return invalid("out_parity must be 0 or 1");
  if (int rc = check_links(lat, prec)) return rc;
  const size_t fb = field_bytes(prec, lat->Vh) * nrhs;
  if (int rc = check_spans({{out_dev, fb, "out_dev"}, {in_dev, fb, "in_dev"}})) return rc;
  int rb = 1;
  while (rb * 2 <= nrhs && rb < 4) rb *= 2;
  return launch_dslash_mrhs(lat, out_dev, in_dev, nrhs, out_parity, prec, rb, as_stream(stream));
}

int qcd_mdagm(const qcd_lattice* lat, void* out_dev, const void* in_dev, double mass, int prec, void* tmp_dev,
              void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(out_dev, "out_dev")) return rc;
  if (int rc = check_dev_ptr(in_dev, "in_dev")) return rc;
  if (int rc = check_dev_ptr(tmp_dev, "tmp_dev")) return rc;
  if (tmp_dev == in_dev || tmp_dev == out_dev) return invalid("tmp_dev must not alias in_dev or out_dev");
  if (!(mass > 0.0) || !std::isfinite(mass)) return invalid("mass must be finite and > 0, got %g", mass);
  if (int rc = check_links(lat, prec)) return rc;
  const size_t fb = field_bytes(prec, lat->Vh);
  if (int rc = check_spans({{out_dev, fb, "out_dev"}, {in_dev, fb, "in_dev"}, {tmp_dev, fb, "tmp_dev"}})) return rc;
  return launch_mdagm(lat, out_dev, in_dev, mass, prec, tmp_dev, as_stream(stream));
}

}  // extern "C"

namespace qcd {
// Shared argument checks of the solver entry points; fills `o` with the effective options.
static int check_solve_args(const qcd_lattice* lat, void* x_dev, const void* b_dev, void* workspace_dev, void* y_dev,
                            double mass, double tol, int max_iter, const qcd_solver_opts* opts, qcd_solver_opts& o) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(x_dev, "x_dev")) return rc;
  if (int rc = check_dev_ptr(b_dev, "b_dev")) return rc;
  if (int rc = check_dev_ptr(workspace_dev, "workspace_dev")) return rc;
  if (y_dev && !aligned(y_dev)) return invalid("y_dev is not 256-byte aligned");
  if (x_dev == b_dev) return invalid("x_dev must not alias b_dev");
  if (!(mass > 0.0) || !std::isfinite(mass)) return invalid("mass must be finite and > 0, got %g", mass);
  if (!(tol > 0.0) || !(tol < 1.0)) return invalid("tol must be in (0, 1), got %g", tol);
  if (max_iter < 1) return invalid("max_iter must be >= 1, got %d", max_iter);
  qcd_solver_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_prec(o.prec_inner)) return invalid("unknown inner precision %d", o.prec_inner);
  if (o.reliable_delta < 0.0 || o.reliable_delta >= 1.0) return invalid("reliable_delta must be in [0, 1)");
  if (o.rhs_block != -1 && o.rhs_block != 0 && o.rhs_block != 1 && o.rhs_block != 2 && o.rhs_block != 4 &&
      o.rhs_block != 8 && o.rhs_block != 16)
    return invalid("rhs_block must be -1, 0, 1, 2, 4, 8 or 16, got %d", o.rhs_block);
  if (int rc = check_links(lat, QCD_PREC_DOUBLE)) return rc;
  if (int rc = check_links(lat, o.prec_inner)) return rc;
  if (o.prec_inner != QCD_PREC_DOUBLE && lat->links[o.prec_inner].recon != o.recon_inner) {
    set_error("inner links loaded with reconstruct-%d, options ask for %d", lat->links[o.prec_inner].recon,
              o.recon_inner);
    return QCD_ERR_INVALID_ARG;
  }
  return QCD_OK;
}

// Checks of a multi-RHS solve (qcd_cg_solve_mrhs and its tuner); fills `o`.
int check_mrhs_args(const qcd_lattice* lat, int nrhs, void* x_dev, const void* b_dev, void* y_dev, double mass,
                    double tol, int max_iter, const qcd_solver_opts* opts, void* workspace_dev, qcd_solver_opts& o) {
  if (nrhs < 1 || nrhs > kMaxRhs) return invalid("nrhs must be in [1, %d], got %d", kMaxRhs, nrhs);
  if (int rc = check_solve_args(lat, x_dev, b_dev, workspace_dev, y_dev, mass, tol, max_iter, opts, o)) return rc;
  const size_t fr = canon_field(lat) * nrhs;
  return check_spans({{x_dev, fr, "x_dev"}, {b_dev, fr, "b_dev"}, {y_dev, fr, "y_dev"},
                      {workspace_dev, cg_workspace_bytes(lat, o.prec_inner, nrhs), "workspace_dev"}});
}

// Checks of a batched solve (qcd_cg_solve_batched and its tuner); fills `o`.
int check_batched_args(int n, qcd_lattice* const lats[], void* const x[], const void* const b[], void* const y[],
                       const double mass[], double tol, int max_iter, const qcd_solver_opts* opts, void* workspace_dev,
                       qcd_solver_opts& o) {
  if (n < 1) return invalid("n must be >= 1, got %d", n);
  if (!lats || !x || !b || !mass) return invalid("lats, x, b and mass must not be NULL");
  if (int rc = check_dev_ptr(workspace_dev, "workspace_dev")) return rc;
  if (!(tol > 0.0) || !(tol < 1.0)) return invalid("tol must be in (0, 1), got %g", tol);
  if (max_iter < 1) return invalid("max_iter must be >= 1, got %d", max_iter);
  qcd_solver_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_prec(o.prec_inner)) return invalid("unknown inner precision %d", o.prec_inner);
  if (o.reliable_delta < 0.0 || o.reliable_delta >= 1.0) return invalid("reliable_delta must be in [0, 1)");
  if (o.cluster_size != 0 && (o.cluster_size < 1 || o.cluster_size > 16 || (o.cluster_size & (o.cluster_size - 1))))
    return invalid("cluster_size must be 0 (tuned) or a power of two <= 16, got %d", o.cluster_size);
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > 256 || o.block_size % 32 != 0))
    return invalid("block_size must be 0 (tuned) or a multiple of 32 in [32, 256], got %d", o.block_size);
  int dev = -1;
  cudaGetDevice(&dev);
  int recon0 = 0;
  for (int i = 0; i < n; ++i) {
    const qcd_lattice* lat = lats[i];
    if (!lat) return invalid("lats[%d] is NULL", i);
    if (lat->device != dev) return invalid("lats[%d] belongs to device %d, current device is %d", i, lat->device, dev);
    if (int rc = check_dev_ptr(x[i], "x[i]")) return rc;
    if (int rc = check_dev_ptr(b[i], "b[i]")) return rc;
    if (y && y[i] && !aligned(y[i])) return invalid("y[%d] is not 256-byte aligned", i);
    if (x[i] == b[i]) return invalid("x[%d] must not alias b[%d]", i, i);
    if (!(mass[i] > 0.0) || !std::isfinite(mass[i])) return invalid("mass[%d] must be finite and > 0", i);
    if (int rc = check_links(lat, QCD_PREC_DOUBLE)) return rc;
    if (int rc = check_links(lat, o.prec_inner)) return rc;
    if (i == 0) recon0 = lat->links[o.prec_inner].recon;
    if (lat->links[o.prec_inner].recon != recon0)
      return invalid("every lattice must load the inner links with the same reconstruction");
    if (int rc = check_spans({{x[i], canon_field(lat), "x[i]"}, {b[i], canon_field(lat), "b[i]"},
                              {y ? y[i] : nullptr, canon_field(lat), "y[i]"}}))
      return rc;
  }
  return check_span(workspace_dev, batch_workspace_bytes(n, (const qcd_lattice* const*)lats, o.prec_inner),
                    "workspace_dev");
}
}  // namespace qcd

extern "C" {

int qcd_cg_solve(qcd_lattice* lat, void* x_dev, const void* b_dev, double mass, double tol, int max_iter,
                 const qcd_solver_opts* opts, void* workspace_dev, void* y_dev, qcd_solve_info* info, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info) std::memset(info, 0, sizeof(*info));
  auto done = [&](int rc) {
    if (info) {
      info->status = rc;
      info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return rc;
  };
  qcd_solver_opts o;
  if (int rc = check_solve_args(lat, x_dev, b_dev, workspace_dev, y_dev, mass, tol, max_iter, opts, o)) return done(rc);
  if (int rc = check_spans({{x_dev, canon_field(lat), "x_dev"}, {b_dev, canon_field(lat), "b_dev"},
                            {y_dev, canon_field(lat), "y_dev"},
                            {workspace_dev, cg_workspace_bytes(lat, o.prec_inner, 1), "workspace_dev"}}))
    return done(rc);
  return done(run_cg(lat, x_dev, b_dev, mass, tol, max_iter, o, workspace_dev, y_dev, info, as_stream(stream)));
}

int qcd_cg_solve_mrhs(qcd_lattice* lat, int nrhs, void* x_dev, const void* b_dev, double mass, double tol,
                      int max_iter, const qcd_solver_opts* opts, void* workspace_dev, void* y_dev,
                      qcd_solve_info* info, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  const int n_info = (nrhs >= 1 && nrhs <= kMaxRhs) ? nrhs : 1;
  if (info) std::memset(info, 0, sizeof(*info) * n_info);
  auto done = [&](int rc) {
    if (info) {
      const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      for (int r = 0; r < n_info; ++r) {
        if (rc != QCD_OK && info[r].status == QCD_OK && info[r].iterations == 0) info[r].status = rc;
        info[r].seconds = sec;
      }
    }
    return rc;
  };
  qcd_solver_opts o;
  if (int rc = check_mrhs_args(lat, nrhs, x_dev, b_dev, y_dev, mass, tol, max_iter, opts, workspace_dev, o))
    return done(rc);
  return done(run_cg_mrhs(lat, nrhs, x_dev, b_dev, mass, tol, max_iter, o, workspace_dev, y_dev, info,
                          as_stream(stream)));
}

size_t qcd_workspace_bytes_batched(int n, qcd_lattice* const lats[], const qcd_solver_opts* opts) {
  if (n < 1 || !lats) return 0;
  for (int i = 0; i < n; ++i)
    if (!lats[i]) return 0;
  qcd_solver_opts o;
  qcd_solver_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_prec(o.prec_inner)) return 0;
  return batch_workspace_bytes(n, (const qcd_lattice* const*)lats, o.prec_inner);
}

int qcd_cg_solve_batched(int n, qcd_lattice* const lats[], void* const x[], const void* const b[], void* const y[],
                         const double mass[], double tol, int max_iter, const qcd_solver_opts* opts,
                         void* workspace_dev, qcd_solve_info info[], void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info && n > 0) std::memset(info, 0, sizeof(*info) * n);
  auto done = [&](int rc) {
    if (info && n > 0) {
      const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      for (int i = 0; i < n; ++i) {
        if (rc != QCD_OK && info[i].status == QCD_OK && info[i].iterations == 0) info[i].status = rc;
        info[i].seconds = sec;
      }
    }
    return rc;
  };
  qcd_solver_opts o;
  if (int rc = check_batched_args(n, lats, x, b, y, mass, tol, max_iter, opts, workspace_dev, o)) return done(rc);
  return done(run_cg_batched(n, lats, x, b, y, mass, tol, max_iter, o, workspace_dev, info, as_stream(stream)));
}

size_t qcd_workspace_bytes_full(const qcd_lattice* lat, const qcd_solver_opts* opts) {
  if (!lat) return 0;
  qcd_solver_opts o;
  qcd_solver_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_prec(o.prec_inner)) return 0;
  return full_workspace_bytes(lat, o.prec_inner);
}

int qcd_solve_full(qcd_lattice* lat, void* x_dev, const void* b_dev, double mass, double tol, int max_iter,
                   const qcd_solver_opts* opts, void* workspace_dev, qcd_solve_info* info, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info) std::memset(info, 0, sizeof(*info));
  auto done = [&](int rc) {
    if (info) {
      info->status = rc;
      info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return rc;
  };
  qcd_solver_opts o;
  if (int rc = check_solve_args(lat, x_dev, b_dev, workspace_dev, nullptr, mass, tol, max_iter, opts, o)) return done(rc);
  if (int rc = check_spans({{x_dev, canon_field(lat), "x_dev"}, {b_dev, canon_field(lat), "b_dev"},
                            {workspace_dev, full_workspace_bytes(lat, o.prec_inner), "workspace_dev"}}))
    return done(rc);
  return done(run_solve_full(lat, x_dev, b_dev, mass, tol, max_iter, o, workspace_dev, info, as_stream(stream)));
}

int qcd_fermion_force(const qcd_lattice* lat, void* force_dev, const void* links_dev, const void* x_dev,
                      const void* y_dev, void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(force_dev, "force_dev")) return rc;
  if (int rc = check_dev_ptr(links_dev, "links_dev")) return rc;
  if (int rc = check_dev_ptr(x_dev, "x_dev")) return rc;
  if (int rc = check_dev_ptr(y_dev, "y_dev")) return rc;
  if (force_dev == links_dev || force_dev == x_dev || force_dev == y_dev)
    return invalid("force_dev must not alias links_dev, x_dev or y_dev");
  if (int rc = check_spans({{force_dev, canon_links(lat), "force_dev"}, {links_dev, canon_links(lat), "links_dev"},
                            {x_dev, canon_field(lat), "x_dev"}, {y_dev, canon_field(lat), "y_dev"}}))
    return rc;
  return launch_fermion_force(lat, force_dev, links_dev, x_dev, y_dev, as_stream(stream));
}

static bool wilson_prec(int p) { return p == QCD_PREC_DOUBLE || p == QCD_PREC_SINGLE || p == QCD_PREC_DF64; }

size_t qcd_wilson_field_bytes(const qcd_lattice* lat, int prec) {
  return (lat && wilson_prec(prec)) ? wfield_bytes(prec, lat->V) : 0;
}

size_t qcd_wilson_links_bytes(const qcd_lattice* lat, int prec) {
  return (lat && wilson_prec(prec)) ? wlinks_bytes(prec, lat->V) : 0;
}

int qcd_wilson_load_links(qcd_lattice* lat, const void* links_dev, void* packed_dev, int prec, void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(links_dev, "links_dev")) return rc;
  if (int rc = check_dev_ptr(packed_dev, "packed_dev")) return rc;
  if (!wilson_prec(prec)) return invalid("Wilson links: precision must be DOUBLE, SINGLE or DF64, got %d", prec);
  if (int rc = check_spans({{links_dev, canon_links(lat), "links_dev"},
                            {packed_dev, wlinks_bytes(prec, lat->V), "packed_dev"}}))
    return rc;
  int rc = launch_wilson_pack_links(lat, links_dev, packed_dev, prec, as_stream(stream));
  if (rc) return rc;
  lat->wilson_links[prec] = packed_dev;
  return QCD_OK;
}

int qcd_wilson_pack_field(const qcd_lattice* lat, void* packed_dev, const void* canonical_dev, int prec, void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(packed_dev, "packed_dev")) return rc;
  if (int rc = check_dev_ptr(canonical_dev, "canonical_dev")) return rc;
  if (!wilson_prec(prec)) return invalid("Wilson fields: precision must be DOUBLE, SINGLE or DF64, got %d", prec);
  if (int rc = check_spans({{packed_dev, wfield_bytes(prec, lat->V), "packed_dev"},
                            {canonical_dev, canon_spinor(lat), "canonical_dev"}}))
    return rc;
  return launch_wilson_pack(lat, packed_dev, canonical_dev, prec, false, as_stream(stream));
}

int qcd_wilson_unpack_field(const qcd_lattice* lat, void* canonical_dev, const void* packed_dev, int prec, void* stream) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(packed_dev, "packed_dev")) return rc;
  if (int rc = check_dev_ptr(canonical_dev, "canonical_dev")) return rc;
  if (!wilson_prec(prec)) return invalid("Wilson fields: precision must be DOUBLE, SINGLE or DF64, got %d", prec);
  if (int rc = check_spans({{packed_dev, wfield_bytes(prec, lat->V), "packed_dev"},
                            {canonical_dev, canon_spinor(lat), "canonical_dev"}}))
    return rc;
  return launch_wilson_pack(lat, const_cast<void*>(packed_dev), canonical_dev, prec, true, as_stream(stream));
}

static int check_wilson_op(const qcd_lattice* lat, void* out_dev, const void* in_dev, double kappa, int op, int prec) {
  if (!lat) return invalid("lat is NULL");
  if (int rc = check_dev_ptr(out_dev, "out_dev")) return rc;
  if (int rc = check_dev_ptr(in_dev, "in_dev")) return rc;
  if (out_dev == in_dev) return invalid("out_dev must not alias in_dev");
  if (op < QCD_WILSON_DSLASH || op > QCD_WILSON_MDAG) return invalid("op must be 0 (D_W), 1 (M) or 2 (M^dagger)");
  if (!std::isfinite(kappa)) return invalid("kappa must be finite");
  if (!wilson_prec(prec)) return invalid("Wilson operator: precision must be DOUBLE, SINGLE or DF64, got %d", prec);
  if (!lat->wilson_links[prec]) {
    set_error("no Wilson links loaded for precision %d (call qcd_wilson_load_links first)", prec);
    return QCD_ERR_NO_LINKS;
  }
  return QCD_OK;
}

int qcd_wilson_op(const qcd_lattice* lat, void* out_dev, const void* in_dev, double kappa, int op, int prec,
                  void* stream) {
  if (int rc = check_wilson_op(lat, out_dev, in_dev, kappa, op, prec)) return rc;
  const size_t fb = wfield_bytes(prec, lat->V);
  if (int rc = check_spans({{out_dev, fb, "out_dev"}, {in_dev, fb, "in_dev"}})) return rc;
  return launch_wilson_op(lat, out_dev, in_dev, kappa, op, prec, as_stream(stream));
}

int qcd_wilson_op_mrhs(const qcd_lattice* lat, void* out_dev, const void* in_dev, int nrhs, double kappa, int op,
                       int prec, void* stream) {
  if (prec == QCD_PREC_DF64) return invalid("multi-RHS Wilson operator: precision must be DOUBLE or SINGLE");
  if (int rc = check_wilson_op(lat, out_dev, in_dev, kappa, op, prec)) return rc;
  if (nrhs < 1 || nrhs > kMaxRhs) return invalid("nrhs must be in [1, %d], got %d", kMaxRhs, nrhs);
  const size_t fb = wfield_bytes(prec, lat->V) * nrhs;
  if (int rc = check_spans({{out_dev, fb, "out_dev"}, {in_dev, fb, "in_dev"}})) return rc;
  return launch_wilson_op_mrhs(lat, out_dev, in_dev, nrhs, kappa, op, prec, as_stream(stream));
}

size_t qcd_wilson_workspace_bytes(const qcd_lattice* lat, const qcd_solver_opts* opts, int nrhs) {
  if (!lat || nrhs < 1 || nrhs > kMaxRhs) return 0;
  qcd_solver_opts o;
  qcd_solver_opts_default(&o);
  if (opts) o = *opts;
  const bool ok = (o.prec_inner == QCD_PREC_DOUBLE && o.prec_outer == QCD_PREC_DOUBLE) ||
                  (o.prec_inner == QCD_PREC_SINGLE && (o.prec_outer == QCD_PREC_DOUBLE || o.prec_outer == QCD_PREC_DF64));
  return ok ? wilson_workspace_bytes(lat, o.prec_inner, nrhs) : 0;
}

static int wilson_cgnr_common(qcd_lattice* lat, int nrhs, void* x_dev, const void* b_dev, double kappa, double tol,
                              int max_iter, const qcd_solver_opts* opts, void* workspace_dev, qcd_solve_info* info,
                              void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  const int n_info = (nrhs >= 1 && nrhs <= kMaxRhs) ? nrhs : 1;
  if (info) std::memset(info, 0, sizeof(*info) * n_info);
  auto done = [&](int rc) {
    if (info) {
      const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      for (int q = 0; q < n_info; ++q) {
        if (rc != QCD_OK && info[q].status == QCD_OK && !info[q].converged) info[q].status = rc;
        info[q].seconds = sec;
      }
    }
    return rc;
  };
  if (!lat) return done(invalid("lat is NULL"));
  if (nrhs < 1 || nrhs > kMaxRhs) return done(invalid("nrhs must be in [1, %d], got %d", kMaxRhs, nrhs));
  if (int rc = check_dev_ptr(x_dev, "x_dev")) return done(rc);
  if (int rc = check_dev_ptr(b_dev, "b_dev")) return done(rc);
  if (int rc = check_dev_ptr(workspace_dev, "workspace_dev")) return done(rc);
  if (x_dev == b_dev) return done(invalid("x_dev must not alias b_dev"));
  if (!std::isfinite(kappa)) return done(invalid("kappa must be finite"));
  if (!(tol > 0.0) || !(tol < 1.0)) return done(invalid("tol must be in (0, 1), got %g", tol));
  if (max_iter < 1) return done(invalid("max_iter must be >= 1, got %d", max_iter));
  qcd_solver_opts o;
  qcd_solver_opts_default(&o);
  if (opts) o = *opts;
  if (o.prec_inner != QCD_PREC_DOUBLE && o.prec_inner != QCD_PREC_SINGLE)
    return done(invalid("Wilson CGNR: inner precision must be DOUBLE or SINGLE"));
  if (o.prec_outer != QCD_PREC_DOUBLE && !(o.prec_outer == QCD_PREC_DF64 && o.prec_inner == QCD_PREC_SINGLE))
    return done(invalid("Wilson CGNR: outer precision must be DOUBLE, or DF64 with a SINGLE inner precision"));
  if (o.reliable_delta < 0.0 || o.reliable_delta >= 1.0) return done(invalid("reliable_delta must be in [0, 1)"));
  if (wilson_rhs_block(o.prec_inner, nrhs, o.rhs_block) == 0)
    return done(invalid("rhs_block %d is not supported for Wilson precision %d (-1 for the shared-link kernel; 1, 2 "
                        "or 4 for SINGLE; 1 or 2 for DOUBLE)",
                        o.rhs_block, o.prec_inner));
  if (!lat->wilson_links[o.prec_outer] || !lat->wilson_links[o.prec_inner]) {
    set_error("Wilson links must be loaded at the outer and at the inner precision");
    return done(QCD_ERR_NO_LINKS);
  }
  const size_t fr = canon_spinor(lat) * nrhs;
  if (int rc = check_spans({{x_dev, fr, "x_dev"}, {b_dev, fr, "b_dev"},
                            {workspace_dev, wilson_workspace_bytes(lat, o.prec_inner, nrhs), "workspace_dev"}}))
    return done(rc);
  return done(run_wilson_cgnr(lat, nrhs, x_dev, b_dev, kappa, tol, max_iter, o, workspace_dev, info,
                              as_stream(stream)));
}

int qcd_wilson_cgnr(qcd_lattice* lat, void* x_dev, const void* b_dev, double kappa, double tol, int max_iter,
                    const qcd_solver_opts* opts, void* workspace_dev, qcd_solve_info* info, void* stream) {
  return wilson_cgnr_common(lat, 1, x_dev, b_dev, kappa, tol, max_iter, opts, workspace_dev, info, stream);
}

int qcd_wilson_cgnr_mrhs(qcd_lattice* lat, int nrhs, void* x_dev, const void* b_dev, double kappa, double tol,
                         int max_iter, const qcd_solver_opts* opts, void* workspace_dev, qcd_solve_info* info,
                         void* stream) {
  return wilson_cgnr_common(lat, nrhs, x_dev, b_dev, kappa, tol, max_iter, opts, workspace_dev, info, stream);
}

}  // extern "C"
