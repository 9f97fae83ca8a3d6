/*
 * qcd.h — C ABI of the GB300 (sm_103a) staggered-fermion Dslash / even-odd CG library.
 *
 * The library computes the staggered hopping operator of the paper's matrix-vector
 * routine (§3) and the conjugate-gradient solve of its congrad routine (§4) on one GPU.
 *
 * Operator (the paper does not write it out; this is the convention the library fixes):
 *   D x(n) = 1/2 sum_mu [ eta_mu(n) zeta_mu(n) U_mu(n) x(n+mu)
 *                         - eta_mu(n-mu) zeta_mu(n-mu) U_mu(n-mu)^dagger x(n-mu) ]
 *   eta_mu(n) = (-1)^(x0+...+x_{mu-1}); zeta_3(n) = tbc (default -1) on links with
 *   x3 = L3-1, else +1. D is anti-Hermitian; M = m + D; M^dagger M = m^2 - D^2.
 *   Even-odd: parity(n) = (x0+x1+x2+x3) mod 2; D_eo: odd -> even, D_oe: even -> odd;
 *   the solved operator is A = m^2 - D_eo D_oe on the even sites (Hermitian, >= m^2).
 *
 * Layouts
 *   canonical site index  i = x0 + L0*(x1 + L1*(x2 + L2*x3))   (x0 fastest, x3 = t slowest)
 *   canonical links       complex128[V][4][3][3]  (links[i][mu] = U_mu(n_i), row-major)
 *   canonical field       complex128[V][3]
 *   packed field          the library's even-odd structure-of-arrays layout of ONE parity
 *                         (V/2 sites) at one precision; size from qcd_field_bytes().
 *                         Site k of parity p is the canonical site i with i >> 1 == k.
 *                         QCD_PREC_DOUBLE: double2[3][V/2]; QCD_PREC_SINGLE: float2[3][V/2];
 *                         QCD_PREC_HALF: 16 bytes per site {3 x half2 colour, float scale};
 *                         QCD_PREC_DF64: float4[3][V/2] {re.hi, re.lo, im.hi, im.lo}.
 *   A multi-RHS packed field is nrhs packed fields back to back.
 *
 * Memory ownership
 *   The library never allocates device memory. The caller allocates every device buffer
 *   (packed links, fields, workspace) and keeps it alive while a handle refers to it.
 *   Device pointers must be 256-byte aligned. Host pointers are only read during a call.
 *   All calls that take a stream are asynchronous on that stream unless stated otherwise;
 *   `stream` is a cudaStream_t (NULL = the legacy default stream).
 *
 * Errors
 *   Every call returns a qcd_status. QCD_ERR_INVALID_ARG leaves all buffers untouched.
 *   qcd_last_error() gives a thread-local message about the last failing call.
 */
#ifndef QCD_H
#define QCD_H

#include <stddef.h>

#if defined(__GNUC__)
#define QCD_API __attribute__((visibility("default")))
#else
#define QCD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QCD_OK = 0,
  QCD_ERR_INVALID_ARG = 1,   /* bad size, pointer, precision, parity, mass or tolerance   */
  QCD_ERR_CUDA = 2,          /* a CUDA runtime call failed (message in qcd_last_error)    */
  QCD_ERR_NOT_CONVERGED = 3, /* max_iter reached before the requested tolerance           */
  QCD_ERR_BREAKDOWN = 4,     /* non-finite or non-positive CG scalar (e.g. NaN in b)      */
  QCD_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up                        */
  QCD_ERR_UNSUPPORTED = 6,   /* valid request this build does not implement               */
  QCD_ERR_NO_LINKS = 7       /* qcd_load_links was not called for this precision          */
} qcd_status;

enum { QCD_EVEN = 0, QCD_ODD = 1 };
/* QCD_PREC_DF64: every real held as an unevaluated sum of two FP32 values (48-bit significand),
 * stored in the same 16 bytes per complex number as FP64 and computed on the FP32 pipes; relative
 * error ~1e-14 against FP64 (links: reconstruct-18 only). */
enum { QCD_PREC_DOUBLE = 0, QCD_PREC_SINGLE = 1, QCD_PREC_HALF = 2, QCD_PREC_DF64 = 3 };
enum { QCD_RECON_18 = 18, QCD_RECON_12 = 12 };

typedef struct qcd_lattice qcd_lattice; /* opaque host-side handle */

/* Solver options (qcd_solver_opts_default fills the defaults noted here). */
typedef struct {
  int prec_inner;        /* QCD_PREC_DOUBLE (plain FP64 CG, default); _SINGLE, _HALF or _DF64 run the
                            recursion in that precision with FP64 reliable updates                */
  int recon_inner;       /* link compression for the inner operator: 18 (default) or 12          */
  double reliable_delta; /* mixed CG: reliable update when |r| < delta * max|r| since the last (0.1) */
  int reliable_interval; /* mixed CG: and at least every this many iterations (100)              */
  int check_interval;    /* host reads the device-side convergence flag every k iterations (8)    */
  int use_graph;         /* replay each k-iteration chunk as a CUDA graph (1)                     */
  int profile;           /* record CUDA events around every operator launch of the iteration (0);
                            profiled chunks run as direct launches, not graph replays         */
  int rhs_block;         /* staggered multi-RHS solves: right-hand sides per register block,
                            1/2/4/8/16; -1 = the shared-link kernel (a block loads each link of
                            its tile once into shared memory and applies it to every RHS);
                            0 = the tuned value if qcd_tune_mrhs recorded one, else -1 from 8
                            RHS on and a register block below. Wilson multi-RHS: see
                            qcd_wilson_cgnr_mrhs                                                */
  int cluster_size;      /* batched solves: thread blocks per cluster (one cluster per lattice
                            at a time), 1/2/4/8/16; 0 = tuned value or 4                        */
  int block_size;        /* batched solves: threads per block, multiple of 32 <= 256; 0 = tuned
                            value or 256                                                        */
  int staged;            /* 1: the FP32 recon-12 operator of the single-RHS CG stages each tile's
                            links and neighbour vectors in shared memory by bulk asynchronous
                            copies (measured 2.4x slower on GB300: ~600 staged bytes per site
                            leave 4 warps per SM); 0 (default): every thread loads its own
                            operands                                                           */
  long long wait_cycles; /* limit of a device-side wait on an mbarrier, in SM clock cycles (the
                            staged operator); 0 = 4e9 (about 2 s). On expiry the solve returns
                            QCD_ERR_TIMEOUT.                                                    */
  int prec_outer;        /* Wilson CGNR with prec_inner = SINGLE: precision of the solution
                            accumulator, the reliable updates and the confirming residual:
                            QCD_PREC_DOUBLE (default) or QCD_PREC_DF64 (the same 16 bytes per
                            complex, 48-bit significand, computed on the FP32 pipes); the
                            staggered solvers ignore it                                        */
} qcd_solver_opts;

/* What a solve reports. */
typedef struct {
  int iterations;           /* CG iterations executed                                             */
  int reliable_updates;     /* FP64 true-residual recomputations inside the solve (mixed CG)      */
  int converged;            /* 1 when the true residual met tol                                   */
  int status;               /* the qcd_status the call returned                                   */
  double true_rel_residual; /* |b_e - A x_e| / |b_e| recomputed in FP64 after the solve           */
  double iterated_rel_residual; /* sqrt(<r,r>/<b,b>) of the solver's recursion                    */
  double seconds;           /* wall time of the call (host clock, includes the final sync)        */
  int kernel_launches;      /* kernels this call launched (graph replays count every node)        */
  int dslash_launches;      /* operator launches inside the iterations (2 per iteration run)     */
  double dslash_ms;         /* with opts.profile: summed CUDA-event time of those launches       */
} qcd_solve_info;

/* ---- status ---------------------------------------------------------------------------------- */

QCD_API const char* qcd_status_string(int status);
/* Thread-local text about the most recent failing call on this thread ("" if none). */
QCD_API const char* qcd_last_error(void);
/* Library version string. */
QCD_API const char* qcd_version(void);

/* ---- lattice handle -------------------------------------------------------------------------- */

/* Create a handle for an L0 x L1 x L2 x L3 lattice (x3 = t). Every extent must be even and >= 2,
 * and the volume must be < 2^31. Antiperiodic in t by default. Allocates host memory only. */
QCD_API int qcd_lattice_create(int L0, int L1, int L2, int L3, qcd_lattice** out);
QCD_API int qcd_lattice_destroy(qcd_lattice* lat);
/* Boundary sign zeta on the t-links of the last time slice: +1 (periodic) or -1 (antiperiodic).
 * Links loaded before the change must be loaded again. */
QCD_API int qcd_lattice_set_tbc(qcd_lattice* lat, int sign);
/* Device on which the handle was created (the current device at qcd_lattice_create). */
QCD_API int qcd_lattice_device(const qcd_lattice* lat);

/* ---- sizes ------------------------------------------------------------------------------------ */

/* Bytes from ptr to the end of the device allocation that holds it, as the argument checks measure
 * it; 0 when unknown (not device memory, no driver, or memory of the virtual-memory or
 * stream-ordered allocators, whose mapped ranges the checks do not measure). Every entry point
 * returns QCD_ERR_INVALID_ARG, before any device work, for a buffer whose known span is shorter
 * than what the call reads or writes (e.g. a workspace sized for other options). */
QCD_API size_t qcd_device_span_bytes(const void* ptr);
/* Bytes of one packed single-parity field at `prec` (0 on a bad argument). */
QCD_API size_t qcd_field_bytes(const qcd_lattice* lat, int prec);
/* Bytes of the packed gauge field at (prec, recon). Supported: DOUBLE/18, SINGLE/18, SINGLE/12,
 * HALF/12, DF64/18. 0 on an unsupported pair. */
QCD_API size_t qcd_links_bytes(const qcd_lattice* lat, int prec, int recon);
/* Bytes of the device workspace qcd_cg_solve (nrhs = 1) or qcd_cg_solve_mrhs (1 <= nrhs <= 16)
 * needs for these options; 0 on a bad argument. */
QCD_API size_t qcd_workspace_bytes(const qcd_lattice* lat, const qcd_solver_opts* opts, int nrhs);

QCD_API void qcd_solver_opts_default(qcd_solver_opts* opts);

/* ---- links (paper §4: linkc_acc prepares the device copy of the gauge field) ---------------- */

/* Pack the canonical gauge field `links_dev` (device, complex128[V][4][3][3]) into `packed_dev`
 * (device, qcd_links_bytes(lat, prec, recon) bytes) and register it as the links used by every
 * later call at precision `prec`. Recon 18 folds 1/2 * eta * zeta into the stored links; recon 12
 * stores the first two rows and the kernels rebuild the third as conj(row0 x row1) and apply
 * the phases from the site coordinates. QCD_PREC_HALF links are 16-bit fixed point (every real v
 * of the two rows as round(v * 2^15) + 2^15, saturated to [0, 65535]; absolute error <= 2^-16,
 * 2^-15 for v within 2^-16 of 1).
 * The caller keeps `packed_dev` alive. */
QCD_API int qcd_load_links(qcd_lattice* lat, const void* links_dev, void* packed_dev, int prec, int recon,
                   void* stream);

/* ---- fields ------------------------------------------------------------------------------------ */

/* canonical (device, complex128[V][3]) -> packed field of parity `parity` at `prec`. */
QCD_API int qcd_pack_field(const qcd_lattice* lat, void* packed_dev, const void* canonical_dev, int parity,
                   int prec, void* stream);
/* packed -> canonical; writes only the sites of `parity`, leaves the other half untouched. */
QCD_API int qcd_unpack_field(const qcd_lattice* lat, void* canonical_dev, const void* packed_dev, int parity,
                     int prec, void* stream);

/* ---- operators (paper §3 matrix-vector routine; §4 fmv / fmtv calls) ------------------------- */

/* Half-lattice hop: out (parity out_parity) = D in (parity 1 - out_parity), packed fields at
 * `prec`, using the links registered for `prec`. `out` is overwritten and must not alias `in`.
 * With QCD_PREC_HALF the arithmetic is FP32 and the output is re-quantised per site. */
QCD_API int qcd_dslash(const qcd_lattice* lat, void* out_dev, const void* in_dev, int out_parity, int prec,
               void* stream);
/* Same operator on nrhs right-hand sides at once (multi-RHS packed fields): every link is loaded
 * once and applied to all nrhs vectors. 1 <= nrhs <= 16. */
QCD_API int qcd_dslash_mrhs(const qcd_lattice* lat, void* out_dev, const void* in_dev, int nrhs, int out_parity,
                    int prec, void* stream);
/* Even-site normal operator: out_e = (m^2 - D_eo D_oe) in_e, packed even fields at `prec`.
 * `tmp_dev` is caller scratch for one packed odd field (qcd_field_bytes(lat, prec) bytes).
 * mass must be > 0. */
QCD_API int qcd_mdagm(const qcd_lattice* lat, void* out_dev, const void* in_dev, double mass, int prec,
              void* tmp_dev, void* stream);

/* Same operator as qcd_mdagm, for callers that cannot allocate device memory. The paper has no
 * counterpart: this exists because some host programs cannot obtain a scratch buffer to pass as
 * `tmp_dev` — their device arrays are all placed by compiler data directives, or every byte of the
 * GPU is owned and accounted for by another framework's memory pool, so calling cudaMalloc is not
 * possible or not permitted. Here the intermediate odd-parity field lives in a 16 MiB array inside
 * the library (a file-scope __device__ array that every GPU loading the library keeps until the
 * process exits); the caller passes only `in_dev` and `out_dev`, and nothing is allocated.
 *   Limit: qcd_field_bytes(lat, prec) must be <= 16 MiB (e.g. FP64 and DF64 up to V/2 = 349525
 *   sites, 24^4; FP32 and FP16 up to 32^4); larger lattices get QCD_ERR_INVALID_ARG.
 *   The lattice's device (qcd_lattice_device) must be the current device, else
 *   QCD_ERR_INVALID_ARG: the array used is the current device's copy.
 *   The first call on each device looks up the array's device address with that device current;
 *   make that first call before any stream capture. The address is looked up again when the
 *   device's context has changed since (after a device reset, for instance).
 *   All calls share the one array and it keeps the last call's contents (the operator overwrites
 *   it completely before reading it). Calls whose executions overlap on the GPU — e.g. on two
 *   streams at once — race on it; serialise them. */
QCD_API int qcd_mdagm_noalloc(const qcd_lattice* lat, void* out_dev, const void* in_dev, double mass, int prec,
                      void* stream);

/* ---- solver (paper §4 congrad) --------------------------------------------------------------- */

/* Solve A x_e = b_e to |b_e - A x_e| / |b_e| <= tol (true FP64 residual) and, when y_dev is not
 * NULL, form y_o = D_oe x_e (the paper's "solution on the second half lattice").
 *   x_dev, b_dev, y_dev : device canonical fields complex128[V][3]; only the even half of b is
 *                         read; x is written on the even sites (odd half set to 0); y on the odd
 *                         sites (even half set to 0).
 *   workspace_dev       : device, qcd_workspace_bytes(lat, opts, 1) bytes.
 *   opts                : NULL = defaults. prec_inner = DOUBLE runs plain FP64 CG; SINGLE/HALF run
 *                         the mixed-precision CG with FP64 reliable updates (links for that
 *                         precision and for DOUBLE must both be loaded).
 *   info                : optional; filled on return.
 * Synchronises `stream` before returning. Returns QCD_ERR_NOT_CONVERGED when max_iter runs out,
 * QCD_ERR_BREAKDOWN when a CG scalar is non-finite or non-positive. */
QCD_API int qcd_cg_solve(qcd_lattice* lat, void* x_dev, const void* b_dev, double mass, double tol, int max_iter,
                 const qcd_solver_opts* opts, void* workspace_dev, void* y_dev, qcd_solve_info* info,
                 void* stream);

/* nrhs independent solves A x_r = b_r on one lattice in one set of launches: every link the
 * operator loads is applied to a register block of right-hand sides (opts->rhs_block), each RHS
 * keeps its own CG scalars and stops on its own (the batched-RHS form of the paper's congrad).
 *   x_dev, b_dev, y_dev : nrhs canonical fields back to back, complex128[nrhs][V][3] (y nullable).
 *   workspace_dev       : qcd_workspace_bytes(lat, opts, nrhs) bytes.
 *   info                : optional array of nrhs entries; the launch/profiling counters are
 *                         reported on entry 0.
 * 1 <= nrhs <= 16. Returns QCD_OK when every RHS converged, else the first failing status
 * (QCD_ERR_BREAKDOWN takes precedence). Synchronises `stream` before returning. */
QCD_API int qcd_cg_solve_mrhs(qcd_lattice* lat, int nrhs, void* x_dev, const void* b_dev, double mass, double tol,
                      int max_iter, const qcd_solver_opts* opts, void* workspace_dev, void* y_dev,
                      qcd_solve_info* info, void* stream);

/* Bytes of the device workspace qcd_cg_solve_batched needs for these n lattices (0 on a bad
 * argument). */
QCD_API size_t qcd_workspace_bytes_batched(int n, qcd_lattice* const lats[], const qcd_solver_opts* opts);

/* n independent solves A_i x_i = b_i on n lattices of any sizes and masses, in ONE persistent
 * launch (the paper's congrad applied to a batch): each thread-block cluster takes the next
 * lattice from a device work queue (longest expected solve first) and runs its whole CG there,
 * reliable updates and the final y / true residual included, with cluster-scope reductions and
 * no host round trip. With opts->use_graph and a non-default stream the launch is replayed from
 * a CUDA graph.
 *   lats[i] : links loaded at QCD_PREC_DOUBLE and at opts->prec_inner (same recon for all i).
 *   x[i], b[i], y[i] : device canonical fields of lattice i (y and its entries nullable).
 *   mass[i] : host array, > 0.   info : optional host array of n entries.
 * Synchronises `stream`. Returns QCD_OK when every lattice converged, else the first failing
 * status (QCD_ERR_BREAKDOWN first). */
QCD_API int qcd_cg_solve_batched(int n, qcd_lattice* const lats[], void* const x[], const void* const b[],
                         void* const y[], const double mass[], double tol, int max_iter,
                         const qcd_solver_opts* opts, void* workspace_dev, qcd_solve_info info[], void* stream);

/* Full-system solve M x = b with M = m + D on both parities (b, x: device canonical fields
 * complex128[V][3]), by even-odd reduction onto qcd_cg_solve: (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o,
 * then x_o = (b_o - D_oe x_e) / m. The even system is solved to tol * m |b| / |b_e'| so that the full
 * FP64 residual |b - M x| / |b|, recomputed at the end and returned in info->true_rel_residual,
 * meets tol. workspace_dev: qcd_workspace_bytes_full(lat, opts) bytes. Synchronises `stream`. */
QCD_API size_t qcd_workspace_bytes_full(const qcd_lattice* lat, const qcd_solver_opts* opts);
QCD_API int qcd_solve_full(qcd_lattice* lat, void* x_dev, const void* b_dev, double mass, double tol, int max_iter,
                   const qcd_solver_opts* opts, void* workspace_dev, qcd_solve_info* info, void* stream);

/* ---- fermion force (for the paper's molecular-dynamics program, §2, fed by the CG of §4) ------ */

/* The force of the even-site pseudofermion action S = phi_e^dagger (m^2 - D_eo D_oe)^-1 phi_e on
 * every link, from the two fields qcd_cg_solve returns: x = A^-1 phi_e (even sites) and
 * y = D_oe x (odd sites). force_dev[n][mu] is the traceless Hermitian 3x3 matrix G_mu(n) with
 * dS = eps tr(H G_mu(n)) when U_mu(n) -> exp(i eps H) U_mu(n) (H traceless Hermitian); with
 * c = eta_mu(n) zeta_mu(n) / 2 (zeta = the handle's tbc on the last time slice's t-links),
 *   n even: W = c (U_mu(n) y(n+mu)) x(n)^dagger;   n odd: W = c y(n) (U_mu(n) x(n+mu))^dagger;
 *   G_mu(n) = i (W - W^dagger) - tr(i (W - W^dagger)) / 3.
 *   links_dev : device, canonical complex128[V][4][3][3] (the field given to qcd_load_links).
 *   x_dev, y_dev : device, complex128[V][3]; only the even half of x and the odd half of y are read.
 *   force_dev : device, complex128[V][4][3][3], overwritten; must not alias the inputs.
 * FP64 throughout; asynchronous on `stream`. */
QCD_API int qcd_fermion_force(const qcd_lattice* lat, void* force_dev, const void* links_dev, const void* x_dev,
                      const void* y_dev, void* stream);

/* ---- Wilson fermions (the paper's second program, §2 and §6) --------------------------------- */

/* Wilson hopping term on the full lattice (no even-odd reduction), DeGrand-Rossi gamma matrices
 * (mu = x, y, z, t), antiperiodic in t by the handle's tbc:
 *   D_W psi(n) = sum_mu [ (1 - gamma_mu) U_mu(n) psi(n+mu) + (1 + gamma_mu) U_mu(n-mu)^dagger psi(n-mu) ]
 *   M = 1 - kappa D_W,  M^dagger = gamma5 M gamma5,  gamma5 = diag(1, 1, -1, -1).
 * Canonical spinor field: complex128[V][4][3] (spin, colour); packed field: the library's
 * structure-of-arrays layout over all V sites (qcd_wilson_field_bytes). Precisions: DOUBLE, SINGLE
 * and DF64 (float4 {re.hi, re.lo, im.hi, im.lo} per complex, 16 bytes like DOUBLE; the multi-RHS
 * operator takes DOUBLE and SINGLE only). */
enum { QCD_WILSON_DSLASH = 0, QCD_WILSON_M = 1, QCD_WILSON_MDAG = 2 };
QCD_API size_t qcd_wilson_field_bytes(const qcd_lattice* lat, int prec);
QCD_API size_t qcd_wilson_links_bytes(const qcd_lattice* lat, int prec);
/* Pack the canonical links for the Wilson operator (the tbc sign folded into the last time slice's
 * t-links) into packed_dev and register them for `prec`. */
QCD_API int qcd_wilson_load_links(qcd_lattice* lat, const void* links_dev, void* packed_dev, int prec, void* stream);
QCD_API int qcd_wilson_pack_field(const qcd_lattice* lat, void* packed_dev, const void* canonical_dev, int prec,
                          void* stream);
QCD_API int qcd_wilson_unpack_field(const qcd_lattice* lat, void* canonical_dev, const void* packed_dev, int prec,
                            void* stream);
/* out = D_W in (op 0), M in (op 1) or M^dagger in (op 2); packed fields at `prec`, no aliasing.
 * A spin-projected kernel: each hop multiplies two colour vectors by the link. */
QCD_API int qcd_wilson_op(const qcd_lattice* lat, void* out_dev, const void* in_dev, double kappa, int op, int prec,
                  void* stream);
/* The same operator on nrhs right-hand sides at once: nrhs packed fields back to back
 * (nrhs * qcd_wilson_field_bytes bytes each side); one thread per site walks all nrhs right-hand
 * sides, applying each loaded link to one RHS at a time. 1 <= nrhs <= 16. */
QCD_API int qcd_wilson_op_mrhs(const qcd_lattice* lat, void* out_dev, const void* in_dev, int nrhs, double kappa,
                       int op, int prec, void* stream);
/* Bytes of the device workspace qcd_wilson_cgnr (nrhs = 1) or qcd_wilson_cgnr_mrhs needs for these
 * options; 0 on a bad argument (nrhs outside [1, 16], unsupported precision). */
QCD_API size_t qcd_wilson_workspace_bytes(const qcd_lattice* lat, const qcd_solver_opts* opts, int nrhs);
/* CGNR: M^dagger M x = M^dagger b to |M^dagger b - M^dagger M x| / |M^dagger b| <= tol (recomputed at
 * the outer precision, returned in info->true_rel_residual); canonical spinor fields
 * complex128[V][4][3].
 * opts->prec_inner = SINGLE runs the recursion in FP32 with reliable updates (opts->reliable_delta,
 * opts->reliable_interval): each update folds the FP32 increment into the high-precision solution,
 * recomputes the true residual b - M x at that precision and restarts the recursion from
 * M^dagger (b - M x); a RHS stops only after the full high-precision residual of the normal
 * equations confirms the tolerance. The high precision is opts->prec_outer: DOUBLE (FP64) or DF64
 * (about 1e-14 relative rounding; on GB300 its operator runs on the FP32 pipes, several times
 * faster than the FP64 pipe). Links must be loaded at prec_inner and at prec_outer. DOUBLE inner
 * precision runs plain FP64 CGNR, confirmed the same way (prec_outer must then be DOUBLE).
 * Synchronises `stream`.
 * Returns QCD_ERR_NOT_CONVERGED when max_iter runs out, QCD_ERR_BREAKDOWN on a non-finite or
 * non-positive CG scalar. */
QCD_API int qcd_wilson_cgnr(qcd_lattice* lat, void* x_dev, const void* b_dev, double kappa, double tol, int max_iter,
                    const qcd_solver_opts* opts, void* workspace_dev, qcd_solve_info* info, void* stream);
/* nrhs independent CGNR solves on one lattice in one set of launches: each loaded link is applied to
 * a register block of right-hand sides (opts->rhs_block: 0 = 1; 1, 2, 4 in SINGLE; 1, 2 in
 * DOUBLE), each RHS keeps its own scalars, reliable updates and exit.
 *   x_dev, b_dev  : nrhs canonical fields back to back, complex128[nrhs][V][4][3].
 *   workspace_dev : qcd_wilson_workspace_bytes(lat, opts, nrhs) bytes.
 *   info          : optional array of nrhs entries; the launch counters and, with opts->profile, the
 *                   summed time of the operator launches (dslash_ms over dslash_launches) are
 *                   reported on entry 0.
 * 1 <= nrhs <= 16. Returns QCD_OK when every RHS converged, else the first failing status
 * (QCD_ERR_BREAKDOWN takes precedence). Synchronises `stream`. */
QCD_API int qcd_wilson_cgnr_mrhs(qcd_lattice* lat, int nrhs, void* x_dev, const void* b_dev, double kappa, double tol,
                         int max_iter, const qcd_solver_opts* opts, void* workspace_dev, qcd_solve_info* info,
                         void* stream);

/* ---- autotuning of launch shapes (no counterpart in the paper) ------------------------------ */

/* Time the multi-RHS solver's operator launches (CUDA events over a 24-iteration run of the real
 * solve on the caller's buffers, the same arguments as qcd_cg_solve_mrhs) for the shared-link
 * kernel (-1, from 2 RHS on) and each register block of right-hand sides, store the fastest in the
 * in-process table used when opts->rhs_block == 0,
 * append it to `cache_path` (nullable) and return it in *best_rhs_block. x_dev is overwritten. */
QCD_API int qcd_tune_mrhs(qcd_lattice* lat, int nrhs, void* x_dev, const void* b_dev, double mass,
                  const qcd_solver_opts* opts, void* workspace_dev, const char* cache_path, int* best_rhs_block,
                  void* stream);
/* Time whole batched solves (same arguments as qcd_cg_solve_batched, y omitted) for every
 * (cluster size in {1,2,4,8,16}, block size in {128,256}) that fits; keep the fastest for
 * opts->cluster_size == 0 / opts->block_size == 0, append it to `cache_path` (nullable). */
QCD_API int qcd_tune_batched(int n, qcd_lattice* const lats[], void* const x[], const void* const b[],
                     const double mass[], double tol, int max_iter, const qcd_solver_opts* opts,
                     void* workspace_dev, const char* cache_path, int* best_cluster, int* best_block,
                     void* stream);
/* Load tuned entries written by the two calls above (missing file = nothing to load; a line whose
 * shape the solvers do not accept, e.g. hand-edited or truncated, is skipped). */
QCD_API int qcd_tune_load(const char* cache_path);

#ifdef __cplusplus
}
#endif

#endif /* QCD_H */
