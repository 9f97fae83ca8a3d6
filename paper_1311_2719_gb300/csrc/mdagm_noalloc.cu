// qcd_mdagm_noalloc: the even-site normal operator with its intermediate odd-parity field kept in
// a library-owned, statically sized device array instead of caller scratch.
//
// Some callers cannot hand the library a scratch buffer: host programs whose device arrays all
// come from compiler data directives or from another framework's memory pool have no way to
// call cudaMalloc (or are not allowed to, because that pool owns and accounts for every byte of
// the GPU). This entry point lets them apply m^2 - D_eo D_oe with only their input and output.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes. Every GPU that loads the
// library holds it until the process exits. Host code only ever sees a host-side stand-in for
// the array's name, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <mutex>

#include "dslash.cuh"

namespace qcd {

int launch_mdagm(const qcd_lattice*, void*, const void*, double, int, void*, cudaStream_t);
void set_error(const char* fmt, ...);
size_t device_span(const void* p);

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB: one packed odd field
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_mdagm_scratch[kNoAllocScratchBytes];

static std::mutex g_scratch_mutex;
// Per device: the context the address was looked up in, and the address. A device reset gives the
// device a new primary context in which the module (and the array) is loaded afresh, so the
// address is looked up again whenever the current context differs from the cached one.
struct ScratchSlot {
  void* ctx = nullptr;
  void* ptr = nullptr;
};
static ScratchSlot g_scratch_slot[kMaxDevices];

// The current context (the driver's cuCtxGetCurrent, fetched at run time), or nullptr when the
// driver does not provide it.
static void* current_context() {
  using GetCurrent = int (*)(void**);
  static const GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    cudaGetLastError();
    return (GetCurrent)f;
  }();
  void* ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

// Device address of g_mdagm_scratch on `dev` (the current device). The first use per device and
// context does the lookup; later calls read the cached pointer.
static int scratch_for_device(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d outside the supported range [0, %d)", dev, kMaxDevices);
    return QCD_ERR_UNSUPPORTED;
  }
  void* ctx = current_context();
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchSlot& slot = g_scratch_slot[dev];
  if (!slot.ptr || slot.ctx != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_mdagm_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
    slot.ptr = p;
    slot.ctx = ctx;
  }
  *out = slot.ptr;
  return QCD_OK;
}

}  // namespace qcd

using namespace qcd;

extern "C" int qcd_mdagm_noalloc(const qcd_lattice* lat, void* out_dev, const void* in_dev, double mass, int prec,
                                 void* stream) {
  if (!lat) { set_error("lat is NULL"); return QCD_ERR_INVALID_ARG; }
  if (!out_dev || !in_dev) { set_error("out_dev and in_dev must not be NULL"); return QCD_ERR_INVALID_ARG; }
  if (((uintptr_t)out_dev & 255u) || ((uintptr_t)in_dev & 255u)) {
    set_error("out_dev and in_dev must be 256-byte aligned");
    return QCD_ERR_INVALID_ARG;
  }
  if (out_dev == in_dev) { set_error("out_dev must not alias in_dev"); return QCD_ERR_INVALID_ARG; }
  if (prec != QCD_PREC_DOUBLE && prec != QCD_PREC_SINGLE && prec != QCD_PREC_HALF && prec != QCD_PREC_DF64) {
    set_error("unknown precision %d", prec);
    return QCD_ERR_INVALID_ARG;
  }
  if (!(mass > 0.0) || !(mass < 1e300)) { set_error("mass must be finite and > 0, got %g", mass); return QCD_ERR_INVALID_ARG; }
  const size_t need = field_bytes(prec, lat->Vh);
  if (need > kNoAllocScratchBytes) {
    set_error("qcd_mdagm_noalloc: one packed field of this lattice needs %zu bytes at precision %d, above the "
              "built-in scratch of %zu bytes; use qcd_mdagm with caller scratch", need, prec, kNoAllocScratchBytes);
    return QCD_ERR_INVALID_ARG;
  }
  if (!lat->links[prec].ptr || !lat->links[prec].recon) {
    set_error("no links loaded for precision %d (call qcd_load_links first)", prec);
    return QCD_ERR_NO_LINKS;
  }
  for (const void* p : {(const void*)out_dev, in_dev}) {
    const size_t have = device_span(p);
    if (have && have < need) {
      set_error("qcd_mdagm_noalloc: a field buffer has %zu bytes to the end of its device allocation, %zu needed",
                have, need);
      return QCD_ERR_INVALID_ARG;
    }
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  // The kernels run on the current device and the scratch is that device's copy of the array, so
  // the lattice's links must live there too.
  if (lat->device != dev) {
    set_error("the lattice belongs to device %d, current device is %d", lat->device, dev);
    return QCD_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;
  if (int rc = scratch_for_device(dev, &scratch)) return rc;
  // The scratch is overwritten at every site by the first half-lattice hop before it is read,
  // so nothing in it has to start at zero.
  return launch_mdagm(lat, out_dev, in_dev, mass, prec, scratch, (cudaStream_t)stream);
}
