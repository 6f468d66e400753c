// tsr_relight_noalloc: the relight of tsr_relight for callers that must not
// allocate device memory.
//
// Who needs it: a host application that hands out all device memory itself
// and forbids allocations after start-up (for example a render loop that owns a
// fixed memory budget, or a plugin inside such a host), and code that must not
// pay for, or may not issue, an allocation call in the middle of a frame.
// tsr_relight takes its intermediate buffers (the light-contracted transfer Y and
// its inverse Haar Z, K (10 P^2 + 2 + N) floats, whatever the number of edits;
// for one or two edits the wavelet images b^w, at most 6 (10 P^2 + 2) floats)
// from cudaMallocAsync; this variant takes them from a fixed array in device
// memory that the library reserves when it is loaded, so the call itself
// allocates nothing.
#include <mutex>

#include "handles.cuh"

namespace {

// Scratch for Y and Z (or b^w) and the run approximations of the two-kernel inverse
// Haar of charts larger than 32 x 32: 8 Mi floats = 32 MiB (the largest case, K = 16
// on a 163,842-vertex mesh, needs 5.2 Mi).  Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t kNoallocScratchFloats = size_t(8) << 20;
static __device__ __align__(256) float g_relight_scratch[kNoallocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_scratch_ptr[kMaxDevices] = {};   // device address of the array, per device (set up once)

// In host code `g_relight_scratch` names a host-side stand-in, not device
// memory; the device address comes from cudaGetSymbolAddress, once per device,
// with that device current.
tsr_status scratch_for_current_device(float **out) {
  int dev = -1;
  TSR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    tsr::set_error("tsr_relight_noalloc: device index %d beyond the supported %d", dev, kMaxDevices);
    return TSR_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    TSR_CUDA(cudaGetSymbolAddress(&p, g_relight_scratch));
    g_scratch_ptr[dev] = static_cast<float *>(p);
  }
  *out = g_scratch_ptr[dev];
  return TSR_OK;
}

}  // namespace

extern "C" tsr_status tsr_relight_noalloc(const tsr_compressed *c, int n_edit, const float *g, const float *l,
                                          float *B, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(c && g && l && B, "tsr_relight_noalloc: NULL argument");
  TSR_CHECK_ARG(n_edit >= 0 && n_edit <= (1 << 20), "tsr_relight_noalloc: n_edit=%d out of range", n_edit);
  TSR_CHECK_ARG(tsr::aligned(g, 4) && tsr::aligned(l, 4) && tsr::aligned(B, 4), "tsr_relight_noalloc: misaligned pointer");
  const size_t need = tsr::relight_scratch_floats(c);
  TSR_CHECK_ARG(need <= kNoallocScratchFloats,
                "tsr_relight_noalloc: the relight needs %zu floats of scratch, beyond the fixed %zu floats", need,
                kNoallocScratchFloats);
  tsr_status st = tsr::require_device();
  if (st == TSR_OK) st = tsr::require_same_device(c->device, "tsr_relight_noalloc");
  if (st != TSR_OK || n_edit == 0) return st;
  float *scratch = nullptr;
  st = scratch_for_current_device(&scratch);
  if (st != TSR_OK) return st;
  // Every intermediate the relight reads from the array is written earlier in the
  // same call, so the array needs no clearing between calls.
  return tsr::relight_with_scratch(c, n_edit, g, l, B, scratch, reinterpret_cast<cudaStream_t>(stream));
}
