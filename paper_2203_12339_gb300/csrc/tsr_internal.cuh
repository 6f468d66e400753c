// Internal helpers shared by the libtsr translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <cstdio>
#include <string>

#include "../../include/tsr.h"

namespace tsr {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();
const char *error_string();

#define TSR_CHECK_ARG(cond, ...)              \
  do {                                        \
    if (!(cond)) {                            \
      ::tsr::set_error(__VA_ARGS__);          \
      return TSR_ERR_INVALID_ARG;             \
    }                                         \
  } while (0)

// Host-side fault injection (tsr_fault_inject): true while injected failures of
// `kind` remain (each call consumes one).
enum { FAULT_ALLOC = 1, FAULT_CUDA = 2, FAULT_TIMEOUT = 3 };
bool fault_hit(int kind);

#define TSR_CUDA(call)                                                                            \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    bool injected_ = false;                                                                       \
    if (e_ == cudaSuccess && ::tsr::fault_hit(::tsr::FAULT_CUDA)) {                               \
      e_ = cudaErrorLaunchFailure; /* the call itself succeeded */                                \
      injected_ = true;                                                                           \
    }                                                                                             \
    if (e_ != cudaSuccess) {                                                                      \
      ::tsr::set_error("%s:%d: %s: %s%s", __FILE__, __LINE__, #call, cudaGetErrorString(e_),       \
                       injected_ ? " (injected fault, tsr_fault_inject)" : "");                   \
      return e_ == cudaErrorMemoryAllocation ? TSR_ERR_OOM : TSR_ERR_CUDA;                        \
    }                                                                                             \
  } while (0)

// NVTX range named after each C-ABI call, for profilers that show them (the NVTX v3
// headers are header-only; without a tool attached a range costs a test of a null
// pointer).  Absent headers leave the ranges out.
#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define TSR_HAVE_NVTX 1
#endif
#endif
struct NvtxRange {
  explicit NvtxRange(const char *name) {
#ifdef TSR_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~NvtxRange() {
#ifdef TSR_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
// First statement of every C-ABI call: clears the thread's error string and opens the call's range.
#define TSR_API_ENTRY()  \
  ::tsr::clear_error(); \
  ::tsr::NvtxRange tsr_api_range_(__func__)

// Device-side status word written by kernels whose bounded waits ran out.
// One word per device; kernels OR in a code, the host reads and clears it.
enum : unsigned { DEV_ERR_TIMEOUT = 1u, DEV_ERR_BOUNDS = 2u };
tsr_status check_device_status(cudaStream_t s);   // synchronises s
unsigned *device_status_ptr();                     // device address of the word (current device)

// Count of kernel launches made by the library (all threads, all devices).
void count_launch();

// Events around one kernel launch on stream s while tsr_kernel_timing is enabled
// (nothing otherwise): construct before the launch, stop() after it.
struct KernelTimer {
  explicit KernelTimer(cudaStream_t stream);
  void stop();
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
};

// Verifies that the current device is an sm_103 part (the only compiled target).
tsr_status require_device();
// TSR_ERR_INVALID_ARG unless `device` (where a handle was made) is the current device.
tsr_status require_same_device(int device, const char *who);
int num_sms();

// Stream-ordered scratch owned by one call.
struct Scratch {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
  tsr_status alloc(size_t bytes, cudaStream_t stream) {
    s = stream;
    if (fault_hit(FAULT_ALLOC)) {
      set_error("injected fault: cudaMallocAsync(%zu) failed (tsr_fault_inject)", bytes);
      return TSR_ERR_OOM;
    }
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? TSR_ERR_OOM : TSR_ERR_CUDA;
    }
    return TSR_OK;
  }
};

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline int chart_side(int nu) {
  int P = 1;
  while (P < nu) P *= 2;
  return P;
}
inline int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

// ---------------------------------------------------------------- PTX helpers (device)
#define TSR_WAIT_LIMIT 20000000u   // bounded spin iterations (~ seconds) before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < TSR_WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 2D tiled TMA load global -> shared, completion counted on an mbarrier.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void report_device_error(unsigned *status, unsigned code) {
  if (status) atomicOr(status, code);
}

}  // namespace tsr
