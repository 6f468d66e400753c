// Diagnostic: exercises the library's bounded-wait path.  One block waits,
// with an iteration limit, on an mbarrier phase that nothing completes; the
// wait gives up, the kernel records a timeout in the device status word and
// returns, leaving the context usable.
#include "tsr_internal.cuh"

namespace {
__global__ void bounded_wait_selftest_kernel(unsigned limit, unsigned *status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tsr::mbar_init(&bar, 1);
    tsr::fence_mbar_init();
  }
  __syncthreads();
  bool done = false;
  for (unsigned it = 0; it < limit && !done; ++it) done = tsr::mbar_try_wait(&bar, 0u);   // phase 0 never completes
  if (!done && threadIdx.x == 0) tsr::report_device_error(status, tsr::DEV_ERR_TIMEOUT);
  __syncthreads();
}
}  // namespace

extern "C" tsr_status tsr_selftest_bounded_wait(unsigned limit, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(limit >= 1 && limit <= 1000000u, "tsr_selftest_bounded_wait: limit=%u outside [1, 1e6]", limit);
  tsr_status st = tsr::require_device();
  if (st != TSR_OK) return st;
  unsigned *status = tsr::device_status_ptr();
  if (!status) {
    tsr::set_error("tsr_selftest_bounded_wait: device status word unavailable");
    return TSR_ERR_CUDA;
  }
  bounded_wait_selftest_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(limit, status);
  tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}
