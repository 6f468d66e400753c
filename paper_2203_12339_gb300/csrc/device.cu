// Per-thread error strings, device checks and the device status word.
#include <atomic>
#include <cstdarg>
#include <mutex>
#include <map>
#include <utility>
#include <vector>

#include "tsr_internal.cuh"

namespace tsr {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

const char *error_string() { return g_err; }

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }

// Optional device timing of the transfer's tensor-core kernel (tsr_kernel_timing): a
// pair of CUDA events around each launch, read and released by tsr_kernel_timing_read.
static std::atomic<int> g_timing{0};
static std::mutex g_timing_mu;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_timing_ev;

KernelTimer::KernelTimer(cudaStream_t stream) : s(stream) {
  if (!g_timing.load(std::memory_order_relaxed)) return;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess || cudaEventRecord(a, s) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    a = b = nullptr;
  }
}

void KernelTimer::stop() {
  if (!a) return;
  if (cudaEventRecord(b, s) == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timing_ev.emplace_back(a, b);
  } else {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  a = b = nullptr;
}

// Host-side fault injection (tsr_fault_inject): per kind, how many more occurrences fail.
static std::atomic<int> g_fault[4];
bool fault_hit(int kind) {
  if (kind < 1 || kind > 3) return false;
  int n = g_fault[kind].load(std::memory_order_relaxed);
  while (n > 0)
    if (g_fault[kind].compare_exchange_weak(n, n - 1, std::memory_order_relaxed)) return true;
  return false;
}

static std::mutex g_mu;
static std::map<int, unsigned *> g_status;   // device -> status word
static std::map<int, int> g_sms;

tsr_status require_device() {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("no CUDA device: %s", cudaGetErrorString(e));
    return TSR_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_sms.count(dev)) return TSR_OK;
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) {
    set_error("cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    return TSR_ERR_CUDA;
  }
  if (!(prop.major == 10 && prop.minor == 3)) {
    set_error("libtsr is built for sm_103a only; device %d is sm_%d%d (%s)", dev, prop.major, prop.minor,
              prop.name);
    return TSR_ERR_UNSUPPORTED;
  }
  g_sms[dev] = prop.multiProcessorCount;
  return TSR_OK;
}

tsr_status require_same_device(int device, const char *who) {
  int dev = -1;
  TSR_CUDA(cudaGetDevice(&dev));
  if (dev != device) {
    set_error("%s: the handle lives on device %d, the current device is %d", who, device, dev);
    return TSR_ERR_INVALID_ARG;
  }
  return TSR_OK;
}

int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_sms.find(dev);
  return it == g_sms.end() ? 148 : it->second;
}

unsigned *device_status_ptr() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_status.find(dev);
  if (it != g_status.end()) return it->second;
  unsigned *p = nullptr;
  if (cudaMalloc(&p, sizeof(unsigned)) != cudaSuccess) return nullptr;
  cudaMemset(p, 0, sizeof(unsigned));
  cudaDeviceSynchronize();
  g_status[dev] = p;
  return p;
}

tsr_status check_device_status(cudaStream_t s) {
  if (fault_hit(FAULT_TIMEOUT)) {
    TSR_CUDA(cudaStreamSynchronize(s));
    set_error("injected fault: a bounded wait ran out (tsr_fault_inject); outputs are undefined");
    return TSR_ERR_TIMEOUT;
  }
  unsigned *p = device_status_ptr();
  if (!p) {
    set_error("device status word unavailable");
    return TSR_ERR_CUDA;
  }
  unsigned h = 0;
  TSR_CUDA(cudaMemcpyAsync(&h, p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  TSR_CUDA(cudaStreamSynchronize(s));
  if (h) {
    TSR_CUDA(cudaMemsetAsync(p, 0, sizeof(unsigned), s));
    TSR_CUDA(cudaStreamSynchronize(s));
    if (h & DEV_ERR_TIMEOUT) {
      set_error("a kernel's bounded wait ran out (status 0x%x); outputs are undefined", h);
      return TSR_ERR_TIMEOUT;
    }
    set_error("a kernel reported an out-of-range access (status 0x%x)", h);
    return TSR_ERR_CUDA;
  }
  return TSR_OK;
}

}  // namespace tsr

extern "C" uint64_t tsr_kernel_launches(void) { return (uint64_t)tsr::launches(); }

extern "C" tsr_status tsr_kernel_timing(int enable) {
  TSR_API_ENTRY();
  tsr::g_timing.store(enable ? 1 : 0, std::memory_order_relaxed);
  return TSR_OK;
}

extern "C" tsr_status tsr_kernel_timing_read(double *total_ms, int *launches) {
  TSR_API_ENTRY();
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  {
    std::lock_guard<std::mutex> lk(tsr::g_timing_mu);
    ev.swap(tsr::g_timing_ev);
  }
  double sum = 0.0;
  cudaError_t err = cudaSuccess;
  for (auto &p : ev) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(p.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.first, p.second);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    sum += ms;
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  if (total_ms) *total_ms = sum;
  if (launches) *launches = (int)ev.size();
  if (err != cudaSuccess) {
    tsr::set_error("tsr_kernel_timing_read: %s", cudaGetErrorString(err));
    return TSR_ERR_CUDA;
  }
  return TSR_OK;
}

extern "C" tsr_status tsr_fault_inject(int kind, int n) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(kind >= TSR_FAULT_ALLOC && kind <= TSR_FAULT_TIMEOUT, "tsr_fault_inject: kind=%d unknown", kind);
  TSR_CHECK_ARG(n >= 0 && n <= (1 << 20), "tsr_fault_inject: n=%d out of range", n);
  tsr::g_fault[kind].store(n, std::memory_order_relaxed);
  return TSR_OK;
}
