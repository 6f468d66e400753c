// Section 3.2, Eq. 9-10 and precompute Step 2: the spatial wavelet w_1 of the
// transfer over the rhombic surface charts and the truncation of its
// coefficients.
//
// Chart d of the mesh holds vertex ids d nu^2 + r nu + c (r, c < nu).  Its
// values are placed at Morton positions of a P x P domain (P = 2^ceil(log2 nu),
// zero padding) and analysed by the orthonormal 1D Haar: each level maps pairs
// (a, b) to ((a+b)/sqrt2, (a-b)/sqrt2); details of the level with current
// length n land at [n/2, n).  The two pole values pass through.
#include <algorithm>
#include <vector>

#include "handles.cuh"

namespace tsr {

__device__ __forceinline__ int morton2(int r, int c, int bits) {
  int m = 0;
  for (int b = 0; b < bits; ++b) {
    m |= ((c >> b) & 1) << (2 * b);
    m |= ((r >> b) & 1) << (2 * b + 1);
  }
  return m;
}

// ---------------------------------------------------------------- Haar forward
// One block per (row, chart).  Approximations ping-pong in shared memory; the
// details of each level are final and are written straight to global memory.
__global__ void __launch_bounds__(1024) haar_forward_kernel(const float *__restrict__ X, int nu, int P, int bits,
                                                           int N, int NW, float *__restrict__ Xw) {
  extern __shared__ float sh[];
  const int P2 = P * P;
  float *b0 = sh, *b1 = sh + P2;
  const int row = blockIdx.x / 10, d = blockIdx.x % 10;
  const float *x = X + (size_t)row * N + (size_t)d * nu * nu;
  float *out = Xw + (size_t)row * NW + (size_t)d * P2;
  if (nu != P)
    for (int q = threadIdx.x; q < P2; q += blockDim.x) b0[q] = 0.0f;
  __syncthreads();
  for (int q = threadIdx.x; q < nu * nu; q += blockDim.x) b0[morton2(q / nu, q % nu, bits)] = x[q];
  __syncthreads();
  const float rs2 = 0.70710678118654752440f;
  float *src = b0, *dst = b1;
  for (int n = P2; n > 1; n >>= 1) {
    const int h = n >> 1;
    for (int t = threadIdx.x; t < h; t += blockDim.x) {
      const float a = src[2 * t], b = src[2 * t + 1];
      dst[t] = (a + b) * rs2;
      out[h + t] = (a - b) * rs2;
    }
    __syncthreads();
    float *tmp = src;
    src = dst;
    dst = tmp;
  }
  if (threadIdx.x == 0) {
    out[0] = src[0];
    if (d == 0) {
      Xw[(size_t)row * NW + 10 * (size_t)P2] = X[(size_t)row * N + 10 * (size_t)nu * nu];
      Xw[(size_t)row * NW + 10 * (size_t)P2 + 1] = X[(size_t)row * N + 10 * (size_t)nu * nu + 1];
    }
  }
}

// ---------------------------------------------------------------- Haar inverse
__global__ void __launch_bounds__(1024) haar_inverse_kernel(const float *__restrict__ Xw, int nu, int P, int bits,
                                                           int N, int NW, float *__restrict__ X) {
  extern __shared__ float sh[];
  const int P2 = P * P;
  float *b0 = sh, *b1 = sh + P2;
  const int row = blockIdx.x / 10, d = blockIdx.x % 10;
  const float *cw = Xw + (size_t)row * NW + (size_t)d * P2;
  float *x = X + (size_t)row * N + (size_t)d * nu * nu;
  if (threadIdx.x == 0) b0[0] = cw[0];
  __syncthreads();
  const float rs2 = 0.70710678118654752440f;
  float *src = b0, *dst = b1;
  for (int n = 1; n < P2; n <<= 1) {   // src holds n approximations, details at [n, 2n)
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const float a = src[t], dd = cw[n + t];
      dst[2 * t] = (a + dd) * rs2;
      dst[2 * t + 1] = (a - dd) * rs2;
    }
    __syncthreads();
    float *tmp = src;
    src = dst;
    dst = tmp;
  }
  for (int q = threadIdx.x; q < nu * nu; q += blockDim.x) x[q] = src[morton2(q / nu, q % nu, bits)];
  if (threadIdx.x == 0 && d == 0) {
    X[(size_t)row * N + 10 * (size_t)nu * nu] = Xw[(size_t)row * NW + 10 * (size_t)P2];
    X[(size_t)row * N + 10 * (size_t)nu * nu + 1] = Xw[(size_t)row * NW + 10 * (size_t)P2 + 1];
  }
}

static int haar_threads(int P2) { return std::min(1024, std::max(32, P2 / 2)); }

tsr_status haar_forward(const float *X, int rows, int nu, float *Xw, cudaStream_t s) {
  const int P = chart_side(nu), bits = ilog2(P);
  const int N = 10 * nu * nu + 2, NW = 10 * P * P + 2;
  const size_t smem = sizeof(float) * (size_t)P * P * 2;
  TSR_CUDA(cudaFuncSetAttribute(haar_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  haar_forward_kernel<<<rows * 10, haar_threads(P * P), smem, s>>>(X, nu, P, bits, N, NW, Xw); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

tsr_status haar_inverse(const float *Xw, int rows, int nu, float *X, cudaStream_t s) {
  const int P = chart_side(nu), bits = ilog2(P);
  const int N = 10 * nu * nu + 2, NW = 10 * P * P + 2;
  const size_t smem = sizeof(float) * (size_t)P * P * 2;
  TSR_CUDA(cudaFuncSetAttribute(haar_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  haar_inverse_kernel<<<rows * 10, haar_threads(P * P), smem, s>>>(Xw, nu, P, bits, N, NW, X); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

// ---------------------------------------------------------------- top-p selection
// One block per (k, j) row.  Radix select (4 x 8 bits) of the n_keep-th largest
// |c| over the chart coefficients, then a block scan in index order that keeps
// every larger value and the first (n_keep - #larger) values equal to it.
__global__ void __launch_bounds__(1024) select_kernel(const float *__restrict__ Mw, int n_coef, int NW, int n_keep,
                                                     uint8_t *__restrict__ keep) {
  __shared__ unsigned hist[256];
  __shared__ unsigned s_sel, s_cum;
  __shared__ unsigned warp_tot[32];
  const int rowi = blockIdx.x;
  const float *c = Mw + (size_t)rowi * NW;
  uint8_t *kp = keep + (size_t)rowi * NW;
  unsigned prefix = 0, mask = 0, remaining = (unsigned)n_keep;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int q = threadIdx.x; q < 256; q += blockDim.x) hist[q] = 0;
    __syncthreads();
    for (int w = threadIdx.x; w < n_coef; w += blockDim.x) {
      const unsigned u = __float_as_uint(c[w]) & 0x7FFFFFFFu;
      if ((u & mask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned cum = 0;
      int sel = 0;
      for (int dgt = 255; dgt >= 0; --dgt) {
        if (cum + hist[dgt] >= remaining) {
          sel = dgt;
          break;
        }
        cum += hist[dgt];
      }
      s_sel = (unsigned)sel;
      s_cum = cum;
    }
    __syncthreads();
    remaining -= s_cum;
    prefix |= s_sel << shift;
    mask |= 255u << shift;
    __syncthreads();
  }
  // prefix = key of the n_keep-th largest; keep `remaining` of the equal keys (lowest index first)
  const unsigned tau = prefix;
  unsigned taken_before = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < n_coef; base += blockDim.x) {
    const int w = base + threadIdx.x;
    unsigned u = 0;
    if (w < n_coef) u = __float_as_uint(c[w]) & 0x7FFFFFFFu;
    const bool eq = (w < n_coef) && (u == tau);
    const unsigned bal = __ballot_sync(0xffffffffu, eq);
    const unsigned before_in_warp = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    unsigned before_warps = 0, total = 0;
    for (int q = 0; q < nw; ++q) {
      const unsigned v = warp_tot[q];
      if (q < warp) before_warps += v;
      total += v;
    }
    if (w < n_coef) {
      const bool keepit = (u > tau) || (eq && (taken_before + before_warps + before_in_warp) < remaining);
      kp[w] = keepit ? 1 : 0;
    }
    taken_before += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    kp[n_coef] = 1;
    kp[n_coef + 1] = 1;
  }
}

// Column view: block per kj compacts its kept rows in ascending order.
__global__ void __launch_bounds__(1024) pack_columns_kernel(const float *__restrict__ Mw,
                                                           const uint8_t *__restrict__ keep, int NW, int ncol,
                                                           int32_t *__restrict__ cidx, float *__restrict__ cval) {
  __shared__ unsigned warp_tot[32];
  const int kj = blockIdx.x;
  const uint8_t *kp = keep + (size_t)kj * NW;
  const float *c = Mw + (size_t)kj * NW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned written = 0;
  for (int base = 0; base < NW; base += blockDim.x) {
    const int w = base + threadIdx.x;
    const bool k = (w < NW) && kp[w];
    const unsigned bal = __ballot_sync(0xffffffffu, k);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, total = 0;
    for (int q = 0; q < nw; ++q) {
      before += (q < warp) ? warp_tot[q] : 0u;
      total += warp_tot[q];
    }
    const unsigned pos = written + before + __popc(bal & ((1u << lane) - 1u));
    if (k && pos < (unsigned)ncol) {
      cidx[(size_t)kj * ncol + pos] = w;
      cval[(size_t)kj * ncol + pos] = c[w];
    }
    written += total;
    __syncthreads();
  }
}

// entries per wavelet row w (over all kj)
__global__ void count_kernel(const uint8_t *__restrict__ keep, int KJ, int NW, int64_t *__restrict__ cnt) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= NW) return;
  int64_t n = 0;
  for (int kj = 0; kj < KJ; ++kj) n += keep[(size_t)kj * NW + w];
  cnt[w] = n;
}

// exclusive scan of cnt[0..n) into row_ptr[0..n] (single block; n is a few 1e5)
__global__ void __launch_bounds__(1024) scan_kernel(const int64_t *__restrict__ cnt, int n, int64_t *__restrict__ row_ptr) {
  __shared__ int64_t warp_sum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int64_t v = i < n ? cnt[i] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t ws = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sum[lane] = ws;
    }
    __syncthreads();
    const int64_t incl = x + (warp > 0 ? warp_sum[warp - 1] : 0) + carry;
    if (i < n) row_ptr[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) row_ptr[n] = carry;
}

__global__ void fill_kernel(const float *__restrict__ Mw, const uint8_t *__restrict__ keep, int KJ, int NW,
                            const int64_t *__restrict__ row_ptr, uint16_t *__restrict__ col, float *__restrict__ val) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= NW) return;
  int64_t p = row_ptr[w];
  for (int kj = 0; kj < KJ; ++kj) {
    if (keep[(size_t)kj * NW + w]) {
      col[p] = (uint16_t)kj;
      val[p] = Mw[(size_t)kj * NW + w];
      ++p;
    }
  }
}

static int keep_count(double p, int n_coef) {
  double v = std::floor(p * (double)n_coef + 0.5);
  if (v < 1.0) v = 1.0;
  if (v > (double)n_coef) v = (double)n_coef;
  return (int)v;
}

// Selection + packing into an existing handle (its K, J, nu and n_keep).
tsr_status wavelet_compress_into(const float *Mw, tsr_compressed *c, cudaStream_t s) {
  const int NW = c->n_rows, n_coef = NW - 2, KJ = c->K * c->J;
  Scratch keep_s, cnt_s;
  tsr_status st = keep_s.alloc((size_t)KJ * NW, s);
  if (st == TSR_OK) st = cnt_s.alloc(sizeof(int64_t) * NW, s);
  if (st != TSR_OK) return st;
  uint8_t *keep = static_cast<uint8_t *>(keep_s.p);
  int64_t *cnt = static_cast<int64_t *>(cnt_s.p);
  select_kernel<<<KJ, 1024, 0, s>>>(Mw, n_coef, NW, c->n_keep, keep); ::tsr::count_launch();
  count_kernel<<<(NW + 255) / 256, 256, 0, s>>>(keep, KJ, NW, cnt); ::tsr::count_launch();
  scan_kernel<<<1, 1024, 0, s>>>(cnt, NW, c->row_ptr); ::tsr::count_launch();
  fill_kernel<<<(NW + 255) / 256, 256, 0, s>>>(Mw, keep, KJ, NW, c->row_ptr, c->col, c->val); ::tsr::count_launch();
  pack_columns_kernel<<<KJ, 1024, 0, s>>>(Mw, keep, NW, c->n_keep + 2, c->cidx, c->cval); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

tsr_status wavelet_compress(const float *Mw, int K, int J, int nu, double p, tsr_compressed **out, cudaStream_t s) {
  const int P = chart_side(nu);
  const int n_coef = 10 * P * P, NW = n_coef + 2, KJ = K * J;
  tsr_compressed *c = new tsr_compressed();
  cudaGetDevice(&c->device);
  c->K = K;
  c->J = J;
  c->nu = nu;
  c->P = P;
  c->n_rows = NW;
  c->n_keep = keep_count(p, n_coef);
  c->nnz = (int64_t)KJ * (c->n_keep + 2);
  cudaError_t e = cudaMalloc(&c->row_ptr, sizeof(int64_t) * (NW + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->col, sizeof(uint16_t) * c->nnz);
  if (e == cudaSuccess) e = cudaMalloc(&c->val, sizeof(float) * c->nnz);
  if (e == cudaSuccess) e = cudaMalloc(&c->cidx, sizeof(int32_t) * c->nnz);
  if (e == cudaSuccess) e = cudaMalloc(&c->cval, sizeof(float) * c->nnz);
  if (e != cudaSuccess) {
    set_error("wavelet_compress: %s", cudaGetErrorString(e));
    tsr_compressed_destroy(c);
    return e == cudaErrorMemoryAllocation ? TSR_ERR_OOM : TSR_ERR_CUDA;
  }
  tsr_status st = wavelet_compress_into(Mw, c, s);
  if (st != TSR_OK) {
    tsr_compressed_destroy(c);
    return st;
  }
  *out = c;
  return TSR_OK;
}

}  // namespace tsr

extern "C" void tsr_compressed_destroy(tsr_compressed *c) {
  if (!c) return;
  cudaFree(c->row_ptr);
  cudaFree(c->col);
  cudaFree(c->val);
  cudaFree(c->cidx);
  cudaFree(c->cval);
  delete c;
}
