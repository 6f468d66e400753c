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

// Morton position m of (r, c) in a P x P chart: c's bits at even positions of m,
// r's at odd ones; compact_bits recovers c from m and r from m >> 1.
__device__ __forceinline__ unsigned compact_bits(unsigned x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  x = (x | (x >> 8)) & 0x0000FFFFu;
  return x;
}

// Charts of more than HAAR_SEG Morton positions are transformed in two kernels:
// the first log2(HAAR_SEG) levels act on independent runs of HAAR_SEG positions
// (one block per run), the remaining levels on the runs' approximations (one
// block per chart).  Smaller charts take one block per chart.
constexpr int HAAR_SEG = 1024;
constexpr int HAAR_SEG_THREADS = 256;

// ---------------------------------------------------------------- Haar forward
// A problem is positions [seg S, (seg + 1) S) of chart d of a row (S = min(P^2, HAAR_SEG),
// a power of 4).  A thread takes Q = min(16, S) consecutive Morton positions (a square of the
// chart) and does the first log2 Q levels in registers; the next levels pair lanes of its
// warp through shuffles; a problem wider than a warp (S = 1024) finishes its last level in
// its first warp after one barrier.  Problems are packed HF_THREADS / (S / Q) to a logical
// block, and a persistent grid loops over the logical blocks.  Each level maps the pair
// (a, b) to (a + b) / sqrt2 and the detail (a - b) / sqrt2 (rounded adds and multiplies, no
// contraction); details are final and go straight to their global positions; the problem's
// approximation goes to A[row][d][seg] (or, for a whole chart, to Xw position 0, with the
// poles).
constexpr int HF_THREADS = 256;
constexpr int HF_GRID = 2048;   // persistent grid (logical blocks beyond it loop)
__host__ __device__ inline int hf_per_thread(int S) { return S < 16 ? S : 16; }
__host__ __device__ inline int hf_problems_per_block(int S) { return HF_THREADS / (S / hf_per_thread(S)); }

__device__ __forceinline__ void haar_forward_problems(const float *__restrict__ X, int nu, int P, long long ldx, int NW,
                                                      int S, float *__restrict__ Xw, float *__restrict__ A, int p0,
                                                      int n_prob, float *part) {
  const float rs2 = 0.70710678118654752440f;
  const int Q = hf_per_thread(S), T = S / Q;   // positions per thread, threads per problem
  const int P2 = P * P, nseg = P2 / S;
  const int slot = threadIdx.x / T, t = threadIdx.x - slot * T;
  const int p = p0 + slot;
  const bool act = p < n_prob;
  const int seg = act ? p % nseg : 0, d = act ? (p / nseg) % 10 : 0, row = act ? p / (nseg * 10) : 0;
  const float *x = X + (size_t)row * ldx + (size_t)d * nu * nu;
  float *out = Xw + (size_t)row * NW + (size_t)d * P2;
  float v[16];
  {
    const unsigned m0 = (unsigned)(seg * S + Q * t);
    const int r0 = (int)compact_bits(m0 >> 1), c0 = (int)compact_bits(m0);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      v[i] = 0.0f;
      const int r = r0 + (((i >> 1) & 1) | ((i >> 2) & 2)), c = c0 + ((i & 1) | ((i >> 1) & 2));
      if (i < Q && act && r < nu && c < nu) v[i] = x[r * nu + c];
    }
  }
  int n = S, ng = P2;   // the problem's and the whole chart's current approximation lengths
#pragma unroll
  for (int len = 16; len > 1; len >>= 1) {
    if (len <= Q) {
      const int h = len >> 1;
      float dd[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j < h) {
          dd[j] = __fmul_rn(__fsub_rn(v[2 * j], v[2 * j + 1]), rs2);
          v[j] = __fmul_rn(__fadd_rn(v[2 * j], v[2 * j + 1]), rs2);
        }
      }
      if (act) {
        float *o = out + (ng >> 1) + seg * (n >> 1) + h * t;   // h consecutive details, 8-byte aligned for h >= 2
        if (h >= 2) {
#pragma unroll
          for (int j = 0; j < 8; j += 2)
            if (j < h) *reinterpret_cast<float2 *>(o + j) = make_float2(dd[j], dd[j + 1]);
        } else {
          o[0] = dd[0];
        }
      }
      n >>= 1;
      ng >>= 1;
    }
  }
  // thread t now holds approximation t of the problem's n = T
  float a = v[0];
  const int TW = T < 32 ? T : 32;
  for (int w = 1; w < TW; w <<= 1) {
    const float o = __shfl_down_sync(0xffffffffu, a, w);
    if ((t & (2 * w - 1)) == 0) {
      if (act) out[(ng >> 1) + seg * (n >> 1) + t / (2 * w)] = __fmul_rn(__fsub_rn(a, o), rs2);
      a = __fmul_rn(__fadd_rn(a, o), rs2);
    }
    n >>= 1;
    ng >>= 1;
  }
  if (T > 32) {   // uniform: W = T / 32 warps per problem, one value each
    const int W = T / 32;
    if ((t & 31) == 0) part[threadIdx.x >> 5] = a;
    __syncthreads();
    if (t < 32) {   // the problem's first warp
      a = t < W ? part[(threadIdx.x >> 5) + t] : 0.0f;
      for (int w = 1; w < W; w <<= 1) {
        const float o = __shfl_down_sync(0xffffffffu, a, w);
        if ((t & (2 * w - 1)) == 0 && t < W) {
          if (act) out[(ng >> 1) + seg * (n >> 1) + t / (2 * w)] = __fmul_rn(__fsub_rn(a, o), rs2);
          a = __fmul_rn(__fadd_rn(a, o), rs2);
        }
        n >>= 1;
        ng >>= 1;
      }
    }
    __syncthreads();   // part is reused by the next logical block
  }
  if (t == 0 && act) {
    if (nseg == 1) {
      out[0] = a;
      if (d == 0) {
        Xw[(size_t)row * NW + 10 * (size_t)P2] = X[(size_t)row * ldx + 10 * (size_t)nu * nu];
        Xw[(size_t)row * NW + 10 * (size_t)P2 + 1] = X[(size_t)row * ldx + 10 * (size_t)nu * nu + 1];
      }
    } else {
      A[((size_t)row * 10 + d) * nseg + seg] = a;
    }
  }
}

__global__ void __launch_bounds__(HF_THREADS) haar_forward_kernel(const float *__restrict__ X, int nu, int P,
                                                                 long long ldx, int NW, int S, float *__restrict__ Xw,
                                                                 float *__restrict__ A, int n_prob, int n_lb) {
  __shared__ float part[HF_THREADS / 32];   // the warps' approximations (S = 1024)
  for (int lb = blockIdx.x; lb < n_lb; lb += gridDim.x)
    haar_forward_problems(X, nu, P, ldx, NW, S, Xw, A, lb * hf_problems_per_block(S), n_prob, part);
}

// The levels above the runs: block per (row, chart) over its nseg approximations.
__device__ __forceinline__ void haar_forward_top_block(const float *__restrict__ X, const float *__restrict__ A, int nu,
                                                       int P, long long ldx, int NW, int nseg, float *__restrict__ Xw,
                                                       int d, int row) {
  __shared__ float b[2][HAAR_SEG];
  const int P2 = P * P;
  float *out = Xw + (size_t)row * NW + (size_t)d * P2;
  for (int q = threadIdx.x; q < nseg; q += blockDim.x) b[0][q] = A[((size_t)row * 10 + d) * nseg + q];
  __syncthreads();
  const float rs2 = 0.70710678118654752440f;
  int cur = 0;
  for (int n = nseg; n > 1; n >>= 1) {
    const int h = n >> 1;
    for (int t = threadIdx.x; t < h; t += blockDim.x) {
      const float a = b[cur][2 * t], bb = b[cur][2 * t + 1];
      b[cur ^ 1][t] = (a + bb) * rs2;
      out[h + t] = (a - bb) * rs2;
    }
    __syncthreads();
    cur ^= 1;
  }
  if (threadIdx.x == 0) {
    out[0] = b[cur][0];
    if (d == 0) {
      Xw[(size_t)row * NW + 10 * (size_t)P2] = X[(size_t)row * ldx + 10 * (size_t)nu * nu];
      Xw[(size_t)row * NW + 10 * (size_t)P2 + 1] = X[(size_t)row * ldx + 10 * (size_t)nu * nu + 1];
    }
  }
}

__global__ void haar_forward_top_kernel(const float *__restrict__ X, const float *__restrict__ A, int nu, int P,
                                        long long ldx, int NW, int nseg, float *__restrict__ Xw) {
  haar_forward_top_block(X, A, nu, P, ldx, NW, nseg, Xw, blockIdx.x % 10, blockIdx.x / 10);
}

// ---------------------------------------------------------------- Haar inverse
// The levels above the runs: the nseg approximations of each (row, chart) into A.
__global__ void haar_inverse_top_kernel(const float *__restrict__ Xw, int P, int NW, int nseg,
                                        float *__restrict__ A) {
  __shared__ float b[2][HAAR_SEG];
  const int d = blockIdx.x % 10, row = blockIdx.x / 10;
  const float *cw = Xw + (size_t)row * NW + (size_t)d * P * P;
  if (threadIdx.x == 0) b[0][0] = cw[0];
  __syncthreads();
  const float rs2 = 0.70710678118654752440f;
  int cur = 0;
  for (int n = 1; n < nseg; n <<= 1) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const float a = b[cur][t], dd = cw[n + t];
      b[cur ^ 1][2 * t] = (a + dd) * rs2;
      b[cur ^ 1][2 * t + 1] = (a - dd) * rs2;
    }
    __syncthreads();
    cur ^= 1;
  }
  for (int q = threadIdx.x; q < nseg; q += blockDim.x) A[((size_t)row * 10 + d) * nseg + q] = b[cur][q];
}

// Levels inside run seg of chart d (its approximation from A, or cw[0] for a whole
// chart), then the values scattered from Morton positions to vertex ids.
__global__ void __launch_bounds__(1024) haar_inverse_kernel(const float *__restrict__ Xw, const float *__restrict__ A,
                                                           int nu, int P, int N, int NW, int seg_len,
                                                           float *__restrict__ X) {
  extern __shared__ float sh[];
  float *b0 = sh, *b1 = sh + seg_len;
  const int P2 = P * P, nseg = P2 / seg_len;
  const int seg = blockIdx.x % nseg, d = (blockIdx.x / nseg) % 10, row = blockIdx.x / (nseg * 10);
  const float *cw = Xw + (size_t)row * NW + (size_t)d * P2;
  float *x = X + (size_t)row * N + (size_t)d * nu * nu;
  if (threadIdx.x == 0) b0[0] = (nseg == 1) ? cw[0] : A[((size_t)row * 10 + d) * nseg + seg];
  __syncthreads();
  const float rs2 = 0.70710678118654752440f;
  float *src = b0, *dst = b1;
  for (int n = 1; n < seg_len; n <<= 1) {   // src: n approximations of the run; details at [ng, 2 ng) globally
    const int ng = nseg * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const float a = src[t], dd = cw[ng + seg * n + t];
      dst[2 * t] = (a + dd) * rs2;
      dst[2 * t + 1] = (a - dd) * rs2;
    }
    __syncthreads();
    float *tmp = src;
    src = dst;
    dst = tmp;
  }
  for (int q = threadIdx.x; q < seg_len; q += blockDim.x) {
    const unsigned m = (unsigned)(seg * seg_len + q);
    const int r = (int)compact_bits(m >> 1), c = (int)compact_bits(m);
    if (r < nu && c < nu) x[r * nu + c] = src[q];
  }
  if (threadIdx.x == 0 && d == 0 && seg == 0) {
    X[(size_t)row * N + 10 * (size_t)nu * nu] = Xw[(size_t)row * NW + 10 * (size_t)P2];
    X[(size_t)row * N + 10 * (size_t)nu * nu + 1] = Xw[(size_t)row * NW + 10 * (size_t)P2 + 1];
  }
}

static int haar_threads(int len) { return std::min(1024, std::max(32, len / 2)); }

tsr_status haar_forward(const float *X, int rows, int nu, float *Xw, cudaStream_t s) {
  return haar_forward_ld(X, 10 * (long long)nu * nu + 2, rows, nu, Xw, s);
}

tsr_status haar_forward_ld(const float *X, long long ldx, int rows, int nu, float *Xw, cudaStream_t s) {
  const int P = chart_side(nu), P2 = P * P;
  const int NW = 10 * P2 + 2;
  const int S = std::min(P2, HAAR_SEG), nseg = P2 / S;
  const int n_prob = rows * 10 * nseg, npb = hf_problems_per_block(S);
  if (n_prob == 0) return TSR_OK;
  const int n_lb = (n_prob + npb - 1) / npb, grid = std::min(n_lb, HF_GRID);
  if (nseg == 1) {
    haar_forward_kernel<<<grid, HF_THREADS, 0, s>>>(X, nu, P, ldx, NW, S, Xw, nullptr, n_prob, n_lb);
    ::tsr::count_launch();
    TSR_CUDA(cudaGetLastError());
    return TSR_OK;
  }
  Scratch as;
  tsr_status st = as.alloc(sizeof(float) * (size_t)rows * 10 * nseg, s);
  if (st != TSR_OK) return st;
  float *A = static_cast<float *>(as.p);
  haar_forward_kernel<<<grid, HF_THREADS, 0, s>>>(X, nu, P, ldx, NW, S, Xw, A, n_prob, n_lb);
  ::tsr::count_launch();
  haar_forward_top_kernel<<<rows * 10, 256, 0, s>>>(X, A, nu, P, ldx, NW, nseg, Xw); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

size_t haar_inverse_seg_floats(int rows, int nu) {
  const int P = chart_side(nu), P2 = P * P;
  return P2 <= HAAR_SEG ? 0 : (size_t)rows * 10 * (P2 / HAAR_SEG);
}

tsr_status haar_inverse(const float *Xw, int rows, int nu, float *X, cudaStream_t s, float *seg) {
  const int P = chart_side(nu), P2 = P * P;
  const int N = 10 * nu * nu + 2, NW = 10 * P2 + 2;
  if (P2 <= HAAR_SEG) {
    const size_t smem = sizeof(float) * (size_t)P2 * 2;
    haar_inverse_kernel<<<rows * 10, haar_threads(P2), smem, s>>>(Xw, nullptr, nu, P, N, NW, P2, X);
    ::tsr::count_launch();
    TSR_CUDA(cudaGetLastError());
    return TSR_OK;
  }
  const int nseg = P2 / HAAR_SEG;
  Scratch as;
  float *A = seg;   // the run approximations: the caller's buffer, else stream-ordered scratch
  if (!A) {
    tsr_status st = as.alloc(sizeof(float) * haar_inverse_seg_floats(rows, nu), s);
    if (st != TSR_OK) return st;
    A = static_cast<float *>(as.p);
  }
  haar_inverse_top_kernel<<<rows * 10, 256, 0, s>>>(Xw, P, NW, nseg, A); ::tsr::count_launch();
  const size_t smem = sizeof(float) * HAAR_SEG * 2;
  haar_inverse_kernel<<<rows * 10 * nseg, HAAR_SEG_THREADS, smem, s>>>(Xw, A, nu, P, N, NW, HAAR_SEG, X);
  ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

// ---------------------------------------------------------------- top-p selection
// Exclusive scan of one value per thread across a block of SEL_NT threads; `total`
// receives the block sum.  wsum: SEL_NT / 32 shared words.
constexpr int SEL_NT = 512;
__device__ __forceinline__ unsigned block_excl_scan(unsigned x, unsigned *wsum, unsigned &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned v = lane < SEL_NT / 32 ? wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < SEL_NT / 32) wsum[lane] = v;
  }
  __syncthreads();
  const unsigned excl = incl - x + (warp > 0 ? wsum[warp - 1] : 0u);
  total = wsum[SEL_NT / 32 - 1];
  __syncthreads();
  return excl;
}

// Keep flags of one (k, j) row and its column list, in index order: every key above
// tau, and the first `remaining` keys equal to it (all of them when all_eq).  Chunks of
// SEL_NT x 8 consecutive coefficients, 8 per thread; a block scan of the per-thread
// counts places each kept value.  Both poles are kept and end the column list, which
// holds n_keep + 2 entries.
__device__ void keep_pass(const float *__restrict__ c, int n_coef, unsigned tau, unsigned remaining, bool all_eq,
                          int n_keep, uint8_t *__restrict__ kp, int32_t *__restrict__ ci, float *__restrict__ cv,
                          unsigned *wsum) {
  unsigned written = 0, eq_seen = 0;
  for (int base = 0; base < n_coef; base += 8 * SEL_NT) {
    const int w0 = base + 8 * threadIdx.x;
    float v[8];
    unsigned u[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      v[q] = (w0 + q < n_coef) ? c[w0 + q] : 0.f;
      u[q] = __float_as_uint(v[q]) & 0x7FFFFFFFu;
    }
    unsigned er = 0, eq_tot = 0;
    if (!all_eq) {
      unsigned neq = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) neq += (w0 + q < n_coef && u[q] == tau) ? 1u : 0u;
      er = eq_seen + block_excl_scan(neq, wsum, eq_tot);
    }
    unsigned kmask = 0, nk = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      bool k = false;
      if (w0 + q < n_coef) {
        if (u[q] > tau) {
          k = true;
        } else if (u[q] == tau) {
          k = all_eq || er < remaining;
          ++er;
        }
      }
      kmask |= (k ? 1u : 0u) << q;
      nk += k ? 1u : 0u;
    }
    unsigned k_tot;
    unsigned pos = written + block_excl_scan(nk, wsum, k_tot);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (w0 + q < n_coef) kp[w0 + q] = (uint8_t)((kmask >> q) & 1u);
      if (((kmask >> q) & 1u) && pos < (unsigned)n_keep) {
        ci[pos] = w0 + q;
        cv[pos] = v[q];
        ++pos;
      }
    }
    written += k_tot;
    eq_seen += eq_tot;
  }
  if (threadIdx.x == 0) {
    kp[n_coef] = 1;
    kp[n_coef + 1] = 1;
    ci[n_keep] = n_coef;
    cv[n_keep] = c[n_coef];
    ci[n_keep + 1] = n_coef + 1;
    cv[n_keep + 1] = c[n_coef + 1];
  }
}

// One radix digit of `width` bits at `shift` (bins = 2^width <= 4096) over the n keys of
// src (|c| bits: the sign is masked off) whose bits above the digit equal `prefix` under
// `mask`: a histogram (one shared atomic per key: integer counts, the same in any order;
// aggregating the lanes of a digit first with __match_any_sync was 15 % slower per call;
// four independent loads per thread in flight), then the digit where the count of
// larger keys, taken from the top, reaches `remaining`.  Out: the digit, the count of keys
// in larger digits and the count in the digit.  src may be global or shared memory.
__device__ void sel_digit(const unsigned *src, int n, int shift, int width, unsigned prefix, unsigned mask,
                          unsigned remaining, unsigned *hist, unsigned *wsum, unsigned *s_out, unsigned &sel,
                          unsigned &cum, unsigned &eq) {
  const int bins = 1 << width;
  for (int q = threadIdx.x; q < bins; q += SEL_NT) hist[q] = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 4 * SEL_NT) {
    unsigned u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int w = base + q * SEL_NT + threadIdx.x;
      u[q] = (w < n) ? (src[w] & 0x7FFFFFFFu) : 0u;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int w = base + q * SEL_NT + threadIdx.x;
      const bool in = (w < n) && ((u[q] & mask) == prefix);
      const unsigned digit = in ? ((u[q] >> shift) & (unsigned)(bins - 1)) : (unsigned)bins;
      if (in) atomicAdd(&hist[digit], 1u);
    }
  }
  __syncthreads();
  // thread t holds the `per` digits just below bins - per t; a block scan from the top finds
  // the thread, then the digit, where the running count reaches `remaining`
  const int per = bins > SEL_NT ? bins / SEL_NT : 1;
  const int top = bins - per * (int)threadIdx.x;   // the thread's digits: [top - per, top)
  unsigned h[8] = {0, 0, 0, 0, 0, 0, 0, 0}, sum = 0;
  if (top > 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < per) {
        h[q] = hist[top - 1 - q];
        sum += h[q];
      }
  }
  unsigned total;
  const unsigned before = block_excl_scan(sum, wsum, total);
  if (top > 0 && before < remaining && before + sum >= remaining) {
    unsigned c0 = before;
    int q = 0;
    for (; q < per - 1; ++q) {
      if (c0 + h[q] >= remaining) break;
      c0 += h[q];
    }
    s_out[0] = (unsigned)(top - 1 - q);
    s_out[1] = c0;
    s_out[2] = h[q];
  }
  __syncthreads();
  sel = s_out[0];
  cum = s_out[1];
  eq = s_out[2];
  __syncthreads();
}

// One block per (k, j) row: the n_keep-th largest |c| over the chart coefficients, then, in
// index order, the keep flags and the column list (every larger value, and the first
// (n_keep - #larger) values equal to it; both poles kept and ending the list).  The key is
// found digit by digit: the top 12 bits over the row; then, when the keys sharing those bits
// fit the 4,096-word scratch (big), they are gathered there and the last 19 bits are two
// digits over the gathered keys; otherwise three more digits over the row.  The key and the
// number of its equals are the same either way, so the keep set does not depend on the path.
__device__ __forceinline__ void select_block(const float *__restrict__ Mw, int n_coef, int NW, int n_keep,
                                             uint8_t *__restrict__ keep, int32_t *__restrict__ cidx,
                                             float *__restrict__ cval, int rowi, unsigned *big) {
  __shared__ unsigned hist[1024];
  __shared__ unsigned s_out[3], s_n;
  __shared__ unsigned wsum[SEL_NT / 32];
  const float *c = Mw + (size_t)rowi * NW;
  const unsigned *keys = reinterpret_cast<const unsigned *>(c);
  uint8_t *kp = keep + (size_t)rowi * NW;
  unsigned remaining = (unsigned)n_keep, sel, cum, eq;
  sel_digit(keys, n_coef, 19, 12, 0u, 0u, remaining, big, wsum, s_out, sel, cum, eq);
  remaining -= cum;
  unsigned prefix = sel << 19, mask = 0xFFFu << 19, n_eq = eq;
  if (n_eq <= 4096u) {
    // gather the keys of the chosen 12-bit digit (in any order: only counts depend on them)
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < n_coef; base += 4 * SEL_NT) {
      unsigned u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {   // four independent loads per thread in flight
        const int w = base + q * SEL_NT + threadIdx.x;
        u[q] = w < n_coef ? (keys[w] & 0x7FFFFFFFu) : 0u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int w = base + q * SEL_NT + threadIdx.x;
        const bool in = w < n_coef && (u[q] & mask) == prefix;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (bal == 0u) continue;
        unsigned at = 0;
        if (lane == __ffs(bal) - 1) at = atomicAdd(&s_n, (unsigned)__popc(bal));
        at = __shfl_sync(0xffffffffu, at, __ffs(bal) - 1);
        if (in) big[at + __popc(bal & ((1u << lane) - 1u))] = u[q];
      }
    }
    __syncthreads();
    const int ng = (int)s_n;
    sel_digit(big, ng, 9, 10, prefix, mask, remaining, hist, wsum, s_out, sel, cum, eq);
    remaining -= cum;
    prefix |= sel << 9;
    mask |= 0x3FFu << 9;
    sel_digit(big, ng, 0, 9, prefix, mask, remaining, hist, wsum, s_out, sel, cum, eq);
    remaining -= cum;
    prefix |= sel;
    mask |= 0x1FFu;
    n_eq = eq;
  } else {
    const int shifts[3] = {11, 3, 0}, widths[3] = {8, 8, 3};
    for (int d = 0; d < 3; ++d) {
      sel_digit(keys, n_coef, shifts[d], widths[d], prefix, mask, remaining, hist, wsum, s_out, sel, cum, eq);
      remaining -= cum;
      prefix |= sel << shifts[d];
      mask |= ((1u << widths[d]) - 1u) << shifts[d];
      n_eq = eq;
    }
  }
  // prefix = key of the n_keep-th largest; keep `remaining` of its n_eq equal keys (lowest index first)
  keep_pass(c, n_coef, prefix, remaining, remaining >= n_eq, n_keep, kp, cidx + (size_t)rowi * (n_keep + 2),
            cval + (size_t)rowi * (n_keep + 2), wsum);
}

// The same selection for a row of at most SEL_WARP_MAX coefficients by one warp: the four
// radix digits histogrammed in the warp's own 256 bins, the keep flags and the column list
// placed by warp scans.  Same keys, same digits, same tie rule: the same keep set and list.
#ifndef TSR_SEL_WARP_MAX
#define TSR_SEL_WARP_MAX (10 * 256)
#endif
constexpr int SEL_WARP_MAX = TSR_SEL_WARP_MAX;
__device__ __forceinline__ unsigned warp_excl_scan(unsigned x, unsigned &total) {
  const int lane = threadIdx.x & 31;
  unsigned incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - x;
}

__device__ void select_warp(const float *__restrict__ c, int n_coef, int n_keep, uint8_t *__restrict__ kp,
                            int32_t *__restrict__ ci, float *__restrict__ cv, unsigned *hist) {
  const int lane = threadIdx.x & 31;
  unsigned prefix = 0, mask = 0, remaining = (unsigned)n_keep, n_eq = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int q = lane; q < 256; q += 32) hist[q] = 0;
    __syncwarp();
    for (int base = 0; base < n_coef; base += 4 * 32) {
      unsigned u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int w = base + q * 32 + lane;
        u[q] = (w < n_coef) ? (__float_as_uint(c[w]) & 0x7FFFFFFFu) : 0u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int w = base + q * 32 + lane;
        const bool in = (w < n_coef) && ((u[q] & mask) == prefix);
        if (__ballot_sync(0xffffffffu, in) == 0u) continue;
        const unsigned digit = in ? ((u[q] >> shift) & 255u) : 256u;
        if (in) atomicAdd(&hist[digit], 1u);
      }
    }
    __syncwarp();
    // lane l holds digits 255 - 8 l down to 248 - 8 l; the digit where the running count
    // from the top reaches `remaining`
    unsigned h[8], sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      h[q] = hist[255 - 8 * lane - q];
      sum += h[q];
    }
    unsigned incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, incl >= remaining);
    const int ldr = __ffs(hit) - 1;
    unsigned sel = 0, cum = incl - sum, eq = 0;
    {
      int q = 0;
      for (; q < 7; ++q) {
        if (cum + h[q] >= remaining) break;
        cum += h[q];
      }
      sel = (unsigned)(255 - 8 * lane - q);
      eq = h[q];
    }
    sel = __shfl_sync(0xffffffffu, sel, ldr);
    cum = __shfl_sync(0xffffffffu, cum, ldr);
    eq = __shfl_sync(0xffffffffu, eq, ldr);
    remaining -= cum;
    prefix |= sel << shift;
    mask |= 255u << shift;
    n_eq = eq;
    __syncwarp();
  }
  // keep flags and column list in index order: chunks of 256 coefficients, 8 per lane
  const unsigned tau = prefix;
  const bool all_eq = remaining >= n_eq;
  unsigned written = 0, eq_seen = 0;
  for (int base = 0; base < n_coef; base += 8 * 32) {
    const int w0 = base + 8 * lane;
    float v[8];
    unsigned u[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      v[q] = (w0 + q < n_coef) ? c[w0 + q] : 0.f;
      u[q] = __float_as_uint(v[q]) & 0x7FFFFFFFu;
    }
    unsigned er = 0, eq_tot = 0;
    if (!all_eq) {
      unsigned neq = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) neq += (w0 + q < n_coef && u[q] == tau) ? 1u : 0u;
      er = eq_seen + warp_excl_scan(neq, eq_tot);
    }
    unsigned kmask = 0, nk = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      bool k = false;
      if (w0 + q < n_coef) {
        if (u[q] > tau) {
          k = true;
        } else if (u[q] == tau) {
          k = all_eq || er < remaining;
          ++er;
        }
      }
      kmask |= (k ? 1u : 0u) << q;
      nk += k ? 1u : 0u;
    }
    unsigned k_tot;
    unsigned pos = written + warp_excl_scan(nk, k_tot);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (w0 + q < n_coef) kp[w0 + q] = (uint8_t)((kmask >> q) & 1u);
      if (((kmask >> q) & 1u) && pos < (unsigned)n_keep) {
        ci[pos] = w0 + q;
        cv[pos] = v[q];
        ++pos;
      }
    }
    written += k_tot;
    eq_seen += eq_tot;
  }
  if (lane == 0) {
    kp[n_coef] = 1;
    kp[n_coef + 1] = 1;
    ci[n_keep] = n_coef;
    cv[n_keep] = c[n_coef];
    ci[n_keep + 1] = n_coef + 1;
    cv[n_keep + 1] = c[n_coef + 1];
  }
}

// Rows per select block: SEL_NT / 32 rows by warps when the row has at most SEL_WARP_MAX
// coefficients, else one row by the whole block.
__host__ __device__ inline int sel_rows_per_block(int n_coef) { return n_coef <= SEL_WARP_MAX ? SEL_NT / 32 : 1; }

__device__ __forceinline__ void select_rows(const float *__restrict__ Mw, int n_coef, int NW, int n_keep, int rows,
                                            uint8_t *__restrict__ keep, int32_t *__restrict__ cidx,
                                            float *__restrict__ cval, int blk, unsigned (*whist)[256]) {
  if (n_coef <= SEL_WARP_MAX) {
    const int warp = threadIdx.x >> 5, rowi = blk * (SEL_NT / 32) + warp;
    if (rowi < rows)
      select_warp(Mw + (size_t)rowi * NW, n_coef, n_keep, keep + (size_t)rowi * NW, cidx + (size_t)rowi * (n_keep + 2),
                  cval + (size_t)rowi * (n_keep + 2), whist[warp]);
  } else {
    select_block(Mw, n_coef, NW, n_keep, keep, cidx, cval, blk, &whist[0][0]);
  }
}

__global__ void __launch_bounds__(SEL_NT) select_kernel(const float *__restrict__ Mw, int n_coef, int NW, int n_keep,
                                                       int rows, uint8_t *__restrict__ keep,
                                                       int32_t *__restrict__ cidx, float *__restrict__ cval) {
  __shared__ unsigned whist[SEL_NT / 32][256];
  select_rows(Mw, n_coef, NW, n_keep, rows, keep, cidx, cval, blockIdx.x, whist);
}

// Energy rule: per (k, j) row the smallest n >= 1 whose n largest |c| (ties: lower
// index) hold at least a fraction e of the row's energy, the FP64 sum of c^2 over the
// chart coefficients.  The same radix descent as the count rule on per-digit energies:
// each warp histograms a contiguous part of the row (lanes holding the same digit are
// added in lane order by their leader) and the warps' histograms are added in warp
// order, so the choice is deterministic.  Out: n_keep, the key tau of the n_keep-th
// largest, how many of the keys equal to tau are kept and how many there are.
constexpr int EN_NT = 512;
constexpr int EN_W = EN_NT / 32;
__global__ void __launch_bounds__(EN_NT) select_energy_kernel(const float *__restrict__ Mw, int n_coef, int NW,
                                                             double e, int *__restrict__ nk_out,
                                                             unsigned *__restrict__ tau_out,
                                                             unsigned *__restrict__ rem_out,
                                                             unsigned *__restrict__ neq_out) {
  extern __shared__ double en_smem[];
  double *he = en_smem;                                        // [EN_W][256]
  unsigned *hc = reinterpret_cast<unsigned *>(he + EN_W * 256);   // [EN_W][256]
  __shared__ double Es[256];
  __shared__ unsigned Cs[256];
  __shared__ double red[EN_W];
  __shared__ double s_total, s_eabove;
  __shared__ unsigned s_sel, s_cabove;
  const int rowi = blockIdx.x;
  const float *c = Mw + (size_t)rowi * NW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (int w = threadIdx.x; w < n_coef; w += EN_NT) {
    const double x = c[w];
    acc = fma(x, x, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < EN_W; ++q) t += red[q];
    s_total = t;
  }
  __syncthreads();
  const double total = s_total;
  if (total == 0.0) {   // every coefficient is 0: keep the first
    if (threadIdx.x == 0) {
      nk_out[rowi] = 1;
      tau_out[rowi] = 0u;
      rem_out[rowi] = 1u;
      neq_out[rowi] = (unsigned)n_coef;
    }
    return;
  }
  double rem_e = e * total;
  unsigned prefix = 0, mask = 0, cnt_above = 0, n_eq = 0;
  const int chunk = (n_coef + EN_W - 1) / EN_W;
  const int w0 = warp * chunk, w1 = min(n_coef, w0 + chunk);
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int d = lane; d < 256; d += 32) {
      he[warp * 256 + d] = 0.0;
      hc[warp * 256 + d] = 0u;
    }
    __syncwarp();
    for (int base = w0; base < w1; base += 32) {
      const int w = base + lane;
      const float v = (w < w1) ? c[w] : 0.0f;
      const unsigned u = __float_as_uint(v) & 0x7FFFFFFFu;
      const bool in = (w < w1) && ((u & mask) == prefix);
      if (__ballot_sync(0xffffffffu, in) == 0u) continue;
      const unsigned digit = in ? ((u >> shift) & 255u) : 256u;
      const double x = in ? (double)v * (double)v : 0.0;
      const unsigned peers = __match_any_sync(0xffffffffu, digit);
      double sum = 0.0;
      for (int src = 0; src < 32; ++src) {
        const double y = __shfl_sync(0xffffffffu, x, src);
        if ((peers >> src) & 1u) sum += y;
      }
      if (in && lane == __ffs(peers) - 1) {
        he[warp * 256 + digit] += sum;
        hc[warp * 256 + digit] += (unsigned)__popc(peers);
      }
      __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += EN_NT) {
      double E = 0.0;
      unsigned C = 0u;
      for (int q = 0; q < EN_W; ++q) {
        E += he[q * 256 + d];
        C += hc[q * 256 + d];
      }
      Es[d] = E;
      Cs[d] = C;
    }
    __syncthreads();
    if (warp == 0) {
      // lane l holds digits 255 - 8 l down to 248 - 8 l; the first digit (from the top) where
      // the running energy reaches rem_e is selected (if rounding leaves it short, the lowest
      // non-empty digit: everything in the set is kept)
      double he8[8], se = 0.0;
      unsigned hc8[8], sc = 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        he8[q] = Es[255 - 8 * lane - q];
        hc8[q] = Cs[255 - 8 * lane - q];
        se += he8[q];
        sc += hc8[q];
      }
      double ie = se;
      unsigned ic = sc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double ye = __shfl_up_sync(0xffffffffu, ie, o);
        const unsigned yc = __shfl_up_sync(0xffffffffu, ic, o);
        if (lane >= o) {
          ie += ye;
          ic += yc;
        }
      }
      const unsigned hit = __ballot_sync(0xffffffffu, ie >= rem_e);
      const unsigned nonempty = __ballot_sync(0xffffffffu, sc > 0u);
      const int L = hit ? __ffs(hit) - 1 : 31 - __clz(nonempty);
      if (lane == L) {
        double cum = ie - se;
        unsigned ccum = ic - sc;
        int q = 0;
        if (hit) {
          for (; q < 7; ++q) {
            if (cum + he8[q] >= rem_e) break;
            cum += he8[q];
            ccum += hc8[q];
          }
        } else {
          int last = 0;
          for (int t = 0; t < 8; ++t)
            if (hc8[t] > 0u) last = t;
          for (; q < last; ++q) {
            cum += he8[q];
            ccum += hc8[q];
          }
        }
        s_sel = (unsigned)(255 - 8 * lane - q);
        s_eabove = cum;
        s_cabove = ccum;
      }
    }
    __syncthreads();
    rem_e -= s_eabove;
    cnt_above += s_cabove;
    prefix |= s_sel << shift;
    mask |= 255u << shift;
    n_eq = Cs[s_sel];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tv = (double)__uint_as_float(prefix);
    const double t2 = tv * tv;
    double m = (t2 > 0.0) ? ceil(rem_e / t2) : 1.0;
    m = fmin(fmax(m, 1.0), (double)n_eq);
    nk_out[rowi] = (int)(cnt_above + (unsigned)m);
    tau_out[rowi] = prefix;
    rem_out[rowi] = (unsigned)m;
    neq_out[rowi] = n_eq;
  }
}

// Keep flags and column lists of the energy rule: column kj's n_keep + 2 entries at col_ptr[kj].
__global__ void __launch_bounds__(SEL_NT) keep_energy_kernel(const float *__restrict__ Mw, int n_coef, int NW,
                                                            const int *__restrict__ nk, const unsigned *__restrict__ tau,
                                                            const unsigned *__restrict__ rem,
                                                            const unsigned *__restrict__ neq,
                                                            const int64_t *__restrict__ col_ptr,
                                                            uint8_t *__restrict__ keep, int32_t *__restrict__ cidx,
                                                            float *__restrict__ cval) {
  __shared__ unsigned wsum[SEL_NT / 32];
  const int rowi = blockIdx.x;
  keep_pass(Mw + (size_t)rowi * NW, n_coef, tau[rowi], rem[rowi], rem[rowi] >= neq[rowi], nk[rowi],
            keep + (size_t)rowi * NW, cidx + col_ptr[rowi], cval + col_ptr[rowi], wsum);
}

// CSR by wavelet row, in three launches over tiles of 32 rows:
//  count: warp q sums the rows' flags of kj = q, q + 8, ... (32 consecutive bytes per
//         load); the tile's total goes to tsum[tile];
//  scan:  exclusive scan of the tile totals (one block);
//  fill:  warp q owns the kj chunk [q KJ / 8, (q+1) KJ / 8); row offsets come from the
//         tile offset and a scan of the 32 row counts, the warp writes its entries
//         (kj ascending within each row) and row_ptr.
constexpr int ROW_TILE = 32;
__device__ __forceinline__ void count_block(const uint8_t *__restrict__ keep, int KJ, int NW,
                                            int64_t *__restrict__ tsum, int tile) {
  __shared__ int part[8][ROW_TILE];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = tile * ROW_TILE + lane;
  int n = 0;
  if (w < NW)
    for (int kj = warp; kj < KJ; kj += 8) n += keep[(size_t)kj * NW + w];
  part[warp][lane] = n;
  __syncthreads();
  if (warp == 0) {
    int t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) tsum[tile] = t;
  }
}

__global__ void __launch_bounds__(256) count_kernel(const uint8_t *__restrict__ keep, int KJ, int NW,
                                                    int64_t *__restrict__ tsum) {
  count_block(keep, KJ, NW, tsum, blockIdx.x);
}

// exclusive scan of v[0..n) in place; v[n] = total (single block; n = tiles, a few thousand)
__device__ __forceinline__ void scan_block(int64_t *__restrict__ v, int n) {
  __shared__ int64_t warp_sum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b = min(n, (int)threadIdx.x * per), e = min(n, b + per);
  int64_t sum = 0;
  for (int i = b; i < e; ++i) sum += v[i];
  int64_t x = sum;
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
  int64_t run = x - sum + (warp > 0 ? warp_sum[warp - 1] : 0);
  for (int i = b; i < e; ++i) {
    const int64_t c = v[i];
    v[i] = run;
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) v[n] = run;
}

__global__ void __launch_bounds__(1024) scan_kernel(int64_t *__restrict__ v, int n) { scan_block(v, n); }

__device__ __forceinline__ void fill_block(const float *__restrict__ Mw, const uint8_t *__restrict__ keep, int KJ,
                                           int NW, const int64_t *__restrict__ toff, int64_t *__restrict__ row_ptr,
                                           uint16_t *__restrict__ col, float *__restrict__ val, int tile) {
  __shared__ int part[8][ROW_TILE];
  __shared__ int64_t rbase[ROW_TILE];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = tile * ROW_TILE + lane;
  const int kb = warp * KJ / 8, ke = (warp + 1) * KJ / 8;
  int n = 0;
  if (w < NW)
    for (int kj = kb; kj < ke; ++kj) n += keep[(size_t)kj * NW + w];
  part[warp][lane] = n;
  __syncthreads();
  if (warp == 0) {
    int t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][lane];
    int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int64_t rb = toff[tile] + (incl - t);
    rbase[lane] = rb;
    if (w < NW) row_ptr[w] = rb;
    if (w == NW - 1) row_ptr[NW] = rb + t;
  }
  __syncthreads();
  if (w >= NW) return;
  int64_t p = rbase[lane];
  for (int q = 0; q < warp; ++q) p += part[q][lane];
  for (int kj = kb; kj < ke; ++kj) {
    if (keep[(size_t)kj * NW + w]) {
      col[p] = (uint16_t)kj;
      val[p] = Mw[(size_t)kj * NW + w];
      ++p;
    }
  }
}

__global__ void __launch_bounds__(256) fill_kernel(const float *__restrict__ Mw, const uint8_t *__restrict__ keep,
                                                   int KJ, int NW, const int64_t *__restrict__ toff,
                                                   int64_t *__restrict__ row_ptr, uint16_t *__restrict__ col,
                                                   float *__restrict__ val) {
  fill_block(Mw, keep, KJ, NW, toff, row_ptr, col, val, blockIdx.x);
}

static int keep_count(double p, int n_coef) {
  double v = std::floor(p * (double)n_coef + 0.5);
  if (v < 1.0) v = 1.0;
  if (v > (double)n_coef) v = (double)n_coef;
  return (int)v;
}

// CSR by wavelet row from the keep flags [K J][n_rows].
static tsr_status csr_from_keep(const float *Mw, const uint8_t *keep, tsr_compressed *c, cudaStream_t s) {
  const int NW = c->n_rows, KJ = c->K * c->J;
  const int row_tiles = (NW + ROW_TILE - 1) / ROW_TILE;
  Scratch cnt_s;
  tsr_status st = cnt_s.alloc(sizeof(int64_t) * (row_tiles + 1), s);
  if (st != TSR_OK) return st;
  int64_t *cnt = static_cast<int64_t *>(cnt_s.p);
  count_kernel<<<row_tiles, 256, 0, s>>>(keep, KJ, NW, cnt); ::tsr::count_launch();
  scan_kernel<<<1, 1024, 0, s>>>(cnt, row_tiles); ::tsr::count_launch();
  fill_kernel<<<row_tiles, 256, 0, s>>>(Mw, keep, KJ, NW, cnt, c->row_ptr, c->col, c->val); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

// Selection + packing into an existing top-p handle (its K, J, nu and n_keep).
tsr_status wavelet_compress_into(const float *Mw, tsr_compressed *c, cudaStream_t s) {
  if (c->keep_rule != 0) {
    set_error("haar_recompress: the energy rule's sizes depend on the data; compress anew");
    return TSR_ERR_UNSUPPORTED;
  }
  const int NW = c->n_rows, n_coef = NW - 2, KJ = c->K * c->J;
  Scratch keep_s;
  tsr_status st = keep_s.alloc((size_t)KJ * NW, s);
  if (st != TSR_OK) return st;
  uint8_t *keep = static_cast<uint8_t *>(keep_s.p);
  const int rpb = sel_rows_per_block(n_coef);
  select_kernel<<<(KJ + rpb - 1) / rpb, SEL_NT, 0, s>>>(Mw, n_coef, NW, c->n_keep, KJ, keep, c->cidx, c->cval);
  ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return csr_from_keep(Mw, keep, c, s);
}

// A handle with its arrays for the given column lengths (n_keep of each (k, j) + 2 poles).
static tsr_status compressed_alloc(int K, int J, int nu, const std::vector<int> &n_keep_col, tsr_compressed **out) {
  const int P = chart_side(nu);
  const int KJ = K * J;
  tsr_compressed *c = new tsr_compressed();
  cudaGetDevice(&c->device);
  c->K = K;
  c->J = J;
  c->nu = nu;
  c->P = P;
  c->n_rows = 10 * P * P + 2;
  std::vector<int64_t> cp(KJ + 1, 0);
  for (int q = 0; q < KJ; ++q) cp[q + 1] = cp[q] + n_keep_col[q] + 2;
  c->nnz = cp[KJ];
  cudaError_t e = cudaMalloc(&c->row_ptr, sizeof(int64_t) * (c->n_rows + 1));
  // col and val padded to whole groups of 4 entries (the fused relight reads aligned 4-entry groups)
  const size_t nnz4 = ((size_t)c->nnz + 3) & ~(size_t)3;
  if (e == cudaSuccess) e = cudaMalloc(&c->col, sizeof(uint16_t) * nnz4);
  if (e == cudaSuccess) e = cudaMalloc(&c->val, sizeof(float) * nnz4);
  // the padding holds column 0 and value 0, so every entry of a group is a valid term
  if (e == cudaSuccess && nnz4 > (size_t)c->nnz) e = cudaMemset(c->col + c->nnz, 0, sizeof(uint16_t) * (nnz4 - c->nnz));
  if (e == cudaSuccess && nnz4 > (size_t)c->nnz) e = cudaMemset(c->val + c->nnz, 0, sizeof(float) * (nnz4 - c->nnz));
  if (e == cudaSuccess) e = cudaMalloc(&c->cidx, sizeof(int32_t) * c->nnz);
  if (e == cudaSuccess) e = cudaMalloc(&c->cval, sizeof(float) * c->nnz);
  if (e == cudaSuccess) e = cudaMalloc(&c->col_ptr, sizeof(int64_t) * (KJ + 1));
  if (e == cudaSuccess) e = cudaMemcpy(c->col_ptr, cp.data(), sizeof(int64_t) * (KJ + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error("compressed transfer: %s", cudaGetErrorString(e));
    tsr_compressed_destroy(c);
    return e == cudaErrorMemoryAllocation ? TSR_ERR_OOM : TSR_ERR_CUDA;
  }
  *out = c;
  return TSR_OK;
}

tsr_status wavelet_compress(const float *Mw, int K, int J, int nu, double p, tsr_compressed **out, cudaStream_t s) {
  const int P = chart_side(nu);
  const int n_coef = 10 * P * P;
  const int n_keep = keep_count(p, n_coef);
  tsr_compressed *c = nullptr;
  tsr_status st = compressed_alloc(K, J, nu, std::vector<int>(K * J, n_keep), &c);
  if (st != TSR_OK) return st;
  c->n_keep = n_keep;
  c->keep_rule = 0;
  st = wavelet_compress_into(Mw, c, s);
  if (st != TSR_OK) {
    tsr_compressed_destroy(c);
    return st;
  }
  *out = c;
  return TSR_OK;
}

// Energy rule: the column lengths depend on the data, so the call reads them back
// (one stream synchronisation) to size the handle before packing.
tsr_status wavelet_compress_energy(const float *Mw, int K, int J, int nu, double energy, tsr_compressed **out,
                                   cudaStream_t s) {
  const int P = chart_side(nu);
  const int n_coef = 10 * P * P, NW = n_coef + 2, KJ = K * J;
  Scratch meta_s, keep_s;
  tsr_status st = meta_s.alloc(sizeof(int) * 4 * (size_t)KJ, s);
  if (st == TSR_OK) st = keep_s.alloc((size_t)KJ * NW, s);
  if (st != TSR_OK) return st;
  int *nk = static_cast<int *>(meta_s.p);
  unsigned *tau = reinterpret_cast<unsigned *>(nk + KJ), *rem = tau + KJ, *neq = rem + KJ;
  const size_t smem = (sizeof(double) + sizeof(unsigned)) * EN_W * 256;
  TSR_CUDA(cudaFuncSetAttribute(select_energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  select_energy_kernel<<<KJ, EN_NT, smem, s>>>(Mw, n_coef, NW, energy, nk, tau, rem, neq); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  std::vector<int> nk_h(KJ);
  TSR_CUDA(cudaMemcpyAsync(nk_h.data(), nk, sizeof(int) * KJ, cudaMemcpyDeviceToHost, s));
  TSR_CUDA(cudaStreamSynchronize(s));
  tsr_compressed *c = nullptr;
  st = compressed_alloc(K, J, nu, nk_h, &c);
  if (st != TSR_OK) return st;
  c->n_keep = -1;
  c->keep_rule = 1;
  uint8_t *keep = static_cast<uint8_t *>(keep_s.p);
  keep_energy_kernel<<<KJ, SEL_NT, 0, s>>>(Mw, n_coef, NW, nk, tau, rem, neq, c->col_ptr, keep, c->cidx, c->cval);
  ::tsr::count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) st = csr_from_keep(Mw, keep, c, s);
  else {
    set_error("keep_energy_kernel: %s", cudaGetErrorString(e));
    st = TSR_ERR_CUDA;
  }
  if (st != TSR_OK) {
    tsr_compressed_destroy(c);
    return st;
  }
  *out = c;
  return TSR_OK;
}


// ---------------------------------------------------------------- Step 2 of many meshes
// Haar analysis, top-p selection and CSR packing of up to TSR_CB_MAX meshes per launch of
// each stage, from a descriptor table passed by value (no host copies: capturable in a
// CUDA graph).  Mesh b's columns of the concatenated M start at X (row stride ldx); its
// wavelet coefficients, keep flags and tile counts live in stream-ordered scratch.  Every
// block does exactly what the per-mesh kernels do for the same (mesh, row, ...), so the
// handles are bit-identical to compressing each mesh alone.
constexpr int TSR_CB_MAX = 32;
struct CompressMesh {
  const float *X;
  float *Mw, *A;
  uint8_t *keep;
  int64_t *tcnt;
  int64_t *row_ptr;
  uint16_t *col;
  float *val;
  int32_t *cidx;
  float *cval;
  int nu, P, NW, n_keep, seg_len, nseg, row_tiles;
  int b_haar, b_top, b_sel, b_tile;   // first block of the mesh in the Haar, top-level, selection and row-tile launches
};
struct CompressBatch {
  int n, KJ;
  long long ldx;
  CompressMesh m[TSR_CB_MAX];
};

// the mesh whose first block (field B) is the largest one <= blk
#define TSR_CB_FIND(cb, field, blk)                                      \
  ([&]() {                                                              \
    int b_ = 0;                                                         \
    while (b_ + 1 < (cb).n && (cb).m[b_ + 1].field <= (blk)) ++b_;      \
    return b_;                                                          \
  }())

__global__ void __launch_bounds__(HF_THREADS) haar_forward_batched_kernel(const __grid_constant__ CompressBatch cb,
                                                                         int n_lb) {
  __shared__ float part[HF_THREADS / 32];
  for (int lb = blockIdx.x; lb < n_lb; lb += gridDim.x) {
    const int b = TSR_CB_FIND(cb, b_haar, lb);
    const CompressMesh &m = cb.m[b];
    haar_forward_problems(m.X, m.nu, m.P, cb.ldx, m.NW, m.seg_len, m.Mw, m.A,
                          (lb - m.b_haar) * hf_problems_per_block(m.seg_len), cb.KJ * 10 * m.nseg, part);
  }
}

__global__ void haar_forward_top_batched_kernel(const __grid_constant__ CompressBatch cb) {
  const int blk = blockIdx.x;
  const int b = TSR_CB_FIND(cb, b_top, blk);
  const CompressMesh &m = cb.m[b];
  const int local = blk - m.b_top;
  haar_forward_top_block(m.X, m.A, m.nu, m.P, cb.ldx, m.NW, m.nseg, m.Mw, local % 10, local / 10);
}

__global__ void __launch_bounds__(SEL_NT) select_batched_kernel(const __grid_constant__ CompressBatch cb) {
  __shared__ unsigned whist[SEL_NT / 32][256];
  const int b = TSR_CB_FIND(cb, b_sel, (int)blockIdx.x);
  const CompressMesh &m = cb.m[b];
  select_rows(m.Mw, m.NW - 2, m.NW, m.n_keep, cb.KJ, m.keep, m.cidx, m.cval, blockIdx.x - m.b_sel, whist);
}

__global__ void __launch_bounds__(256) count_batched_kernel(const __grid_constant__ CompressBatch cb) {
  const int b = TSR_CB_FIND(cb, b_tile, (int)blockIdx.x);
  const CompressMesh &m = cb.m[b];
  count_block(m.keep, cb.KJ, m.NW, m.tcnt, blockIdx.x - m.b_tile);
}

__global__ void __launch_bounds__(1024) scan_batched_kernel(const __grid_constant__ CompressBatch cb) {
  scan_block(cb.m[blockIdx.x].tcnt, cb.m[blockIdx.x].row_tiles);
}

__global__ void __launch_bounds__(256) fill_batched_kernel(const __grid_constant__ CompressBatch cb) {
  const int b = TSR_CB_FIND(cb, b_tile, (int)blockIdx.x);
  const CompressMesh &m = cb.m[b];
  fill_block(m.Mw, m.keep, cb.KJ, m.NW, m.tcnt, m.row_ptr, m.col, m.val, blockIdx.x - m.b_tile);
}

// Step 2 (Haar, top-p selection, packing) of n meshes into their existing top-p Haar handles
// c[b] (K, J, nu and n_keep fixed); mesh b's columns of M start at M + offsets[b], row stride
// offsets[n].  One launch per stage and group of TSR_CB_MAX meshes.
tsr_status haar_recompress_many(int n, const int64_t *offsets, const float *M, tsr_compressed *const *c,
                                cudaStream_t s) {
  const long long ldx = offsets[n];
  const int KJ = c[0]->K * c[0]->J;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  for (int b0 = 0; b0 < n; b0 += TSR_CB_MAX) {
    const int nb = std::min(TSR_CB_MAX, n - b0);
    CompressBatch cb{};
    cb.n = nb;
    cb.KJ = KJ;
    cb.ldx = ldx;
    size_t bytes = 0;
    int n_haar = 0, n_top = 0, n_sel = 0, n_tile = 0;
    for (int q = 0; q < nb; ++q) {
      const tsr_compressed *h = c[b0 + q];
      CompressMesh &m = cb.m[q];
      m.nu = h->nu;
      m.P = h->P;
      m.NW = h->n_rows;
      m.n_keep = h->n_keep;
      m.seg_len = std::min(m.P * m.P, HAAR_SEG);
      m.nseg = m.P * m.P / m.seg_len;
      m.row_tiles = (m.NW + ROW_TILE - 1) / ROW_TILE;
      m.b_haar = n_haar;
      m.b_top = n_top;
      m.b_sel = n_sel;
      m.b_tile = n_tile;
      n_haar += (KJ * 10 * m.nseg + hf_problems_per_block(m.seg_len) - 1) / hf_problems_per_block(m.seg_len);
      n_top += m.nseg > 1 ? KJ * 10 : 0;
      n_tile += m.row_tiles;
      n_sel += (KJ + sel_rows_per_block(m.NW - 2) - 1) / sel_rows_per_block(m.NW - 2);
      bytes += al(sizeof(float) * (size_t)KJ * m.NW) + al(sizeof(float) * (size_t)KJ * 10 * m.nseg) +
               al((size_t)KJ * m.NW) + al(sizeof(int64_t) * (m.row_tiles + 1));
    }
    Scratch sc;
    tsr_status st = sc.alloc(bytes, s);
    if (st != TSR_OK) return st;
    uint8_t *p = static_cast<uint8_t *>(sc.p);
    for (int q = 0; q < nb; ++q) {
      const tsr_compressed *h = c[b0 + q];
      CompressMesh &m = cb.m[q];
      m.X = M + offsets[b0 + q];
      m.Mw = reinterpret_cast<float *>(p);
      p += al(sizeof(float) * (size_t)KJ * m.NW);
      m.A = reinterpret_cast<float *>(p);
      p += al(sizeof(float) * (size_t)KJ * 10 * m.nseg);
      m.keep = p;
      p += al((size_t)KJ * m.NW);
      m.tcnt = reinterpret_cast<int64_t *>(p);
      p += al(sizeof(int64_t) * (m.row_tiles + 1));
      m.row_ptr = h->row_ptr;
      m.col = h->col;
      m.val = h->val;
      m.cidx = h->cidx;
      m.cval = h->cval;
    }
    haar_forward_batched_kernel<<<std::min(n_haar, HF_GRID), HF_THREADS, 0, s>>>(cb, n_haar);
    ::tsr::count_launch();
    if (n_top > 0) {
      haar_forward_top_batched_kernel<<<n_top, 256, 0, s>>>(cb);
      ::tsr::count_launch();
    }
    select_batched_kernel<<<n_sel, SEL_NT, 0, s>>>(cb); ::tsr::count_launch();
    count_batched_kernel<<<n_tile, 256, 0, s>>>(cb); ::tsr::count_launch();
    scan_batched_kernel<<<nb, 1024, 0, s>>>(cb); ::tsr::count_launch();
    fill_batched_kernel<<<n_tile, 256, 0, s>>>(cb); ::tsr::count_launch();
    TSR_CUDA(cudaGetLastError());
  }
  return TSR_OK;
}

// The top-p Haar handles of n meshes: sized on the host (n_keep is fixed by p and the
// chart size), then filled by haar_recompress_many.
tsr_status haar_compress_many(int n, const int64_t *offsets, const float *M, int K, int J, double p,
                              tsr_compressed **out, cudaStream_t s) {
  for (int b = 0; b < n; ++b) out[b] = nullptr;
  tsr_status st = TSR_OK;
  for (int b = 0; b < n && st == TSR_OK; ++b) {
    const long long nv = offsets[b + 1] - offsets[b];
    int nu = 1;
    while (10LL * nu * nu + 2 < nv) ++nu;
    const int P = chart_side(nu), n_coef = 10 * P * P, n_keep = keep_count(p, n_coef);
    st = compressed_alloc(K, J, nu, std::vector<int>(K * J, n_keep), &out[b]);
    if (st == TSR_OK) {
      out[b]->n_keep = n_keep;
      out[b]->keep_rule = 0;
    }
  }
  if (st == TSR_OK) st = haar_recompress_many(n, offsets, M, out, s);
  if (st != TSR_OK)
    for (int b = 0; b < n; ++b) {
      tsr_compressed_destroy(out[b]);
      out[b] = nullptr;
    }
  return st;
}

}  // namespace tsr

extern "C" void tsr_compressed_destroy(tsr_compressed *c) {
  if (!c) return;
  cudaFree(c->row_ptr);
  cudaFree(c->col);
  cudaFree(c->val);
  cudaFree(c->cidx);
  cudaFree(c->cval);
  cudaFree(c->col_ptr);
  delete c;
}
