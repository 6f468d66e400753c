// The paper's Step-2 spatial wavelet (Section 5: "Daubechies 9/7"): the CDF 9/7
// biorthogonal pair by lifting, whole-sample symmetric extension, low band
// scaled by zeta and high band by 1/zeta (DC gain sqrt 2, as the orthonormal
// Haar), as a separable 2D Mallat pyramid of each chart's P x P image (row-major,
// chart pixel (r, c) = vertex d nu^2 + r nu + c, zero padding), every level
// transforming the rows, then the columns, of the low-low band, down to 1 x 1.
// Coefficients of chart d at [d P^2, (d+1) P^2); the two poles pass through.
//
// Three operators, one block per (row of the input, chart), the image in shared
// memory, each 1D pass as four parallel lifting steps:
//   analysis A       (compression);
//   synthesis S = A^-1 (relight, Step 5);
//   S^T              (the reverse mode: the transpose of every synthesis step,
//                     in the reverse order; S^T != A for a biorthogonal pair).
#include <algorithm>

#include "handles.cuh"

namespace tsr {

constexpr float C97_ALPHA = -1.586134342059924f;
constexpr float C97_BETA = -0.052980118572961f;
constexpr float C97_GAMMA = 0.882911075530934f;
constexpr float C97_DELTA = 0.443506852043971f;
constexpr float C97_ZETA = 1.149604398860241f;

// Element q of line l of the n x n band of a P-stride image, along rows (ROWS) or columns.
template <bool ROWS>
__device__ __forceinline__ float &el(float *img, int P, int l, int q) {
  return ROWS ? img[l * P + q] : img[q * P + l];
}

// Analysis of every line of the n x n band of `a` (interleaved) into `b` as [low | high].
template <bool ROWS>
__device__ void c97_analysis_pass(float *a, float *b, int P, int n) {
  const int m = n >> 1, total = n * m;
  // d_i += alpha (s_i + s_{i+1}), s_m = s_{m-1}
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    const float sn = el<ROWS>(a, P, l, (i + 1 < m) ? 2 * i + 2 : 2 * i);
    el<ROWS>(a, P, l, 2 * i + 1) += C97_ALPHA * (el<ROWS>(a, P, l, 2 * i) + sn);
  }
  __syncthreads();
  // s_i += beta (d_{i-1} + d_i), d_{-1} = d_0
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    const float dp = el<ROWS>(a, P, l, i > 0 ? 2 * i - 1 : 1);
    el<ROWS>(a, P, l, 2 * i) += C97_BETA * (dp + el<ROWS>(a, P, l, 2 * i + 1));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    const float sn = el<ROWS>(a, P, l, (i + 1 < m) ? 2 * i + 2 : 2 * i);
    el<ROWS>(a, P, l, 2 * i + 1) += C97_GAMMA * (el<ROWS>(a, P, l, 2 * i) + sn);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    const float dp = el<ROWS>(a, P, l, i > 0 ? 2 * i - 1 : 1);
    el<ROWS>(a, P, l, 2 * i) += C97_DELTA * (dp + el<ROWS>(a, P, l, 2 * i + 1));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    el<ROWS>(b, P, l, i) = C97_ZETA * el<ROWS>(a, P, l, 2 * i);
    el<ROWS>(b, P, l, m + i) = el<ROWS>(a, P, l, 2 * i + 1) / C97_ZETA;
  }
  __syncthreads();
}

// Synthesis of every line of the band of `a` ([low | high]) into `b` (interleaved).
template <bool ROWS>
__device__ void c97_synthesis_pass(float *a, float *b, int P, int n) {
  const int m = n >> 1, total = n * m;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    el<ROWS>(b, P, l, 2 * i) = el<ROWS>(a, P, l, i) / C97_ZETA;
    el<ROWS>(b, P, l, 2 * i + 1) = el<ROWS>(a, P, l, m + i) * C97_ZETA;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < total; t += blockDim.x) {   // s_i -= delta (d_{i-1} + d_i)
    const int l = t / m, i = t % m;
    const float dp = el<ROWS>(b, P, l, i > 0 ? 2 * i - 1 : 1);
    el<ROWS>(b, P, l, 2 * i) -= C97_DELTA * (dp + el<ROWS>(b, P, l, 2 * i + 1));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < total; t += blockDim.x) {   // d_i -= gamma (s_i + s_{i+1})
    const int l = t / m, i = t % m;
    const float sn = el<ROWS>(b, P, l, (i + 1 < m) ? 2 * i + 2 : 2 * i);
    el<ROWS>(b, P, l, 2 * i + 1) -= C97_GAMMA * (el<ROWS>(b, P, l, 2 * i) + sn);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    const float dp = el<ROWS>(b, P, l, i > 0 ? 2 * i - 1 : 1);
    el<ROWS>(b, P, l, 2 * i) -= C97_BETA * (dp + el<ROWS>(b, P, l, 2 * i + 1));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    const float sn = el<ROWS>(b, P, l, (i + 1 < m) ? 2 * i + 2 : 2 * i);
    el<ROWS>(b, P, l, 2 * i + 1) -= C97_ALPHA * (el<ROWS>(b, P, l, 2 * i) + sn);
  }
  __syncthreads();
}

// Transpose of the synthesis of every line of the band of `a` (interleaved) into `b`
// ([low | high]).  The synthesis applies unscale, U_delta, U_gamma, U_beta, U_alpha,
// interleave; its transpose applies deinterleave, U_alpha^T, U_beta^T, U_gamma^T,
// U_delta^T, unscale, where for d -= c E s (E: s_{i} + s_{i+1}, s_m = s_{m-1}) the
// transpose is s_j -= c (d_j [doubled at j = m-1] + d_{j-1}), and for s -= c F d
// (F: d_{i-1} + d_i, d_{-1} = d_0) it is d_j -= c (s_j [doubled at j = 0] + s_{j+1}).
template <bool ROWS>
__device__ void c97_synthesis_transpose_pass(float *a, float *b, int P, int n) {
  const int m = n >> 1, total = n * m;
  float *s = b, *d = b;   // s_i at line position i, d_i at m + i of b
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    el<ROWS>(b, P, l, i) = el<ROWS>(a, P, l, 2 * i);
    el<ROWS>(b, P, l, m + i) = el<ROWS>(a, P, l, 2 * i + 1);
  }
  __syncthreads();
  const float cE[2] = {C97_ALPHA, C97_GAMMA}, cF[2] = {C97_BETA, C97_DELTA};
  for (int r = 0; r < 2; ++r) {
    for (int t = threadIdx.x; t < total; t += blockDim.x) {   // s_j -= c (w_j d_j + d_{j-1})
      const int l = t / m, j = t % m;
      const float dj = el<ROWS>(d, P, l, m + j) * (j == m - 1 ? 2.0f : 1.0f);
      const float dm = (j > 0) ? el<ROWS>(d, P, l, m + j - 1) : 0.0f;
      el<ROWS>(s, P, l, j) -= cE[r] * (dj + dm);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < total; t += blockDim.x) {   // d_j -= c (w_j s_j + s_{j+1})
      const int l = t / m, j = t % m;
      const float sj = el<ROWS>(s, P, l, j) * (j == 0 ? 2.0f : 1.0f);
      const float sp = (j + 1 < m) ? el<ROWS>(s, P, l, j + 1) : 0.0f;
      el<ROWS>(d, P, l, m + j) -= cF[r] * (sj + sp);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / m, i = t % m;
    el<ROWS>(b, P, l, i) /= C97_ZETA;
    el<ROWS>(b, P, l, m + i) *= C97_ZETA;
  }
  __syncthreads();
}

enum { C97_ANALYSIS = 0, C97_SYNTHESIS = 1, C97_SYNTHESIS_T = 2 };

// Block (row, chart d).  ANALYSIS / SYNTHESIS_T: vertex data [rows][N] -> coefficients
// [rows][NW]; SYNTHESIS: coefficients -> vertex data.
template <int OP>
__global__ void __launch_bounds__(1024) cdf97_kernel(const float *__restrict__ in, int nu, int P, int N, int NW,
                                                    float *__restrict__ out) {
  extern __shared__ float sh[];
  float *A = sh, *B = sh + P * P;
  const int row = blockIdx.x / 10, d = blockIdx.x % 10;
  const int P2 = P * P;
  if (OP == C97_SYNTHESIS) {
    const float *cw = in + (size_t)row * NW + (size_t)d * P2;
    for (int q = threadIdx.x; q < P2; q += blockDim.x) A[q] = cw[q];
  } else {
    const float *x = in + (size_t)row * N + (size_t)d * nu * nu;
    for (int q = threadIdx.x; q < P2; q += blockDim.x) {
      const int r = q / P, c = q % P;
      A[q] = (r < nu && c < nu) ? x[r * nu + c] : 0.0f;
    }
  }
  __syncthreads();
  if (OP == C97_ANALYSIS) {
    for (int n = P; n >= 2; n >>= 1) {
      c97_analysis_pass<true>(A, B, P, n);    // rows: A -> B
      c97_analysis_pass<false>(B, A, P, n);   // columns: B -> A
    }
  } else if (OP == C97_SYNTHESIS) {
    for (int n = 2; n <= P; n <<= 1) {
      c97_synthesis_pass<false>(A, B, P, n);   // columns: A -> B
      c97_synthesis_pass<true>(B, A, P, n);    // rows: B -> A (leaves the band interleaved in A)
    }
  } else {
    for (int n = P; n >= 2; n >>= 1) {
      c97_synthesis_transpose_pass<true>(A, B, P, n);    // rows: A -> B
      c97_synthesis_transpose_pass<false>(B, A, P, n);   // columns: B -> A
    }
  }
  if (OP == C97_SYNTHESIS) {
    float *x = out + (size_t)row * N + (size_t)d * nu * nu;
    for (int q = threadIdx.x; q < nu * nu; q += blockDim.x) x[q] = A[(q / nu) * P + q % nu];
    if (threadIdx.x == 0 && d == 0) {
      out[(size_t)row * N + 10 * (size_t)nu * nu] = in[(size_t)row * NW + 10 * (size_t)P2];
      out[(size_t)row * N + 10 * (size_t)nu * nu + 1] = in[(size_t)row * NW + 10 * (size_t)P2 + 1];
    }
  } else {
    float *cw = out + (size_t)row * NW + (size_t)d * P2;
    for (int q = threadIdx.x; q < P2; q += blockDim.x) cw[q] = A[q];
    if (threadIdx.x == 0 && d == 0) {
      out[(size_t)row * NW + 10 * (size_t)P2] = in[(size_t)row * N + 10 * (size_t)nu * nu];
      out[(size_t)row * NW + 10 * (size_t)P2 + 1] = in[(size_t)row * N + 10 * (size_t)nu * nu + 1];
    }
  }
}

template <int OP>
static tsr_status cdf97_launch(const float *in, int rows, int nu, float *out, cudaStream_t s) {
  const int P = chart_side(nu);
  const int N = 10 * nu * nu + 2, NW = 10 * P * P + 2;
  const size_t smem = sizeof(float) * 2 * (size_t)P * P;
  TSR_CUDA(cudaFuncSetAttribute(cdf97_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int threads = std::min(1024, std::max(64, P * P / 2));
  cdf97_kernel<OP><<<rows * 10, threads, smem, s>>>(in, nu, P, N, NW, out); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

tsr_status cdf97_forward(const float *X, int rows, int nu, float *Xw, cudaStream_t s) {
  return cdf97_launch<C97_ANALYSIS>(X, rows, nu, Xw, s);
}
tsr_status cdf97_inverse(const float *Xw, int rows, int nu, float *X, cudaStream_t s) {
  return cdf97_launch<C97_SYNTHESIS>(Xw, rows, nu, X, s);
}
tsr_status cdf97_inverse_transpose(const float *X, int rows, int nu, float *Xw, cudaStream_t s) {
  return cdf97_launch<C97_SYNTHESIS_T>(X, rows, nu, Xw, s);
}

tsr_status spatial_forward(int wavelet, const float *X, int rows, int nu, float *Xw, cudaStream_t s) {
  return wavelet == 1 ? cdf97_forward(X, rows, nu, Xw, s) : haar_forward(X, rows, nu, Xw, s);
}
tsr_status spatial_inverse(int wavelet, const float *Xw, int rows, int nu, float *X, cudaStream_t s, float *seg) {
  return wavelet == 1 ? cdf97_inverse(Xw, rows, nu, X, s) : haar_inverse(Xw, rows, nu, X, s, seg);
}
tsr_status spatial_inverse_transpose(int wavelet, const float *X, int rows, int nu, float *Xw, cudaStream_t s) {
  return wavelet == 1 ? cdf97_inverse_transpose(X, rows, nu, Xw, s) : haar_forward(X, rows, nu, Xw, s);
}

}  // namespace tsr
