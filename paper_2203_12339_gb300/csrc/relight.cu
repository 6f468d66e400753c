// Section 4, rendering Steps 3-5: relight / material edit from the compressed
// wavelet transfer, and its reverse mode.
//
// Steps 3-5 give, per vector v = (edit e, channel c) of a call,
//   c_v[kj] = g[e][c][k] * l[j],   b^w_v = S c_v,   B_v = w_1^{-1} b^w_v.
// All vectors of a call share the light l, so c_v factorises and the same B is
// reached by contracting the light first (the Haar transform is linear):
//   Y[k][w] = sum_j S[w][kj] l[j]          one pass over the kept entries
//   Z[k]    = w_1^{-1} Y[k]                K inverse Haar transforms
//   B_v     = sum_k g_v[k] Z[k]            a K-term combination per output value
// The compressed transfer is read once per call whatever the number of edits,
// and the per-edit work is K multiply-adds per vertex.  Calls with at most
// RL_DV vectors (one or two edits) take Steps 4-5 as written instead, which
// moves less data for so few outputs.
//
// Reverse, for an upstream gradient dL/dB (with w_1^{-T} the transpose of the
// synthesis: the analysis w_1 itself for the orthonormal Haar, the transposed
// lifting steps for CDF 9/7):
//   dg_v[k] = <dL/dB_v, Z[k]>
//   Q[k]    = sum_v g_v[k] dL/dB_v,   R[k] = w_1^{-T} Q[k]
//   dl[j]   = sum_k sum_w S[w][kj] R[k][w]
#include <algorithm>

#include "handles.cuh"

namespace tsr {

constexpr int RL_KMAX = 16;   // bases (the library's K limit)

// Y[k][w] for every wavelet row w, a warp per row: lane q takes entry q (then
// q + 32, ...) of the row, which is sorted by kj, so the entries of basis k form a
// run; a segmented scan over the lanes sums each run and the run's last lane adds
// it to Y[k][w] (Y is zeroed first).
__global__ void __launch_bounds__(256) relight_y_kernel(const int64_t *__restrict__ row_ptr,
                                                       const uint16_t *__restrict__ col,
                                                       const float *__restrict__ val, int n_rows, int J,
                                                       const float *__restrict__ l, float *__restrict__ Y) {
  __shared__ float ls[32];
  if (threadIdx.x < J) ls[threadIdx.x] = l[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= n_rows) return;
  const int64_t p0 = row_ptr[w], pe = row_ptr[w + 1];
  for (int64_t base = p0; base < pe; base += 32) {
    const int64_t p = base + lane;
    const bool in = p < pe;
    const int kj = in ? (int)col[p] : 0;
    const int k = in ? kj / J : -1 - lane;   // inactive lanes: keys of their own
    float x = in ? val[p] * ls[kj - (kj / J) * J] : 0.0f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float y = __shfl_up_sync(0xffffffffu, x, o);
      const int ky = __shfl_up_sync(0xffffffffu, k, o);
      if (lane >= o && ky == k) x += y;
    }
    const int k_next = __shfl_down_sync(0xffffffffu, k, 1);
    if (in && (lane == 31 || k_next != k)) Y[(size_t)k * n_rows + w] += x;
  }
}

// Few vectors (V = 3 n_edit <= RL_DV: one or two RGB edits): Steps 4-5 as written, since the
// factorised form would move K (10 P^2 + 2 + N) intermediates for 3 outputs.
// b^w[v][w] = sum over row w's entries of val * g[v][k] l[j]: RL_LPR lanes per row
// (rows average n_keep K J / (10 P^2) entries, ~20 at 5 % of K J = 400), four rows
// per warp, a full complement of blocks looping over rows (many rows in flight per
// SM; the c table in shared memory is built once per block); the V partial sums
// are reduced over the row's lanes.
constexpr int RL_DV = 6;
constexpr int RL_LPR = 8;
template <int VV>
__global__ void __launch_bounds__(256) relight_direct_kernel(const int64_t *__restrict__ row_ptr,
                                                            const uint16_t *__restrict__ col,
                                                            const float *__restrict__ val, int n_rows, int K, int J,
                                                            const float *__restrict__ g, const float *__restrict__ l,
                                                            float *__restrict__ bw) {
  extern __shared__ float cs[];   // [K J][VV]
  const int KJ = K * J;
  for (int q = threadIdx.x; q < KJ * VV; q += blockDim.x) {
    const int kj = q / VV, v = q % VV;
    cs[q] = g[(size_t)v * K + kj / J] * l[kj % J];
  }
  __syncthreads();
  const int sub = threadIdx.x % RL_LPR;
  const int groups = gridDim.x * (blockDim.x / RL_LPR);
  // the loop runs the same number of times in every lane of a warp (the xor-shuffles
  // below name all 32 lanes); groups past the last row sum nothing
  const int w_first = blockIdx.x * (blockDim.x / RL_LPR) + (threadIdx.x & ~31) / RL_LPR;
  for (int wb = w_first; wb < n_rows; wb += groups) {
    const int w = wb + (threadIdx.x & 31) / RL_LPR;
    float acc[VV];
#pragma unroll
    for (int v = 0; v < VV; ++v) acc[v] = 0.0f;
    const bool row_ok = w < n_rows;
    const int64_t pe = row_ok ? row_ptr[w + 1] : 0;
    for (int64_t p = row_ok ? row_ptr[w] + sub : 0; p < pe; p += RL_LPR) {
      const float a = val[p];
      const float *c = cs + (int)col[p] * VV;
#pragma unroll
      for (int v = 0; v < VV; ++v) acc[v] = fmaf(a, c[v], acc[v]);
    }
#pragma unroll
    for (int v = 0; v < VV; ++v)
#pragma unroll
      for (int o = RL_LPR / 2; o > 0; o >>= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
    if (sub == 0 && row_ok)
#pragma unroll
      for (int v = 0; v < VV; ++v) bw[(size_t)v * n_rows + w] = acc[v];
  }
}

template <int VV>
static void launch_direct(const tsr_compressed *c, const float *g, const float *l, float *bw, cudaStream_t s) {
  const size_t smem = sizeof(float) * (size_t)c->K * c->J * VV;
  const int blocks = std::min((c->n_rows + 255 / RL_LPR) / (256 / RL_LPR), 8 * num_sms());
  relight_direct_kernel<VV><<<blocks, 256, smem, s>>>(c->row_ptr, c->col, c->val, c->n_rows, c->K, c->J, g, l, bw);
  ::tsr::count_launch();
}

// B[v][o] = sum_k g[v][k] Z[k][o]: a thread per two output vertices (o, o + 256) and a
// chunk of RL_VB vectors; g staged as float4 rows of KT = K rounded up to 4 (zero padded: no
// per-basis test in the loop, the padding adds fmaf(0, 0, b) = b).
constexpr int RL_VB = 32;
template <int KT>
__global__ void __launch_bounds__(256) relight_combine_kernel(const float *__restrict__ Z, int N, int K, int V,
                                                             const float *__restrict__ g, float *__restrict__ B) {
  __shared__ float4 gs[RL_VB * KT / 4];
  float *gsf = reinterpret_cast<float *>(gs);
  const int v0 = blockIdx.y * RL_VB;
  for (int q = threadIdx.x; q < RL_VB * KT; q += blockDim.x) {
    const int vv = q / KT, k = q % KT;
    gsf[q] = (v0 + vv < V && k < K) ? g[(size_t)(v0 + vv) * K + k] : 0.0f;
  }
  __syncthreads();
  // two vertices per thread (o and o + 256): each g row read from shared memory serves both
  const int o = blockIdx.x * 512 + threadIdx.x;
  if (o >= N) return;
  const bool two = o + 256 < N;
  float z[2][KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    z[0][k] = (k < K) ? Z[(size_t)k * N + o] : 0.0f;
    z[1][k] = (k < K && two) ? Z[(size_t)k * N + o + 256] : 0.0f;
  }
  const int vn = min(RL_VB, V - v0);
  for (int vv = 0; vv < vn; ++vv) {
    float b0 = 0.0f, b1 = 0.0f;
#pragma unroll
    for (int h = 0; h < KT / 4; ++h) {
      const float4 gq = gs[vv * (KT / 4) + h];
      b0 = fmaf(gq.x, z[0][4 * h], b0);
      b1 = fmaf(gq.x, z[1][4 * h], b1);
      b0 = fmaf(gq.y, z[0][4 * h + 1], b0);
      b1 = fmaf(gq.y, z[1][4 * h + 1], b1);
      b0 = fmaf(gq.z, z[0][4 * h + 2], b0);
      b1 = fmaf(gq.z, z[1][4 * h + 2], b1);
      b0 = fmaf(gq.w, z[0][4 * h + 3], b0);
      b1 = fmaf(gq.w, z[1][4 * h + 3], b1);
    }
    B[(size_t)(v0 + vv) * N + o] = b0;
    if (two) B[(size_t)(v0 + vv) * N + o + 256] = b1;
  }
}

static void launch_combine(const float *Z, int N, int K, int V, const float *g, float *B, cudaStream_t s) {
  const dim3 grid((N + 511) / 512, (V + RL_VB - 1) / RL_VB);
  if (K <= 4)
    relight_combine_kernel<4><<<grid, 256, 0, s>>>(Z, N, K, V, g, B);
  else if (K <= 8)
    relight_combine_kernel<8><<<grid, 256, 0, s>>>(Z, N, K, V, g, B);
  else if (K <= 12)
    relight_combine_kernel<12><<<grid, 256, 0, s>>>(Z, N, K, V, g, B);
  else
    relight_combine_kernel<16><<<grid, 256, 0, s>>>(Z, N, K, V, g, B);
  ::tsr::count_launch();
}

// dg partials: block (vector group of RL_GV, o-split s) forms sum over its o-range of
// dL/dB[v][o] Z[k][o] for its vectors; part[s][v][k].
constexpr int RL_GV = 4;
constexpr int RL_OSPLIT = 8;
__global__ void __launch_bounds__(256) relight_dg_kernel(const float *__restrict__ dLdB, const float *__restrict__ Z,
                                                        int N, int K, int V, float *__restrict__ part) {
  __shared__ float red[RL_GV * RL_KMAX][8];
  const int v0 = blockIdx.x * RL_GV;
  const int s = blockIdx.y;
  const int ob = (int)((long long)N * s / RL_OSPLIT), oe = (int)((long long)N * (s + 1) / RL_OSPLIT);
  float acc[RL_GV][RL_KMAX];
#pragma unroll
  for (int a = 0; a < RL_GV; ++a)
#pragma unroll
    for (int k = 0; k < RL_KMAX; ++k) acc[a][k] = 0.0f;
  for (int o = ob + threadIdx.x; o < oe; o += blockDim.x) {
    float z[RL_KMAX];
#pragma unroll
    for (int k = 0; k < RL_KMAX; ++k) z[k] = (k < K) ? Z[(size_t)k * N + o] : 0.0f;
#pragma unroll
    for (int a = 0; a < RL_GV; ++a) {
      const float d = (v0 + a < V) ? dLdB[(size_t)(v0 + a) * N + o] : 0.0f;
#pragma unroll
      for (int k = 0; k < RL_KMAX; ++k) acc[a][k] = fmaf(d, z[k], acc[a][k]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < RL_GV; ++a)
#pragma unroll
    for (int k = 0; k < RL_KMAX; ++k) {
      float x = acc[a][k];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[a * RL_KMAX + k][warp] = x;
    }
  __syncthreads();
  if (threadIdx.x < RL_GV * RL_KMAX) {
    const int a = threadIdx.x / RL_KMAX, k = threadIdx.x % RL_KMAX;
    if (v0 + a < V && k < K) {
      float x = 0.0f;
      for (int q = 0; q < 8; ++q) x += red[threadIdx.x][q];
      part[((size_t)s * V + v0 + a) * K + k] = x;
    }
  }
}

// Q[k][o] = sum_v g[v][k] dL/dB[v][o], in RL_QS vector chunks (blockIdx.y) for
// parallelism: a thread per vertex writes its chunk's partial Qp[chunk][k][o]; the
// chunks are added in order by relight_qsum_kernel.
constexpr int RL_QS = 4;
__global__ void __launch_bounds__(256) relight_q_kernel(const float *__restrict__ dLdB, int N, int K, int V,
                                                       const float *__restrict__ g, float *__restrict__ Qp) {
  __shared__ float gs[64 * RL_KMAX];
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int vb = (int)((long long)V * blockIdx.y / RL_QS), ve = (int)((long long)V * (blockIdx.y + 1) / RL_QS);
  float q[RL_KMAX];
#pragma unroll
  for (int k = 0; k < RL_KMAX; ++k) q[k] = 0.0f;
  for (int v0 = vb; v0 < ve; v0 += 64) {
    const int vn = min(64, ve - v0);
    __syncthreads();
    for (int t = threadIdx.x; t < 64 * K; t += blockDim.x) {
      const int vv = t / K, k = t % K;
      gs[vv * RL_KMAX + k] = (vv < vn) ? g[(size_t)(v0 + vv) * K + k] : 0.0f;
    }
    __syncthreads();
    if (o < N) {
      int vv = 0;
      for (; vv + 4 <= vn; vv += 4) {   // four independent loads in flight
        float d[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) d[a] = dLdB[(size_t)(v0 + vv + a) * N + o];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int k = 0; k < RL_KMAX; ++k) q[k] = fmaf(gs[(vv + a) * RL_KMAX + k], d[a], q[k]);
      }
      for (; vv < vn; ++vv) {
        const float d = dLdB[(size_t)(v0 + vv) * N + o];
#pragma unroll
        for (int k = 0; k < RL_KMAX; ++k) q[k] = fmaf(gs[vv * RL_KMAX + k], d, q[k]);
      }
    }
  }
  if (o < N)
    for (int k = 0; k < K; ++k) Qp[((size_t)blockIdx.y * K + k) * N + o] = q[k];
}

__global__ void relight_qsum_kernel(const float *__restrict__ Qp, size_t n, float *__restrict__ Q) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float x = Qp[i];
#pragma unroll
    for (int c = 1; c < RL_QS; ++c) x += Qp[(size_t)c * n + i];
    Q[i] = x;
  }
}

// colsum[kj] = sum over the entries (w, val) of column kj of val * R[k][w]: a block per kj.
__global__ void __launch_bounds__(256) relight_colsum_kernel(const int32_t *__restrict__ cidx,
                                                            const float *__restrict__ cval,
                                                            const int64_t *__restrict__ col_ptr, int n_rows, int J,
                                                            const float *__restrict__ R, float *__restrict__ colsum) {
  __shared__ float red[8];
  const int kj = blockIdx.x, k = kj / J;
  const int32_t *ci = cidx + col_ptr[kj];
  const float *cv = cval + col_ptr[kj];
  const int ncol = (int)(col_ptr[kj + 1] - col_ptr[kj]);
  const float *Rk = R + (size_t)k * n_rows;
  float acc = 0.0f;
  for (int q = threadIdx.x; q < ncol; q += blockDim.x) acc = fmaf(cv[q], Rk[ci[q]], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float x = 0.0f;
    for (int w8 = 0; w8 < 8; ++w8) x += red[w8];
    colsum[kj] = x;
  }
}

// dg[v][k] = sum_s part[s][v][k];  dl[j] = sum_k colsum[k J + j]   (one block)
__global__ void __launch_bounds__(1024) relight_grad_finish_kernel(const float *__restrict__ part, int V, int K,
                                                                  int J, const float *__restrict__ colsum,
                                                                  float *__restrict__ dg, float *__restrict__ dl) {
  for (int q = threadIdx.x; q < V * K; q += blockDim.x) {
    float x = 0.0f;
    for (int s = 0; s < RL_OSPLIT; ++s) x += part[(size_t)s * V * K + q];
    dg[q] = x;
  }
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    float x = 0.0f;
    for (int k = 0; k < K; ++k) x += colsum[k * J + j];
    dl[j] = x;
  }
}

// Y[k] = (S (I_K x l))[k] (K x n_rows) and its inverse Haar Z[k] (K x N).  seg: the
// inverse Haar's run approximations (NULL: stream-ordered scratch).
static tsr_status relight_basis_images(const tsr_compressed *c, const float *l, float *Y, float *Z, cudaStream_t s,
                                       float *seg = nullptr) {
  TSR_CUDA(cudaMemsetAsync(Y, 0, sizeof(float) * (size_t)c->K * c->n_rows, s));
  relight_y_kernel<<<(c->n_rows + 7) / 8, 256, 0, s>>>(c->row_ptr, c->col, c->val, c->n_rows, c->J, l, Y);
  ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return spatial_inverse(c->wavelet, Y, c->K, c->nu, Z, s, seg);
}

// Layout of the caller's scratch: [intermediates | run approximations of the inverse Haar]
static size_t relight_main_floats(const tsr_compressed *c) {
  const size_t N = 10 * (size_t)c->nu * c->nu + 2;
  return std::max((size_t)c->K * ((size_t)c->n_rows + N), (size_t)RL_DV * c->n_rows);
}

size_t relight_scratch_floats(const tsr_compressed *c) {
  const size_t seg = c->wavelet == 1 ? 0 : haar_inverse_seg_floats(std::max(c->K, RL_DV), c->nu);
  return relight_main_floats(c) + seg;
}

tsr_status relight_with_scratch(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B,
                                float *scratch, cudaStream_t s) {
  const int V = n_edit * 3;
  if (V == 0) return TSR_OK;
  const int N = 10 * c->nu * c->nu + 2;
  if (relight_fusable(c, n_edit)) return relight_fused(1, &c, n_edit, &g, l, &B, s);
  float *seg = scratch + relight_main_floats(c);   // never handed to the allocating path
  if (V <= RL_DV) {
    if (V == 3)
      launch_direct<3>(c, g, l, scratch, s);
    else
      launch_direct<6>(c, g, l, scratch, s);   // V = 3 n_edit <= RL_DV: 3 or 6
    TSR_CUDA(cudaGetLastError());
    return spatial_inverse(c->wavelet, scratch, V, c->nu, B, s, seg);
  }
  float *Y = scratch, *Z = scratch + (size_t)c->K * c->n_rows;
  tsr_status st = relight_basis_images(c, l, Y, Z, s, seg);
  if (st != TSR_OK) return st;
  launch_combine(Z, N, c->K, V, g, B, s);
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

tsr_status relight(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B, cudaStream_t s) {
  Scratch sc;
  tsr_status st = sc.alloc(sizeof(float) * relight_scratch_floats(c), s);
  if (st != TSR_OK) return st;
  return relight_with_scratch(c, n_edit, g, l, B, static_cast<float *>(sc.p), s);
}

tsr_status relight_backward(const tsr_compressed *c, int n_edit, const float *g, const float *l, const float *dLdB,
                            float *dg, float *dl, cudaStream_t s) {
  const int V = n_edit * 3;
  const int K = c->K, J = c->J, KJ = K * J;
  const int N = 10 * c->nu * c->nu + 2;
  const size_t nY = (size_t)K * c->n_rows, nZ = (size_t)K * N;
  Scratch sc;
  tsr_status st = sc.alloc(sizeof(float) * (2 * nY + (2 + RL_QS) * nZ + (size_t)RL_OSPLIT * V * K + KJ), s);
  if (st != TSR_OK) return st;
  float *Y = static_cast<float *>(sc.p), *Z = Y + nY, *Q = Z + nZ, *R = Q + nZ, *part = R + nY;
  float *colsum = part + (size_t)RL_OSPLIT * V * K, *Qp = colsum + KJ;
  st = relight_basis_images(c, l, Y, Z, s);
  if (st != TSR_OK) return st;
  relight_dg_kernel<<<dim3((V + RL_GV - 1) / RL_GV, RL_OSPLIT), 256, 0, s>>>(dLdB, Z, N, K, V, part);
  ::tsr::count_launch();
  relight_q_kernel<<<dim3((N + 255) / 256, RL_QS), 256, 0, s>>>(dLdB, N, K, V, g, Qp); ::tsr::count_launch();
  relight_qsum_kernel<<<4 * num_sms(), 256, 0, s>>>(Qp, nZ, Q); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  st = spatial_inverse_transpose(c->wavelet, Q, K, c->nu, R, s);
  if (st != TSR_OK) return st;
  relight_colsum_kernel<<<KJ, 256, 0, s>>>(c->cidx, c->cval, c->col_ptr, c->n_rows, J, R, colsum);
  ::tsr::count_launch();
  relight_grad_finish_kernel<<<1, 1024, 0, s>>>(part, V, K, J, colsum, dg, dl); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

}  // namespace tsr
