// Section 4, rendering Steps 3-5: relight / material edit from the compressed
// wavelet transfer, and its reverse mode.
//
// Forward, per vector v = (edit e, channel c):
//   c_v[kj]  = g[e][c][k] * l[j]                       (Steps 3-4 weights)
//   b^w_v[w] = sum over the kept entries (kj, val) of row w of val * c_v[kj]
//   B_v      = w_1^{-1} b^w_v                           (Step 5, inverse Haar per chart)
// Reverse, for an upstream gradient dL/dB:
//   r^w_v    = w_1 dL/dB_v          (w_1 is orthonormal: the adjoint of w_1^{-1} is w_1)
//   dc_v[kj] = sum_w S[w][kj] r^w_v[w]
//   dg[e][c][k] = sum_j l_j dc_v[kj],   dl[j] = sum_{v,k} g_v[k] dc_v[kj].
#include <algorithm>

#include "handles.cuh"

namespace tsr {

constexpr int RL_VG = 8;   // vectors per block

// b^w[v][w] for a group of RL_VG vectors; one thread per wavelet row.
__global__ void __launch_bounds__(256) relight_spmm_kernel(const int64_t *__restrict__ row_ptr,
                                                          const uint16_t *__restrict__ col,
                                                          const float *__restrict__ val, int n_rows, int K, int J,
                                                          int V, const float *__restrict__ g,
                                                          const float *__restrict__ l, float *__restrict__ bw) {
  extern __shared__ float cw[];   // [KJ][RL_VG]
  const int KJ = K * J;
  const int v0 = blockIdx.y * RL_VG;
  for (int q = threadIdx.x; q < KJ * RL_VG; q += blockDim.x) {
    const int kj = q / RL_VG, vv = q % RL_VG, v = v0 + vv;
    const int k = kj / J, j = kj % J;
    cw[q] = (v < V) ? g[(size_t)v * K + k] * l[j] : 0.0f;
  }
  __syncthreads();
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_rows) return;
  float acc[RL_VG];
#pragma unroll
  for (int vv = 0; vv < RL_VG; ++vv) acc[vv] = 0.0f;
  const int64_t p1 = row_ptr[w + 1];
  for (int64_t p = row_ptr[w]; p < p1; ++p) {
    const float a = val[p];
    const float4 *cr = reinterpret_cast<const float4 *>(cw + (int)col[p] * RL_VG);
    const float4 c0 = cr[0], c1 = cr[1];
    acc[0] = fmaf(a, c0.x, acc[0]);
    acc[1] = fmaf(a, c0.y, acc[1]);
    acc[2] = fmaf(a, c0.z, acc[2]);
    acc[3] = fmaf(a, c0.w, acc[3]);
    acc[4] = fmaf(a, c1.x, acc[4]);
    acc[5] = fmaf(a, c1.y, acc[5]);
    acc[6] = fmaf(a, c1.z, acc[6]);
    acc[7] = fmaf(a, c1.w, acc[7]);
  }
#pragma unroll
  for (int vv = 0; vv < RL_VG; ++vv)
    if (v0 + vv < V) bw[(size_t)(v0 + vv) * n_rows + w] = acc[vv];
}

// dc[v][kj] = sum over the n_keep+2 entries (w, val) of column kj of val * r^w[v][w]:
// one block per (kj, group of RL_VG vectors), no atomics.
__global__ void __launch_bounds__(256) relight_colgather_kernel(const int32_t *__restrict__ cidx,
                                                               const float *__restrict__ cval, int ncol, int n_rows,
                                                               int KJ, int V, const float *__restrict__ rw,
                                                               float *__restrict__ dc) {
  __shared__ float red[RL_VG][8];
  const int kj = blockIdx.x;
  const int v0 = blockIdx.y * RL_VG;
  float acc[RL_VG];
#pragma unroll
  for (int vv = 0; vv < RL_VG; ++vv) acc[vv] = 0.0f;
  const int32_t *ci = cidx + (size_t)kj * ncol;
  const float *cv = cval + (size_t)kj * ncol;
  for (int q = threadIdx.x; q < ncol; q += blockDim.x) {
    const int w = ci[q];
    const float a = cv[q];
#pragma unroll
    for (int vv = 0; vv < RL_VG; ++vv)
      if (v0 + vv < V) acc[vv] = fmaf(a, rw[(size_t)(v0 + vv) * n_rows + w], acc[vv]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int vv = 0; vv < RL_VG; ++vv) {
    float x = acc[vv];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[vv][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < RL_VG && v0 + threadIdx.x < V) {
    float x = 0.0f;
    for (int w8 = 0; w8 < 8; ++w8) x += red[threadIdx.x][w8];
    dc[(size_t)(v0 + threadIdx.x) * KJ + kj] = x;
  }
}

// dg[v][k] = sum_j l_j dc[v][kj];  dl[j] = sum_{v,k} g[v][k] dc[v][kj]  (single block)
__global__ void __launch_bounds__(1024) relight_grad_finish_kernel(const float *__restrict__ dc, int K, int J, int V,
                                                                  const float *__restrict__ g,
                                                                  const float *__restrict__ l, float *__restrict__ dg,
                                                                  float *__restrict__ dl) {
  for (int q = threadIdx.x; q < V * K; q += blockDim.x) {
    const int v = q / K, k = q % K;
    float s = 0.0f;
    for (int j = 0; j < J; ++j) s = fmaf(l[j], dc[((size_t)v * K + k) * J + j], s);
    dg[q] = s;
  }
  // dl: one warp per j, lanes over (v, k)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < J; j += nw) {
    float s = 0.0f;
    for (int q = lane; q < V * K; q += 32) s = fmaf(g[q], dc[(size_t)q * J + j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dl[j] = s;
  }
}

tsr_status relight(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B, cudaStream_t s) {
  const int V = n_edit * 3;
  const int KJ = c->K * c->J;
  Scratch bw_s;
  tsr_status st = bw_s.alloc(sizeof(float) * (size_t)V * c->n_rows, s);
  if (st != TSR_OK) return st;
  float *bw = static_cast<float *>(bw_s.p);
  const dim3 grid((c->n_rows + 255) / 256, (V + RL_VG - 1) / RL_VG);
  const size_t smem = sizeof(float) * KJ * RL_VG;
  relight_spmm_kernel<<<grid, 256, smem, s>>>(c->row_ptr, c->col, c->val, c->n_rows, c->K, c->J, V, g, l, bw); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return haar_inverse(bw, V, c->nu, B, s);
}

// Same two launches as relight(), with the b^w buffer supplied by the caller
// (used by the allocation-free entry point).
tsr_status relight_with_scratch(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B,
                                float *bw, cudaStream_t s) {
  const int V = n_edit * 3;
  const int KJ = c->K * c->J;
  const dim3 grid((c->n_rows + 255) / 256, (V + RL_VG - 1) / RL_VG);
  const size_t smem = sizeof(float) * KJ * RL_VG;
  relight_spmm_kernel<<<grid, 256, smem, s>>>(c->row_ptr, c->col, c->val, c->n_rows, c->K, c->J, V, g, l, bw); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return haar_inverse(bw, V, c->nu, B, s);
}

tsr_status relight_backward(const tsr_compressed *c, int n_edit, const float *g, const float *l, const float *dLdB,
                            float *dg, float *dl, cudaStream_t s) {
  const int V = n_edit * 3;
  const int KJ = c->K * c->J;
  Scratch rw_s, dc_s;
  tsr_status st = rw_s.alloc(sizeof(float) * (size_t)V * c->n_rows, s);
  if (st == TSR_OK) st = dc_s.alloc(sizeof(float) * (size_t)V * KJ, s);
  if (st != TSR_OK) return st;
  float *rw = static_cast<float *>(rw_s.p);
  float *dc = static_cast<float *>(dc_s.p);
  st = haar_forward(dLdB, V, c->nu, rw, s);
  if (st != TSR_OK) return st;
  const dim3 grid(KJ, (V + RL_VG - 1) / RL_VG);
  relight_colgather_kernel<<<grid, 256, 0, s>>>(c->cidx, c->cval, c->n_keep + 2, c->n_rows, KJ, V, rw, dc); ::tsr::count_launch();
  relight_grad_finish_kernel<<<1, 1024, 0, s>>>(dc, c->K, c->J, V, g, l, dg, dl); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

}  // namespace tsr
