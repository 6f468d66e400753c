// Section 2.2: PCA of sampled R_d (Eq. 5) by one-sided Jacobi SVD in FP64,
// the lookup tables of the radial basis, and the material projection
// g_k = sum_m f_k(r_m) R_d(r_m) with its Jacobian and vector-Jacobian product.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dipole.cuh"
#include "handles.cuh"

namespace tsr {

// ------------------------------------------------------------------ reductions
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *red /* [NV][32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[q * 32 + warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[threadIdx.x * 32 + w];
    red[threadIdx.x * 32] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = red[q * 32];
  __syncthreads();
}

// ------------------------------------------------------------------ Jacobi SVD
// Columns of A (n_cols x n_r, column c contiguous) are the sampled R_d curves of
// the materials: A = R^T.  One-sided Jacobi orthogonalises the columns, after
// which column c = s_c v_c with v_c a right singular vector of R.
__global__ void jacobi_build_kernel(const double *__restrict__ sa, const double *__restrict__ ss, double eta,
                                    int n_mat, int n_cols, int n_r, double dr, double *__restrict__ A) {
  const int c = blockIdx.x;
  double *col = A + (size_t)c * n_r;
  if (c >= n_mat) {
    for (int m = threadIdx.x; m < n_r; m += blockDim.x) col[m] = 0.0;
    return;
  }
  const DipoleMaterial mat = dipole_material(sa[c], ss[c], eta);
  for (int m = threadIdx.x; m < n_r; m += blockDim.x) col[m] = dipole_rd(dr * m, mat);
}

// One round of the circle-method ordering: n_cols/2 disjoint pairs, one per block.
__global__ void jacobi_round_kernel(double *__restrict__ A, int n_cols, int n_r, int round, double tol,
                                    unsigned *__restrict__ rotations) {
  __shared__ double red[3 * 32];
  const int idx = blockIdx.x;
  const int nm1 = n_cols - 1;
  int p, q;
  if (idx == 0) {
    p = nm1;
    q = round;
  } else {
    p = (round + idx) % nm1;
    q = (round - idx + nm1) % nm1;
  }
  double *ap = A + (size_t)p * n_r;
  double *aq = A + (size_t)q * n_r;
  double v[3] = {0.0, 0.0, 0.0};
  for (int m = threadIdx.x; m < n_r; m += blockDim.x) {
    const double x = ap[m], y = aq[m];
    v[0] += x * x;
    v[1] += y * y;
    v[2] += x * y;
  }
  block_sum<3>(v, red);
  const double alpha = v[0], beta = v[1], gamma = v[2];
  if (gamma == 0.0 || alpha == 0.0 || beta == 0.0) return;
  if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) return;
  const double zeta = (beta - alpha) / (2.0 * gamma);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t);
  const double s = c * t;
  for (int m = threadIdx.x; m < n_r; m += blockDim.x) {
    const double x = ap[m], y = aq[m];
    ap[m] = c * x - s * y;
    aq[m] = s * x + c * y;
  }
  if (threadIdx.x == 0) atomicAdd(rotations, 1u);
}

// The whole solve in one cooperative launch: block b owns pair b of every round of the
// circle ordering, rounds are separated by a grid barrier, and after each sweep every
// block reads that sweep's rotation count (rot[sweep], all blocks see the same value) and
// stops when it is zero.  The barrier's waits are bounded: a block that gives up records
// it in *status and the host reports a timeout.  status[1] receives the sweeps run.
__device__ __forceinline__ bool jacobi_grid_barrier(unsigned *bar, unsigned target, unsigned *status) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 0;
    for (uint32_t it = 0; it < TSR_WAIT_LIMIT; ++it) {
      if (*reinterpret_cast<volatile unsigned *>(bar) >= target) {
        ok = 1;
        break;
      }
    }
    if (!ok) atomicOr(status, 1u);
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(256) jacobi_solve_kernel(double *__restrict__ A, int n_cols, int n_r, double tol,
                                                          int max_sweeps, unsigned *__restrict__ rot,
                                                          unsigned *__restrict__ bar, unsigned *__restrict__ status) {
  __shared__ double red[3 * 32];
  const int idx = blockIdx.x, nb = gridDim.x;
  const int nm1 = n_cols - 1;
  unsigned n_bar = 0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < nm1; ++round) {
      int p, q;
      if (idx == 0) {
        p = nm1;
        q = round;
      } else {
        p = (round + idx) % nm1;
        q = (round - idx + nm1) % nm1;
      }
      double *ap = A + (size_t)p * n_r;
      double *aq = A + (size_t)q * n_r;
      double v[3] = {0.0, 0.0, 0.0};
      for (int m = threadIdx.x; m < n_r; m += blockDim.x) {
        const double x = __ldcg(ap + m), y = __ldcg(aq + m);   // through L2: other blocks rewrote the columns
        v[0] += x * x;
        v[1] += y * y;
        v[2] += x * y;
      }
      block_sum<3>(v, red);
      const double alpha = v[0], beta = v[1], gamma = v[2];
      const bool rotate = !(gamma == 0.0 || alpha == 0.0 || beta == 0.0) &&
                          !(fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta));
      if (rotate) {
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = c * t;
        for (int m = threadIdx.x; m < n_r; m += blockDim.x) {
          const double x = __ldcg(ap + m), y = __ldcg(aq + m);
          ap[m] = c * x - s * y;
          aq[m] = s * x + c * y;
        }
        if (threadIdx.x == 0) atomicAdd(&rot[sweep], 1u);
      }
      if (!jacobi_grid_barrier(bar, (++n_bar) * (unsigned)nb, status)) return;
    }
    if (*reinterpret_cast<volatile unsigned *>(&rot[sweep]) == 0u) {
      if (idx == 0 && threadIdx.x == 0) status[2] = 1u;   // converged
      ++sweep;
      break;
    }
  }
  if (idx == 0 && threadIdx.x == 0) status[1] = (unsigned)sweep;
}

// Column norms (= singular values), ranks by descending norm (ties: lower column).
__global__ void jacobi_rank_kernel(const double *__restrict__ A, int n_cols, int n_r, int n_sv,
                                   double *__restrict__ norms, int *__restrict__ col_of_rank,
                                   double *__restrict__ sing_vals) {
  extern __shared__ double nrm[];
  for (int c = threadIdx.x; c < n_cols; c += blockDim.x) {
    const double *col = A + (size_t)c * n_r;
    double s = 0.0;
    for (int m = 0; m < n_r; ++m) s += col[m] * col[m];
    nrm[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n_cols; c += blockDim.x) {
    const double x = nrm[c];
    int rank = 0;
    for (int d = 0; d < n_cols; ++d) {
      const double y = nrm[d];
      rank += (y > x) || (y == x && d < c);
    }
    norms[c] = x;
    col_of_rank[rank] = c;
    if (sing_vals && rank < n_sv) sing_vals[rank] = x;
  }
}

// f_k = column(rank k) / norm, flipped so its largest-|.| entry (lowest m on ties) is positive.
__global__ void jacobi_emit_kernel(const double *__restrict__ A, const double *__restrict__ norms,
                                   const int *__restrict__ col_of_rank, int n_r, double *__restrict__ f) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  const int k = blockIdx.x;
  const int c = col_of_rank[k];
  const double *col = A + (size_t)c * n_r;
  double best = -1.0;
  int besti = 0x7fffffff;
  for (int m = threadIdx.x; m < n_r; m += blockDim.x) {
    const double a = fabs(col[m]);
    if (a > best || (a == best && m < besti)) {
      best = a;
      besti = m;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
    if (ob > best || (ob == best && oi < besti)) {
      best = ob;
      besti = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    bv[warp] = best;
    bi[warp] = besti;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > bv[0] || (bv[w] == bv[0] && bi[w] < bi[0])) {
        bv[0] = bv[w];
        bi[0] = bi[w];
      }
  }
  __syncthreads();
  const double sign = col[bi[0]] < 0.0 ? -1.0 : 1.0;
  const double inv = sign / norms[c];
  for (int m = threadIdx.x; m < n_r; m += blockDim.x) f[(size_t)k * n_r + m] = col[m] * inv;
}

// ------------------------------------------------------------------ tables
__global__ void build_tables_kernel(const double *__restrict__ f, int K, int KP, int n_r,
                                    float2 *__restrict__ tab32, uint32_t *__restrict__ tab16) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (n_r + 1) * KP) return;
  const int m = idx / KP, k = idx % KP;
  double v = 0.0, s = 0.0;
  if (k < K && m < n_r) {
    v = f[(size_t)k * n_r + m];
    if (m + 1 < n_r) s = f[(size_t)k * n_r + m + 1] - v;
  }
  tab32[idx] = make_float2((float)v, (float)s);
  const __nv_bfloat16 bv = __double2bfloat16(v), bs = __double2bfloat16(s);
  tab16[idx] = (uint32_t)__bfloat16_as_ushort(bv) | ((uint32_t)__bfloat16_as_ushort(bs) << 16);
}

// Far-field series of the BF16 transfer.  On [r_near, r_max] the weighted basis
// g_k(r) = r^2 f_k(r) (R_d falls off like 1/r^2 away from the source, so g_k has
// little dynamic range) is projected on Chebyshev polynomials in the variable
// x = 2 (ln r - ln r_near)/(ln r_max - ln r_near) - 1, at the nodes
// x_n = cos(theta_n), theta_n = pi (n + 1/2)/N:
//   c_p = (2 - [p = 0]) / N * sum_n g_k(r(x_n)) cos(p theta_n).
// Then f_k(r) ~= sum_p c_p T_p(x) / r^2.  The transfer kernel generates
// W_p = sigma_p T_p(x) / r^2 with sigma_p = (-1)^(p(p-1)/2), for which the
// Chebyshev recurrence needs only additions: W_{p+1} = (-1)^p 2x W_p + W_{p-1};
// the stored coefficients carry the sign, cheb[k][p] = sigma_p c_p.
// One block per basis function, FP64.
__global__ void __launch_bounds__(256) cheb_fit_kernel(const double *__restrict__ f, int n_r, double r_max,
                                                       double r_near, float *__restrict__ cheb) {
  __shared__ double red[TSR_CHEB_P * 32];
  const int k = blockIdx.x;
  const double lo = log(r_near), hi = log(r_max), dr = r_max / (n_r - 1);
  double acc[TSR_CHEB_P];
#pragma unroll
  for (int p = 0; p < TSR_CHEB_P; ++p) acc[p] = 0.0;
  for (int n = threadIdx.x; n < TSR_CHEB_NODES; n += blockDim.x) {
    const double th = 3.14159265358979323846 * (n + 0.5) / TSR_CHEB_NODES;
    const double x = cos(th);
    const double r = exp(lo + 0.5 * (x + 1.0) * (hi - lo));
    const double xm = r / dr;
    int m = (int)floor(xm);
    if (m > n_r - 2) m = n_r - 2;
    if (m < 0) m = 0;
    const double t = xm - m;
    const double gv = r * r * (f[(size_t)k * n_r + m] * (1.0 - t) + f[(size_t)k * n_r + m + 1] * t);
#pragma unroll
    for (int p = 0; p < TSR_CHEB_P; ++p) acc[p] += gv * cos(p * th);
  }
  block_sum<TSR_CHEB_P>(acc, red);
  if (threadIdx.x < TSR_CHEB_P) {
    const int p = threadIdx.x;
    const double sigma = ((p * (p - 1) / 2) & 1) ? -1.0 : 1.0;
    cheb[k * TSR_CHEB_P + p] = (float)(sigma * (p == 0 ? 1.0 : 2.0) / TSR_CHEB_NODES * acc[p]);
  }
}

// Quality of the truncated series (TSR_CHEB_BF16 terms) per basis: max over a
// log-spaced grid of [r_near, r_max] of |sum_p c_p T_p(x) - g_k(r)| / max |g_k|.
// err[k] is written; the BF16 transfer uses the series only when every err[k]
// is small (the PCA bases of R_d are smooth there; an arbitrary basis may not be).
__global__ void __launch_bounds__(256) cheb_check_kernel(const double *__restrict__ f, int n_r, double r_max,
                                                         double r_near, const float *__restrict__ cheb,
                                                         double *__restrict__ err) {
  __shared__ double red[2 * 32];
  const int k = blockIdx.x;
  const double lo = log(r_near), hi = log(r_max), dr = r_max / (n_r - 1);
  constexpr int NPT = 4096;
  double e = 0.0, gmax = 0.0;
  for (int n = threadIdx.x; n < NPT; n += blockDim.x) {
    const double x = -1.0 + 2.0 * n / (NPT - 1);
    const double r = exp(lo + 0.5 * (x + 1.0) * (hi - lo));
    const double xm = r / dr;
    int m = (int)floor(xm);
    if (m > n_r - 2) m = n_r - 2;
    if (m < 0) m = 0;
    const double t = xm - m;
    const double gv = r * r * (f[(size_t)k * n_r + m] * (1.0 - t) + f[(size_t)k * n_r + m + 1] * t);
    double t0 = 1.0, t1 = x, approx = 0.0;
    for (int p = 0; p < TSR_CHEB_BF16; ++p) {
      const double sigma = ((p * (p - 1) / 2) & 1) ? -1.0 : 1.0;
      approx += sigma * (double)cheb[k * TSR_CHEB_P + p] * t0;
      const double t2 = 2.0 * x * t1 - t0;
      t0 = t1;
      t1 = t2;
    }
    e = fmax(e, fabs(approx - gv));
    gmax = fmax(gmax, fabs(gv));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
    gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  }
  if (lane == 0) {
    red[warp] = e;
    red[32 + warp] = gmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double em = 0.0, gm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      em = fmax(em, red[w]);
      gm = fmax(gm, red[32 + w]);
    }
    err[k] = gm > 0.0 ? em / gm : 0.0;
  }
}

tsr_status basis_build_tables(tsr_basis *b, cudaStream_t s) {
  const int n = (b->n_r + 1) * b->KP;
  build_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(b->f64, b->K, b->KP, b->n_r, b->tab32, b->tab16); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  // far-field series on [r_near, r_max], r_near = r_max / 16 (2.5 mm at r_max = 40 mm)
  b->r_near = 0.0625 * b->r_max;
  const double lo = std::log(b->r_near), hi = std::log(b->r_max);
  b->x_alpha = (float)(std::log(2.0) / (hi - lo));
  b->x_beta = (float)(-1.0 - 2.0 * lo / (hi - lo));
  if (!b->cheb) TSR_CUDA(cudaMalloc(&b->cheb, sizeof(float) * b->K * TSR_CHEB_P + sizeof(double) * 16));
  cheb_fit_kernel<<<b->K, 256, 0, s>>>(b->f64, b->n_r, b->r_max, b->r_near, b->cheb); ::tsr::count_launch();
  double *d_err = reinterpret_cast<double *>(b->cheb + (((size_t)b->K * TSR_CHEB_P + 1) & ~(size_t)1));
  cheb_check_kernel<<<b->K, 256, 0, s>>>(b->f64, b->n_r, b->r_max, b->r_near, b->cheb, d_err); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  double h_err[16] = {0.0};
  TSR_CUDA(cudaMemcpyAsync(h_err, d_err, sizeof(double) * b->K, cudaMemcpyDeviceToHost, s));
  TSR_CUDA(cudaStreamSynchronize(s));   // basis creation is a one-time, synchronous step
  double worst = 0.0;
  for (int k = 0; k < b->K; ++k) worst = std::max(worst, h_err[k]);
  b->cheb_err = worst;
  b->cheb_ok = worst <= TSR_CHEB_MAX_ERR;
  return TSR_OK;
}

// ------------------------------------------------------------------ projection
// One block per (edit, channel): g_k = sum_m f_k(r_m) R_d(r_m); with GRAD also
// the Jacobian dg_k/d(sigma_a, sigma_s', eta).
template <bool GRAD>
__global__ void __launch_bounds__(256) project_kernel(const double *__restrict__ f, int K, int n_r, double dr,
                                                      const double *__restrict__ sa, const double *__restrict__ ss,
                                                      const double *__restrict__ eta, double *__restrict__ g,
                                                      float *__restrict__ g32, double *__restrict__ dg,
                                                      double *__restrict__ part) {
  // block (edit e, channel c) x (sample range blockIdx.y of gridDim.y): with one range
  // the block writes g (and dg); with several it writes part[range][e c][NV] for
  // project_finish_kernel to add in range order.
  constexpr int NV = GRAD ? 64 : 16;
  __shared__ double red[NV * 32];
  const int e = blockIdx.x / 3;
  const int ch = blockIdx.x % 3;
  const int m0 = (int)((long long)n_r * blockIdx.y / gridDim.y), m1 = (int)((long long)n_r * (blockIdx.y + 1) / gridDim.y);
  const DipoleMaterial mat = dipole_material(sa[e * 3 + ch], ss[e * 3 + ch], eta[e]);
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  for (int m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
    const double r = dr * m;
    double R, dRa = 0.0, dRs = 0.0, dRe = 0.0;
    if (GRAD)
      dipole_rd_grad(r, mat, R, dRa, dRs, dRe);
    else
      R = dipole_rd(r, mat);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < K) {
        const double fk = f[(size_t)k * n_r + m];
        acc[k] += fk * R;
        if (GRAD) {
          acc[16 + 3 * k + 0] += fk * dRa;
          acc[16 + 3 * k + 1] += fk * dRs;
          acc[16 + 3 * k + 2] += fk * dRe;
        }
      }
    }
  }
  block_sum<NV>(acc, red);
  if (threadIdx.x != 0) return;
  if (gridDim.y > 1) {
    double *pp = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * NV;
    for (int q = 0; q < NV; ++q) pp[q] = acc[q];
    return;
  }
  const size_t base = (size_t)(e * 3 + ch) * K;
  for (int k = 0; k < K; ++k) {
    g[base + k] = acc[k];
    if (g32) g32[base + k] = (float)acc[k];
    if (GRAD) {
      dg[(base + k) * 3 + 0] = acc[16 + 3 * k + 0];
      dg[(base + k) * 3 + 1] = acc[16 + 3 * k + 1];
      dg[(base + k) * 3 + 2] = acc[16 + 3 * k + 2];
    }
  }
}

template <bool GRAD>
__global__ void project_finish_kernel(const double *__restrict__ part, int n3, int n_split, int K,
                                      double *__restrict__ g, float *__restrict__ g32, double *__restrict__ dg) {
  constexpr int NV = GRAD ? 64 : 16;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // (e c, k)
  if (idx >= n3 * K) return;
  const int ec = idx / K, k = idx % K;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int sp = 0; sp < n_split; ++sp) {
    const double *pp = part + ((size_t)sp * n3 + ec) * NV;
    v[0] += pp[k];
    if (GRAD)
      for (int a = 0; a < 3; ++a) v[1 + a] += pp[16 + 3 * k + a];
  }
  g[idx] = v[0];
  if (g32) g32[idx] = (float)v[0];
  if (GRAD)
    for (int a = 0; a < 3; ++a) dg[(size_t)idx * 3 + a] = v[1 + a];
}

// One block per (edit, channel): dL/dtheta = sum_k dL/dg_k dg_k/dtheta.  The
// eta part of each channel goes to de_part[e][c]; project_eta_finish_kernel adds
// the three channels of an edit in order.
__global__ void __launch_bounds__(256) project_backward_kernel(
    const double *__restrict__ f, int K, int n_r, double dr, const double *__restrict__ sa,
    const double *__restrict__ ss, const double *__restrict__ eta, const float *__restrict__ dLdg,
    float *__restrict__ dsa, float *__restrict__ dss, double *__restrict__ de_part) {
  __shared__ double red[3 * 32];
  const int e = blockIdx.x / 3, ch = blockIdx.x % 3;
  const DipoleMaterial mat = dipole_material(sa[e * 3 + ch], ss[e * 3 + ch], eta[e]);
  const float *w = dLdg + (size_t)(e * 3 + ch) * K;
  double v[3] = {0.0, 0.0, 0.0};
  for (int m = threadIdx.x; m < n_r; m += blockDim.x) {
    double wm = 0.0;
    for (int k = 0; k < K; ++k) wm += (double)w[k] * f[(size_t)k * n_r + m];
    double R, dRa, dRs, dRe;
    dipole_rd_grad(dr * m, mat, R, dRa, dRs, dRe);
    v[0] += wm * dRa;
    v[1] += wm * dRs;
    v[2] += wm * dRe;
  }
  block_sum<3>(v, red);
  if (threadIdx.x == 0) {
    dsa[e * 3 + ch] = (float)v[0];
    dss[e * 3 + ch] = (float)v[1];
    de_part[e * 3 + ch] = v[2];
  }
}

__global__ void project_eta_finish_kernel(const double *__restrict__ de_part, int n, float *__restrict__ deta) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) deta[e] = (float)((de_part[e * 3] + de_part[e * 3 + 1]) + de_part[e * 3 + 2]);
}

}  // namespace tsr

using namespace tsr;

extern "C" tsr_status tsr_fit_pca_basis(int n_mat, const double *sigma_a, const double *sigma_s, double eta,
                                        int n_r, double r_max, int K, double *sing_vals, tsr_basis **out,
                                        tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(out && sigma_a && sigma_s, "tsr_fit_pca_basis: NULL argument");
  TSR_CHECK_ARG(n_mat >= 2 && n_mat <= 1024, "tsr_fit_pca_basis: n_mat=%d outside [2, 1024]", n_mat);
  TSR_CHECK_ARG(n_r >= 16 && n_r <= 4096, "tsr_fit_pca_basis: n_r=%d outside [16, 4096]", n_r);
  TSR_CHECK_ARG(K >= 1 && K <= 16 && K <= std::min(n_mat, n_r), "tsr_fit_pca_basis: K=%d invalid", K);
  TSR_CHECK_ARG(r_max > 0.0, "tsr_fit_pca_basis: r_max must be > 0");
  TSR_CHECK_ARG(eta >= 1.0 && eta <= 2.0, "tsr_fit_pca_basis: eta=%g outside [1, 2]", eta);
  *out = nullptr;
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n_cols = n_mat + (n_mat & 1);
  const double dr = r_max / (n_r - 1);

  tsr_basis *b = new tsr_basis();
  cudaGetDevice(&b->device);
  b->K = K;
  b->n_r = n_r;
  b->KP = (K + 3) & ~3;
  b->r_max = r_max;
  double *A = nullptr, *norms = nullptr;
  int *col_of_rank = nullptr;
  unsigned *rot = nullptr;
  auto fail = [&](tsr_status code) {
    cudaStreamSynchronize(s);
    cudaFree(A);
    cudaFree(norms);
    cudaFree(col_of_rank);
    cudaFree(rot);
    tsr_basis_destroy(b);
    return code;
  };
#define FIT_CUDA(call)                                                                           \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      set_error("tsr_fit_pca_basis: %s: %s", #call, cudaGetErrorString(e_));                     \
      return fail(e_ == cudaErrorMemoryAllocation ? TSR_ERR_OOM : TSR_ERR_CUDA);                 \
    }                                                                                            \
  } while (0)
  FIT_CUDA(cudaMalloc(&b->f64, sizeof(double) * K * n_r));
  FIT_CUDA(cudaMalloc(&b->tab32, sizeof(float2) * (n_r + 1) * b->KP));
  FIT_CUDA(cudaMalloc(&b->tab16, sizeof(uint32_t) * (n_r + 1) * b->KP));
  FIT_CUDA(cudaMalloc(&A, sizeof(double) * (size_t)n_cols * n_r));
  FIT_CUDA(cudaMalloc(&norms, sizeof(double) * n_cols));
  FIT_CUDA(cudaMalloc(&col_of_rank, sizeof(int) * n_cols));
  constexpr int kMaxSweeps = 60;
  FIT_CUDA(cudaMalloc(&rot, sizeof(unsigned) * (kMaxSweeps + 4)));   // per-sweep counts | barrier | status[3]

  jacobi_build_kernel<<<n_cols, 256, 0, s>>>(sigma_a, sigma_s, eta, n_mat, n_cols, n_r, dr, A); ::tsr::count_launch();
  FIT_CUDA(cudaGetLastError());
  const double tol = 1e-14;
  bool converged = false;
  // the whole solve in one cooperative launch (all n_cols / 2 blocks resident: the grid
  // barrier between rounds needs it); one launch per round where that is not possible
  FIT_CUDA(cudaMemsetAsync(rot, 0, sizeof(unsigned) * (kMaxSweeps + 4), s));
  {
    unsigned *bar = rot + kMaxSweeps, *status = rot + kMaxSweeps + 1;
    int nc = n_cols, nr = n_r, ms = kMaxSweeps;
    double tl = tol;
    void *kargs[] = {&A, &nc, &nr, &tl, &ms, &rot, &bar, &status};
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device);
    cudaError_t le = coop ? cudaLaunchCooperativeKernel((const void *)jacobi_solve_kernel, dim3(n_cols / 2), dim3(256),
                                                        kargs, 0, s)
                          : cudaErrorNotSupported;
    if (le == cudaSuccess) {
      ::tsr::count_launch();
      unsigned h[3] = {0u, 0u, 0u};
      FIT_CUDA(cudaMemcpyAsync(h, status, sizeof(unsigned) * 3, cudaMemcpyDeviceToHost, s));
      FIT_CUDA(cudaStreamSynchronize(s));
      if (h[0] & 1u) {
        set_error("tsr_fit_pca_basis: a grid barrier of the Jacobi solve gave up its bounded wait");
        return fail(TSR_ERR_TIMEOUT);
      }
      converged = h[2] != 0u;
    } else {
      (void)cudaGetLastError();   // clear the refused cooperative launch
      for (int sweep = 0; sweep < kMaxSweeps && !converged; ++sweep) {
        for (int r = 0; r < n_cols - 1; ++r) {
          jacobi_round_kernel<<<n_cols / 2, 256, 0, s>>>(A, n_cols, n_r, r, tol, rot + sweep);
          ::tsr::count_launch();
        }
        FIT_CUDA(cudaGetLastError());
        unsigned h = 0;
        FIT_CUDA(cudaMemcpyAsync(&h, rot + sweep, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        FIT_CUDA(cudaStreamSynchronize(s));
        converged = (h == 0);
      }
    }
  }
  if (!converged) {
    set_error("tsr_fit_pca_basis: Jacobi SVD did not converge in %d sweeps", kMaxSweeps);
    return fail(TSR_ERR_CUDA);
  }
  const int n_sv = std::min(n_mat, n_r);
  jacobi_rank_kernel<<<1, 1024, sizeof(double) * n_cols, s>>>(A, n_cols, n_r, n_sv, norms, col_of_rank,
                                                                sing_vals); ::tsr::count_launch();
  jacobi_emit_kernel<<<K, 256, 0, s>>>(A, norms, col_of_rank, n_r, b->f64); ::tsr::count_launch();
  FIT_CUDA(cudaGetLastError());
  st = basis_build_tables(b, s);
  if (st != TSR_OK) return fail(st);
  FIT_CUDA(cudaStreamSynchronize(s));
  cudaFree(A);
  cudaFree(norms);
  cudaFree(col_of_rank);
  cudaFree(rot);
#undef FIT_CUDA
  *out = b;
  return TSR_OK;
}

extern "C" tsr_status tsr_basis_create(int K, int n_r, double r_max, const double *f_host, tsr_basis **out) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(out && f_host, "tsr_basis_create: NULL argument");
  TSR_CHECK_ARG(K >= 1 && K <= 16, "tsr_basis_create: K=%d outside [1, 16]", K);
  TSR_CHECK_ARG(n_r >= 16 && n_r <= 4096, "tsr_basis_create: n_r=%d outside [16, 4096]", n_r);
  TSR_CHECK_ARG(r_max > 0.0, "tsr_basis_create: r_max must be > 0");
  *out = nullptr;
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  tsr_basis *b = new tsr_basis();
  cudaGetDevice(&b->device);
  b->K = K;
  b->n_r = n_r;
  b->KP = (K + 3) & ~3;
  b->r_max = r_max;
  cudaError_t e = cudaMalloc(&b->f64, sizeof(double) * K * n_r);
  if (e == cudaSuccess) e = cudaMalloc(&b->tab32, sizeof(float2) * (n_r + 1) * b->KP);
  if (e == cudaSuccess) e = cudaMalloc(&b->tab16, sizeof(uint32_t) * (n_r + 1) * b->KP);
  if (e == cudaSuccess) e = cudaMemcpy(b->f64, f_host, sizeof(double) * K * n_r, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error("tsr_basis_create: %s", cudaGetErrorString(e));
    tsr_basis_destroy(b);
    return e == cudaErrorMemoryAllocation ? TSR_ERR_OOM : TSR_ERR_CUDA;
  }
  st = basis_build_tables(b, nullptr);
  if (st == TSR_OK && cudaDeviceSynchronize() != cudaSuccess) {
    set_error("tsr_basis_create: table build failed");
    st = TSR_ERR_CUDA;
  }
  if (st != TSR_OK) {
    tsr_basis_destroy(b);
    return st;
  }
  *out = b;
  return TSR_OK;
}

extern "C" tsr_status tsr_basis_table(const tsr_basis *basis, double *f, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(basis && f, "tsr_basis_table: NULL argument");
  TSR_CUDA(cudaMemcpyAsync(f, basis->f64, sizeof(double) * basis->K * basis->n_r, cudaMemcpyDeviceToDevice,
                           reinterpret_cast<cudaStream_t>(stream)));
  return TSR_OK;
}

extern "C" tsr_status tsr_basis_info(const tsr_basis *basis, int *K, int *n_r, double *r_max) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(basis, "tsr_basis_info: NULL basis");
  if (K) *K = basis->K;
  if (n_r) *n_r = basis->n_r;
  if (r_max) *r_max = basis->r_max;
  return TSR_OK;
}

extern "C" tsr_status tsr_basis_far_series(const tsr_basis *basis, double *rel_err, int *used) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(basis, "tsr_basis_far_series: NULL basis");
  if (rel_err) *rel_err = basis->cheb_err;
  if (used) *used = basis->cheb_ok ? 1 : 0;
  return TSR_OK;
}

extern "C" void tsr_basis_destroy(tsr_basis *b) {
  if (!b) return;
  cudaFree(b->f64);
  cudaFree(b->tab32);
  cudaFree(b->tab16);
  cudaFree(b->cheb);
  delete b;
}

extern "C" tsr_status tsr_project_material(const tsr_basis *basis, int n, const double *sigma_a,
                                           const double *sigma_s, const double *eta, double *g, float *g32,
                                           double *dg, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(basis && sigma_a && sigma_s && eta && g, "tsr_project_material: NULL argument");
  TSR_CHECK_ARG(n >= 0 && n <= (1 << 22), "tsr_project_material: n=%d out of range", n);
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(basis->device, "tsr_project_material");
  if (st != TSR_OK) return st;
  if (n == 0) return TSR_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double dr = basis->r_max / (basis->n_r - 1);
  // few edits: cut the samples of each (edit, channel) into ranges so that the grid fills the GPU
  const int n3 = n * 3;
  const int n_split = std::max(1, std::min(8, (2 * num_sms() + n3 - 1) / n3));
  Scratch ps;
  double *part = nullptr;
  if (n_split > 1) {
    st = ps.alloc(sizeof(double) * (size_t)n_split * n3 * (dg ? 64 : 16), s);
    if (st != TSR_OK) return st;
    part = static_cast<double *>(ps.p);
  }
  const dim3 grid(n3, n_split);
  if (dg)
    project_kernel<true><<<grid, 256, 0, s>>>(basis->f64, basis->K, basis->n_r, dr, sigma_a, sigma_s, eta, g, g32,
                                              dg, part);
  else
    project_kernel<false><<<grid, 256, 0, s>>>(basis->f64, basis->K, basis->n_r, dr, sigma_a, sigma_s, eta, g,
                                               g32, nullptr, part);
  ::tsr::count_launch();
  if (n_split > 1) {
    const int nt = n3 * basis->K;
    if (dg)
      project_finish_kernel<true><<<(nt + 255) / 256, 256, 0, s>>>(part, n3, n_split, basis->K, g, g32, dg);
    else
      project_finish_kernel<false><<<(nt + 255) / 256, 256, 0, s>>>(part, n3, n_split, basis->K, g, g32, nullptr);
    ::tsr::count_launch();
  }
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

extern "C" tsr_status tsr_project_material_backward(const tsr_basis *basis, int n, const double *sigma_a,
                                                    const double *sigma_s, const double *eta, const float *dLdg,
                                                    float *dsigma_a, float *dsigma_s, float *deta,
                                                    tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(basis && sigma_a && sigma_s && eta && dLdg && dsigma_a && dsigma_s && deta,
                "tsr_project_material_backward: NULL argument");
  TSR_CHECK_ARG(n >= 0 && n <= (1 << 22), "tsr_project_material_backward: n=%d out of range", n);
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(basis->device, "tsr_project_material_backward");
  if (st != TSR_OK) return st;
  if (n == 0) return TSR_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double dr = basis->r_max / (basis->n_r - 1);
  Scratch de_s;
  st = de_s.alloc(sizeof(double) * 3 * (size_t)n, s);
  if (st != TSR_OK) return st;
  double *de_part = static_cast<double *>(de_s.p);
  project_backward_kernel<<<n * 3, 256, 0, s>>>(basis->f64, basis->K, basis->n_r, dr, sigma_a, sigma_s, eta, dLdg,
                                                dsigma_a, dsigma_s, de_part); ::tsr::count_launch();
  project_eta_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(de_part, n, deta); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}
