// Fresnel transmittance factors of Eq. 3 and Eq. 6: S = (1/pi) F_t(eta, omega_i)
// R_d F_t(eta, omega_o).
//   * output side: B_out[e][c][o] = (1/pi) F_t(eta_e, cos_o[o]) B[e][c][o], with the
//     caller's per-vertex cosine cos_o = n_o . omega_o, and its reverse mode
//     (dL/dB and dL/deta_e, the latter reduced in a fixed order);
//   * incident side: F_t(eta, omega_i) folded into the unshadowed SH irradiance
//     transfer, T[j][i] = A_l(eta) Y_lm(n_i) with the Funk-Hecke zonal coefficients
//     A_l(eta) = 2 pi int_0^1 F_t(eta, mu) mu P_l(mu) dmu (eta = 1: the clamped cosine).
// F_t(eta, mu) = 1 - (r_s^2 + r_p^2) / 2, the exact unpolarised dielectric Fresnel
// reflectance for a direction at cosine mu > 0 outside (0 for mu <= 0).
#include <cmath>

#include "handles.cuh"

namespace tsr {

constexpr float kInvPiF = 0.318309886183790672f;
constexpr double kPi = 3.14159265358979323846;

// F_t and dF_t/deta (FP32)
__device__ __forceinline__ void fresnel_ft(float eta, float mu, float &Ft, float &dFt) {
  if (!(mu > 0.0f)) {
    Ft = 0.0f;
    dFt = 0.0f;
    return;
  }
  const float q = 1.0f - mu * mu;
  const float ct = sqrtf(fmaxf(1.0f - q / (eta * eta), 0.0f));   // cosine of the refracted ray
  const float dct = (ct > 0.0f) ? q / (eta * eta * eta * ct) : 0.0f;
  const float a = eta * ct, da = ct + eta * dct;
  const float rs = (mu - a) / (mu + a);
  const float drs = -2.0f * mu * da / ((mu + a) * (mu + a));
  const float u = eta * mu - ct, w = eta * mu + ct;
  const float rp = u / w;
  const float drp = ((mu - dct) * w - u * (mu + dct)) / (w * w);
  Ft = 1.0f - 0.5f * (rs * rs + rp * rp);
  dFt = -(rs * drs + rp * drp);
}

__device__ __forceinline__ double fresnel_ft64(double eta, double mu) {
  if (!(mu > 0.0)) return 0.0;
  const double ct = sqrt(fmax(1.0 - (1.0 - mu * mu) / (eta * eta), 0.0));
  const double rs = (mu - eta * ct) / (mu + eta * ct);
  const double rp = (eta * mu - ct) / (eta * mu + ct);
  return 1.0 - 0.5 * (rs * rs + rp * rp);
}

// Thread per (e, o): the factor once, applied to the three channels.
__global__ void fresnel_output_kernel(int E, int N, const double *__restrict__ eta, const float *__restrict__ cos_o,
                                      const float *__restrict__ B, float *__restrict__ Bout) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)E * N) return;
  const int e = (int)(t / N), o = (int)(t % N);
  float Ft, dFt;
  fresnel_ft((float)eta[e], cos_o[o], Ft, dFt);
  const float f = Ft * kInvPiF;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const size_t q = ((size_t)e * 3 + c) * N + o;
    Bout[q] = f * B[q];
  }
}

// dB = f dBout; the eta partials of block (o-chunk, e) go to part[e][chunk].
__global__ void __launch_bounds__(256) fresnel_output_backward_kernel(int E, int N, const double *__restrict__ eta,
                                                                     const float *__restrict__ cos_o,
                                                                     const float *__restrict__ B,
                                                                     const float *__restrict__ dBout,
                                                                     float *__restrict__ dB, float *__restrict__ part) {
  __shared__ float red[8];
  const int e = blockIdx.y;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.0f;
  if (o < N) {
    float Ft, dFt;
    fresnel_ft((float)eta[e], cos_o[o], Ft, dFt);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t q = ((size_t)e * 3 + c) * N + o;
      const float g = dBout[q];
      dB[q] = Ft * kInvPiF * g;
      acc = fmaf(g * B[q], dFt * kInvPiF, acc);
    }
  }
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float x = 0.0f;
    for (int w = 0; w < 8; ++w) x += red[w];
    part[(size_t)e * gridDim.x + blockIdx.x] = x;
  }
}

__global__ void fresnel_eta_finish_kernel(const float *__restrict__ part, int n_part, int E, float *__restrict__ deta) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  float x = 0.0f;
  for (int q = 0; q < n_part; ++q) x += part[(size_t)e * n_part + q];
  deta[e] = x;
}

// A_l(eta), l < order, by composite Simpson on [0, 1] (n_int intervals) in FP64: one block.
constexpr int SH_LMAX = 5;
__global__ void __launch_bounds__(256) sh_zonal_kernel(double eta, int order, int n_int, double *__restrict__ A) {
  __shared__ double red[SH_LMAX][8];
  double acc[SH_LMAX] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const double h = 1.0 / n_int;
  for (int q = threadIdx.x; q <= n_int; q += blockDim.x) {
    const double mu = q * h;
    const double wq = (q == 0 || q == n_int) ? 1.0 : ((q & 1) ? 4.0 : 2.0);
    const double hv = fresnel_ft64(eta, mu) * mu * wq;
    double p0 = 1.0, p1 = mu;   // Legendre P_0, P_1, then (l+1) P_{l+1} = (2l+1) mu P_l - l P_{l-1}
    acc[0] += hv * p0;
    if (order > 1) acc[1] += hv * p1;
    for (int l = 1; l + 1 < order; ++l) {
      const double p2 = ((2 * l + 1) * mu * p1 - l * p0) / (l + 1);
      acc[l + 1] += hv * p2;
      p0 = p1;
      p1 = p2;
    }
  }
  for (int l = 0; l < SH_LMAX; ++l) {
    double x = acc[l];
    for (int s = 16; s > 0; s >>= 1) x += __shfl_xor_sync(0xffffffffu, x, s);
    if ((threadIdx.x & 31) == 0) red[l][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < order) {
    double x = 0.0;
    for (int w = 0; w < 8; ++w) x += red[threadIdx.x][w];
    A[threadIdx.x] = 2.0 * kPi * x * h / 3.0;
  }
}

// T[j][i] = A_l Y_lm(n_i): real orthonormal SH (j = l^2 + l + m, no Condon-Shortley
// phase; m > 0: sqrt2 K cos(m phi) P_l^m, m < 0: sqrt2 K sin(|m| phi) P_l^|m|) in FP64.
__global__ void sh_transfer_kernel(int N, const float *__restrict__ normals, int order, const double *__restrict__ A,
                                   float *__restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double x = normals[i], y = normals[N + i], z = fmin(fmax((double)normals[2 * N + i], -1.0), 1.0);
  const double st = sqrt(fmax(0.0, 1.0 - z * z));
  const double phi = atan2(y, x);
  double P[SH_LMAX][SH_LMAX];   // P[l][m]
  P[0][0] = 1.0;
  for (int m = 1; m < order; ++m) P[m][m] = P[m - 1][m - 1] * (2 * m - 1) * st;
  for (int m = 0; m < order; ++m) {
    if (m + 1 < order) P[m + 1][m] = z * (2 * m + 1) * P[m][m];
    for (int l = m + 2; l < order; ++l) P[l][m] = ((2 * l - 1) * z * P[l - 1][m] - (l + m - 1) * P[l - 2][m]) / (l - m);
  }
  for (int l = 0; l < order; ++l) {
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      double ratio = 1.0;   // (l - |m|)! / (l + |m|)!
      for (int q = l - am + 1; q <= l + am; ++q) ratio /= q;
      const double K = sqrt((2 * l + 1) / (4.0 * kPi) * ratio);
      double v;
      if (m == 0) v = K * P[l][0];
      else if (m > 0) v = sqrt(2.0) * K * cos(m * phi) * P[l][am];
      else v = sqrt(2.0) * K * sin(am * phi) * P[l][am];
      T[(size_t)(l * l + l + m) * N + i] = (float)(A[l] * v);
    }
  }
}

tsr_status fresnel_output(int E, const double *eta, int N, const float *cos_o, const float *B, float *Bout,
                          cudaStream_t s) {
  const long long n = (long long)E * N;
  fresnel_output_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(E, N, eta, cos_o, B, Bout); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

tsr_status fresnel_output_backward(int E, const double *eta, int N, const float *cos_o, const float *B,
                                   const float *dBout, float *dB, float *deta, cudaStream_t s) {
  const int nb = (N + 255) / 256;
  Scratch ps;
  tsr_status st = ps.alloc(sizeof(float) * (size_t)E * nb, s);
  if (st != TSR_OK) return st;
  float *part = static_cast<float *>(ps.p);
  fresnel_output_backward_kernel<<<dim3(nb, E), 256, 0, s>>>(E, N, eta, cos_o, B, dBout, dB, part);
  ::tsr::count_launch();
  fresnel_eta_finish_kernel<<<(E + 255) / 256, 256, 0, s>>>(part, nb, E, deta); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

tsr_status sh_transfer(int N, const float *normals, int J, double eta, float *T, cudaStream_t s) {
  const int order = (int)lround(std::sqrt((double)J));
  Scratch as;
  tsr_status st = as.alloc(sizeof(double) * SH_LMAX, s);
  if (st != TSR_OK) return st;
  double *A = static_cast<double *>(as.p);
  sh_zonal_kernel<<<1, 256, 0, s>>>(eta, order, 1 << 14, A); ::tsr::count_launch();
  sh_transfer_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, normals, order, A, T); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

}  // namespace tsr
