// extern "C" entry points of libtsr: argument validation and dispatch.
#include <algorithm>
#include <vector>

#include "handles.cuh"

using namespace tsr;

namespace {
cudaStream_t as_stream(tsr_stream s) { return reinterpret_cast<cudaStream_t>(s); }
bool chart_mesh(int N, int nu) { return nu >= 1 && N == 10 * nu * nu + 2; }
}  // namespace

extern "C" const char *tsr_last_error(void) { return error_string(); }

extern "C" int tsr_version(void) { return 100; }

extern "C" tsr_status tsr_stream_status(tsr_stream stream) {
  TSR_API_ENTRY();
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  TSR_CUDA(cudaStreamSynchronize(as_stream(stream)));
  return check_device_status(as_stream(stream));
}

extern "C" tsr_status tsr_precompute_transfer(const tsr_basis *basis, int N, const float *pos, const float *area,
                                              const float *T, int J, tsr_precision prec, float *M,
                                              tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(basis && pos && area && T && M, "tsr_precompute_transfer: NULL argument");
  TSR_CHECK_ARG(N >= 12 && N <= (1 << 24), "tsr_precompute_transfer: N=%d outside [12, 2^24]", N);
  TSR_CHECK_ARG(J >= 1 && J <= 32, "tsr_precompute_transfer: J=%d outside [1, 32]", J);
  TSR_CHECK_ARG(aligned(pos, 16) && aligned(area, 4) && aligned(T, 4) && aligned(M, 4),
                "tsr_precompute_transfer: misaligned pointer");
  TSR_CHECK_ARG((size_t)basis->K * J * (size_t)N < ((size_t)1 << 40), "tsr_precompute_transfer: output too large");
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(basis->device, "tsr_precompute_transfer");
  if (st != TSR_OK) return st;
  switch (prec) {
    case TSR_FP32:
      return transfer_fp32(basis, N, pos, area, T, J, M, as_stream(stream));
    case TSR_BF16:
      return transfer_tc(basis, N, pos, area, T, J, false, M, as_stream(stream));
    case TSR_BF16X3:
      return transfer_tc(basis, N, pos, area, T, J, true, M, as_stream(stream));
    default:
      set_error("tsr_precompute_transfer: unknown precision %d", (int)prec);
      return TSR_ERR_UNSUPPORTED;
  }
}

extern "C" tsr_status tsr_precompute_transfer_batched(const tsr_basis *basis, int n_mesh, const int64_t *offsets,
                                                      const float *pos, const float *area, const float *T, int J,
                                                      tsr_precision prec, float *M, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(basis && offsets && pos && area && T && M, "tsr_precompute_transfer_batched: NULL argument");
  TSR_CHECK_ARG(n_mesh >= 1 && n_mesh <= 65536, "tsr_precompute_transfer_batched: n_mesh=%d out of range", n_mesh);
  TSR_CHECK_ARG(J >= 1 && J <= 32, "tsr_precompute_transfer_batched: J=%d outside [1, 32]", J);
  TSR_CHECK_ARG(offsets[0] == 0, "tsr_precompute_transfer_batched: offsets[0] must be 0");
  for (int b = 0; b < n_mesh; ++b)
    TSR_CHECK_ARG(offsets[b + 1] - offsets[b] >= 12 && offsets[b + 1] - offsets[b] <= (1 << 24),
                  "tsr_precompute_transfer_batched: mesh %d has %lld vertices", b,
                  (long long)(offsets[b + 1] - offsets[b]));
  TSR_CHECK_ARG(aligned(pos, 16), "tsr_precompute_transfer_batched: misaligned pos");
  TSR_CHECK_ARG(prec == TSR_BF16 || prec == TSR_FP32, "tsr_precompute_transfer_batched: precision %d unsupported",
                (int)prec);
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(basis->device, "tsr_precompute_transfer_batched");
  if (st != TSR_OK) return st;
  if (prec == TSR_BF16) return transfer_tc_batched(basis, n_mesh, offsets, pos, area, T, J, M, as_stream(stream));
  return transfer_fp32_batched(basis, n_mesh, offsets, pos, area, T, J, M, as_stream(stream));
}

extern "C" tsr_status tsr_haar_forward(const float *X, int rows, int nu, float *Xw, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(X && Xw, "tsr_haar_forward: NULL argument");
  TSR_CHECK_ARG(rows >= 0 && rows <= (1 << 20), "tsr_haar_forward: rows=%d out of range", rows);
  TSR_CHECK_ARG(nu >= 1 && nu <= 128, "tsr_haar_forward: nu=%d outside [1, 128]", nu);
  tsr_status st = require_device();
  if (st != TSR_OK || rows == 0) return st;
  return haar_forward(X, rows, nu, Xw, as_stream(stream));
}

extern "C" tsr_status tsr_haar_inverse(const float *Xw, int rows, int nu, float *X, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(X && Xw, "tsr_haar_inverse: NULL argument");
  TSR_CHECK_ARG(rows >= 0 && rows <= (1 << 20), "tsr_haar_inverse: rows=%d out of range", rows);
  TSR_CHECK_ARG(nu >= 1 && nu <= 128, "tsr_haar_inverse: nu=%d outside [1, 128]", nu);
  tsr_status st = require_device();
  if (st != TSR_OK || rows == 0) return st;
  return haar_inverse(Xw, rows, nu, X, as_stream(stream));
}

extern "C" tsr_status tsr_wavelet_compress(const float *Mw, int K, int J, int nu, double p, tsr_compressed **out,
                                           tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(Mw && out, "tsr_wavelet_compress: NULL argument");
  TSR_CHECK_ARG(K >= 1 && K <= 16 && J >= 1 && J <= 32, "tsr_wavelet_compress: K=%d J=%d out of range", K, J);
  TSR_CHECK_ARG(nu >= 1 && nu <= 128, "tsr_wavelet_compress: nu=%d outside [1, 128]", nu);
  TSR_CHECK_ARG(p >= 0.0 && p <= 1.0, "tsr_wavelet_compress: p=%g outside [0, 1]", p);
  *out = nullptr;
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  return wavelet_compress(Mw, K, J, nu, p, out, as_stream(stream));
}

extern "C" tsr_status tsr_haar_compress(const float *M, int K, int J, int nu, double p, tsr_compressed **out,
                                        tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(M && out, "tsr_haar_compress: NULL argument");
  TSR_CHECK_ARG(K >= 1 && K <= 16 && J >= 1 && J <= 32, "tsr_haar_compress: K=%d J=%d out of range", K, J);
  TSR_CHECK_ARG(nu >= 1 && nu <= 128, "tsr_haar_compress: nu=%d outside [1, 128]", nu);
  TSR_CHECK_ARG(p >= 0.0 && p <= 1.0, "tsr_haar_compress: p=%g outside [0, 1]", p);
  *out = nullptr;
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  cudaStream_t s = as_stream(stream);
  const int P = chart_side(nu);
  Scratch mw;
  st = mw.alloc(sizeof(float) * (size_t)K * J * (10 * P * P + 2), s);
  if (st != TSR_OK) return st;
  st = haar_forward(M, K * J, nu, static_cast<float *>(mw.p), s);
  if (st != TSR_OK) return st;
  return wavelet_compress(static_cast<float *>(mw.p), K, J, nu, p, out, s);
}

extern "C" tsr_status tsr_haar_compress_energy(const float *M, int K, int J, int nu, double energy,
                                               tsr_compressed **out, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(M && out, "tsr_haar_compress_energy: NULL argument");
  TSR_CHECK_ARG(K >= 1 && K <= 16 && J >= 1 && J <= 32, "tsr_haar_compress_energy: K=%d J=%d out of range", K, J);
  TSR_CHECK_ARG(nu >= 1 && nu <= 128, "tsr_haar_compress_energy: nu=%d outside [1, 128]", nu);
  TSR_CHECK_ARG(energy > 0.0 && energy <= 1.0, "tsr_haar_compress_energy: energy=%g outside (0, 1]", energy);
  *out = nullptr;
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  cudaStream_t s = as_stream(stream);
  const int P = chart_side(nu);
  Scratch mw;
  st = mw.alloc(sizeof(float) * (size_t)K * J * (10 * P * P + 2), s);
  if (st != TSR_OK) return st;
  st = haar_forward(M, K * J, nu, static_cast<float *>(mw.p), s);
  if (st != TSR_OK) return st;
  return wavelet_compress_energy(static_cast<float *>(mw.p), K, J, nu, energy, out, s);
}

extern "C" tsr_status tsr_compress(const float *M, int K, int J, int nu, int wavelet, int rule, double param,
                                   tsr_compressed **out, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(M && out, "tsr_compress: NULL argument");
  TSR_CHECK_ARG(K >= 1 && K <= 16 && J >= 1 && J <= 32, "tsr_compress: K=%d J=%d out of range", K, J);
  TSR_CHECK_ARG(nu >= 1 && nu <= 128, "tsr_compress: nu=%d outside [1, 128]", nu);
  TSR_CHECK_ARG(wavelet == TSR_WAVELET_HAAR || wavelet == TSR_WAVELET_CDF97, "tsr_compress: wavelet=%d unknown",
                wavelet);
  TSR_CHECK_ARG(rule == TSR_KEEP_TOP_FRACTION || rule == TSR_KEEP_ENERGY, "tsr_compress: rule=%d unknown", rule);
  TSR_CHECK_ARG(rule == TSR_KEEP_TOP_FRACTION ? (param >= 0.0 && param <= 1.0) : (param > 0.0 && param <= 1.0),
                "tsr_compress: param=%g out of range for the rule", param);
  *out = nullptr;
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  cudaStream_t s = as_stream(stream);
  const int P = chart_side(nu);
  Scratch mw;
  st = mw.alloc(sizeof(float) * (size_t)K * J * (10 * P * P + 2), s);
  if (st != TSR_OK) return st;
  float *Mw = static_cast<float *>(mw.p);
  st = spatial_forward(wavelet, M, K * J, nu, Mw, s);
  if (st != TSR_OK) return st;
  st = (rule == TSR_KEEP_ENERGY) ? wavelet_compress_energy(Mw, K, J, nu, param, out, s)
                                 : wavelet_compress(Mw, K, J, nu, param, out, s);
  if (st == TSR_OK) (*out)->wavelet = wavelet;
  return st;
}

extern "C" tsr_status tsr_cdf97_forward(const float *X, int rows, int nu, float *Xw, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(X && Xw, "tsr_cdf97_forward: NULL argument");
  TSR_CHECK_ARG(rows >= 1 && nu >= 1 && nu <= 128, "tsr_cdf97_forward: rows=%d nu=%d out of range", rows, nu);
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  return cdf97_forward(X, rows, nu, Xw, as_stream(stream));
}

extern "C" tsr_status tsr_cdf97_inverse(const float *Xw, int rows, int nu, float *X, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(X && Xw, "tsr_cdf97_inverse: NULL argument");
  TSR_CHECK_ARG(rows >= 1 && nu >= 1 && nu <= 128, "tsr_cdf97_inverse: rows=%d nu=%d out of range", rows, nu);
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  return cdf97_inverse(Xw, rows, nu, X, as_stream(stream));
}

extern "C" tsr_status tsr_cdf97_inverse_transpose(const float *X, int rows, int nu, float *Xw, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(X && Xw, "tsr_cdf97_inverse_transpose: NULL argument");
  TSR_CHECK_ARG(rows >= 1 && nu >= 1 && nu <= 128, "tsr_cdf97_inverse_transpose: rows=%d nu=%d out of range", rows,
                nu);
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  return cdf97_inverse_transpose(X, rows, nu, Xw, as_stream(stream));
}

extern "C" tsr_status tsr_fresnel_output(int n_edit, const double *eta, int N, const float *cos_o, const float *B,
                                         float *Bout, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(eta && cos_o && B && Bout, "tsr_fresnel_output: NULL argument");
  TSR_CHECK_ARG(n_edit >= 0 && n_edit <= (1 << 20) && N >= 1, "tsr_fresnel_output: n_edit=%d N=%d out of range",
                n_edit, N);
  TSR_CHECK_ARG(aligned(cos_o, 4) && aligned(B, 4) && aligned(Bout, 4) && aligned(eta, 8),
                "tsr_fresnel_output: misaligned pointer");
  tsr_status st = require_device();
  if (st != TSR_OK || n_edit == 0) return st;
  return fresnel_output(n_edit, eta, N, cos_o, B, Bout, as_stream(stream));
}

extern "C" tsr_status tsr_fresnel_output_backward(int n_edit, const double *eta, int N, const float *cos_o,
                                                  const float *B, const float *dBout, float *dB, float *deta,
                                                  tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(eta && cos_o && B && dBout && dB && deta, "tsr_fresnel_output_backward: NULL argument");
  TSR_CHECK_ARG(n_edit >= 1 && n_edit <= (1 << 20) && N >= 1,
                "tsr_fresnel_output_backward: n_edit=%d N=%d out of range", n_edit, N);
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  return fresnel_output_backward(n_edit, eta, N, cos_o, B, dBout, dB, deta, as_stream(stream));
}

extern "C" tsr_status tsr_sh_transfer(int N, const float *normals, int J, double eta, float *T, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(normals && T, "tsr_sh_transfer: NULL argument");
  TSR_CHECK_ARG(N >= 1, "tsr_sh_transfer: N=%d", N);
  TSR_CHECK_ARG(J == 1 || J == 4 || J == 9 || J == 16 || J == 25, "tsr_sh_transfer: J=%d is not a square <= 25", J);
  TSR_CHECK_ARG(eta >= 1.0 && eta <= 2.0, "tsr_sh_transfer: eta=%g outside [1, 2]", eta);
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  return sh_transfer(N, normals, J, eta, T, as_stream(stream));
}

extern "C" tsr_status tsr_visibility_transfer(int N, const float *pos, const float *normals, int F,
                                              const int32_t *tris, int J, int S, double eta, float eps, float *T,
                                              tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(pos && normals && tris && T, "tsr_visibility_transfer: NULL argument");
  TSR_CHECK_ARG(N >= 1 && F >= 1 && F <= (1 << 26), "tsr_visibility_transfer: N=%d F=%d out of range", N, F);
  TSR_CHECK_ARG(J == 1 || J == 4 || J == 9 || J == 16 || J == 25, "tsr_visibility_transfer: J=%d", J);
  TSR_CHECK_ARG(S >= 1 && S <= 65536, "tsr_visibility_transfer: S=%d outside [1, 65536]", S);
  TSR_CHECK_ARG(eta == 0.0 || (eta >= 1.0 && eta <= 2.0), "tsr_visibility_transfer: eta=%g (0, or [1, 2])", eta);
  TSR_CHECK_ARG(eps >= 0.0f, "tsr_visibility_transfer: eps=%g < 0", (double)eps);
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  return visibility_transfer(N, pos, normals, F, tris, J, S, eta, eps, T, as_stream(stream));
}

extern "C" tsr_status tsr_haar_recompress(const float *M, tsr_compressed *c, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(M && c, "tsr_haar_recompress: NULL argument");
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(c->device, "tsr_haar_recompress");
  if (st != TSR_OK) return st;
  cudaStream_t s = as_stream(stream);
  Scratch mw;
  st = mw.alloc(sizeof(float) * (size_t)c->K * c->J * c->n_rows, s);
  if (st != TSR_OK) return st;
  st = spatial_forward(c->wavelet, M, c->K * c->J, c->nu, static_cast<float *>(mw.p), s);
  if (st != TSR_OK) return st;
  return wavelet_compress_into(static_cast<float *>(mw.p), c, s);
}

// nu of a mesh of N vertices in the chart layout (N = 10 nu^2 + 2), or 0.
static int chart_nu_of(int64_t N) {
  for (int nu = 1; nu <= 128; ++nu)
    if (10 * (int64_t)nu * nu + 2 == N) return nu;
  return 0;
}

extern "C" tsr_status tsr_haar_compress_batched(int n_mesh, const int64_t *offsets, const float *M, int K, int J,
                                                double p, tsr_compressed **out, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(offsets && M && out, "tsr_haar_compress_batched: NULL argument");
  TSR_CHECK_ARG(n_mesh >= 1 && n_mesh <= 65536, "tsr_haar_compress_batched: n_mesh=%d out of range", n_mesh);
  TSR_CHECK_ARG(K >= 1 && K <= 16 && J >= 1 && J <= 32, "tsr_haar_compress_batched: K=%d J=%d out of range", K, J);
  TSR_CHECK_ARG(p >= 0.0 && p <= 1.0, "tsr_haar_compress_batched: p=%g outside [0, 1]", p);
  TSR_CHECK_ARG(offsets[0] == 0, "tsr_haar_compress_batched: offsets[0] must be 0");
  for (int b = 0; b < n_mesh; ++b) {
    out[b] = nullptr;
    TSR_CHECK_ARG(chart_nu_of(offsets[b + 1] - offsets[b]) > 0,
                  "tsr_haar_compress_batched: mesh %d has %lld vertices, not 10 nu^2 + 2 with nu <= 128", b,
                  (long long)(offsets[b + 1] - offsets[b]));
  }
  tsr_status st = require_device();
  if (st != TSR_OK) return st;
  return haar_compress_many(n_mesh, offsets, M, K, J, p, out, as_stream(stream));
}

extern "C" tsr_status tsr_haar_recompress_batched(int n_mesh, const int64_t *offsets, const float *M,
                                                  tsr_compressed *const *c, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(offsets && M && c, "tsr_haar_recompress_batched: NULL argument");
  TSR_CHECK_ARG(n_mesh >= 1 && n_mesh <= 65536, "tsr_haar_recompress_batched: n_mesh=%d out of range", n_mesh);
  TSR_CHECK_ARG(offsets[0] == 0, "tsr_haar_recompress_batched: offsets[0] must be 0");
  for (int b = 0; b < n_mesh; ++b) {
    TSR_CHECK_ARG(c[b], "tsr_haar_recompress_batched: handle %d is NULL", b);
    TSR_CHECK_ARG(c[b]->wavelet == 0 && c[b]->keep_rule == 0,
                  "tsr_haar_recompress_batched: handle %d is not a Haar top-fraction handle", b);
    TSR_CHECK_ARG(offsets[b + 1] - offsets[b] == 10 * (int64_t)c[b]->nu * c[b]->nu + 2,
                  "tsr_haar_recompress_batched: mesh %d has %lld vertices, its handle nu=%d", b,
                  (long long)(offsets[b + 1] - offsets[b]), c[b]->nu);
    TSR_CHECK_ARG(c[b]->K == c[0]->K && c[b]->J == c[0]->J,
                  "tsr_haar_recompress_batched: handle %d has K=%d J=%d, handle 0 K=%d J=%d", b, c[b]->K, c[b]->J,
                  c[0]->K, c[0]->J);
  }
  tsr_status st = require_device();
  for (int b = 0; b < n_mesh && st == TSR_OK; ++b) st = require_same_device(c[b]->device, "tsr_haar_recompress_batched");
  if (st != TSR_OK) return st;
  return haar_recompress_many(n_mesh, offsets, M, c, as_stream(stream));
}

extern "C" tsr_status tsr_compressed_info(const tsr_compressed *c, int *K, int *J, int *nu, int64_t *nnz,
                                          int *n_rows) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(c, "tsr_compressed_info: NULL handle");
  if (K) *K = c->K;
  if (J) *J = c->J;
  if (nu) *nu = c->nu;
  if (nnz) *nnz = c->nnz;
  if (n_rows) *n_rows = c->n_rows;
  return TSR_OK;
}

extern "C" tsr_status tsr_compressed_export(const tsr_compressed *c, int64_t *row_ptr, uint16_t *col, float *val,
                                            tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(c && row_ptr && col && val, "tsr_compressed_export: NULL argument");
  cudaStream_t s = as_stream(stream);
  TSR_CUDA(cudaMemcpyAsync(row_ptr, c->row_ptr, sizeof(int64_t) * (c->n_rows + 1), cudaMemcpyDeviceToDevice, s));
  TSR_CUDA(cudaMemcpyAsync(col, c->col, sizeof(uint16_t) * c->nnz, cudaMemcpyDeviceToDevice, s));
  TSR_CUDA(cudaMemcpyAsync(val, c->val, sizeof(float) * c->nnz, cudaMemcpyDeviceToDevice, s));
  return TSR_OK;
}

extern "C" tsr_status tsr_relight(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B,
                                  tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(c && g && l && B, "tsr_relight: NULL argument");
  TSR_CHECK_ARG(n_edit >= 0 && n_edit <= (1 << 20), "tsr_relight: n_edit=%d out of range", n_edit);
  TSR_CHECK_ARG(aligned(g, 4) && aligned(l, 4) && aligned(B, 4), "tsr_relight: misaligned pointer");
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(c->device, "tsr_relight");
  if (st != TSR_OK || n_edit == 0) return st;
  return relight(c, n_edit, g, l, B, as_stream(stream));
}

extern "C" tsr_status tsr_relight_many(int n_copy, const tsr_compressed *const *c, int n_edit, const float *g,
                                       const float *l, float *B, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(n_copy >= 0 && n_copy <= 65536, "tsr_relight_many: n_copy=%d out of range", n_copy);
  TSR_CHECK_ARG(n_edit >= 0 && n_edit <= (1 << 20), "tsr_relight_many: n_edit=%d out of range", n_edit);
  if (n_copy == 0) return TSR_OK;
  TSR_CHECK_ARG(c && g && l && B, "tsr_relight_many: NULL argument");
  TSR_CHECK_ARG(aligned(g, 4) && aligned(l, 4) && aligned(B, 4), "tsr_relight_many: misaligned pointer");
  for (int i = 0; i < n_copy; ++i) {
    TSR_CHECK_ARG(c[i], "tsr_relight_many: handle %d is NULL", i);
    TSR_CHECK_ARG(c[i]->K == c[0]->K && c[i]->J == c[0]->J, "tsr_relight_many: handle %d has K=%d J=%d, handle 0 K=%d J=%d",
                  i, c[i]->K, c[i]->J, c[0]->K, c[0]->J);
  }
  tsr_status st = require_device();
  for (int i = 0; i < n_copy && st == TSR_OK; ++i) st = require_same_device(c[i]->device, "tsr_relight_many");
  if (st != TSR_OK || n_edit == 0) return st;
  cudaStream_t s = as_stream(stream);
  const size_t V = 3 * (size_t)n_edit, K = (size_t)c[0]->K;
  const bool few = n_edit <= 2;
  std::vector<const tsr_compressed *> fc;
  std::vector<const float *> fg;
  std::vector<float *> fb;
  std::vector<int> fn;
  size_t off = 0, z_total = 0;
  for (int i = 0; i < n_copy; ++i) {
    const float *gi = g + (size_t)i * V * K;
    float *Bi = B + off;
    const int Ni = 10 * c[i]->nu * c[i]->nu + 2;
    off += V * (size_t)Ni;
    if (few ? relight_fusable(c[i], n_edit) : relight_fusable_basis(c[i])) {
      fc.push_back(c[i]);
      fg.push_back(gi);
      fb.push_back(Bi);
      fn.push_back(Ni);
      z_total += K * (size_t)Ni;
    } else {
      st = relight(c[i], n_edit, gi, l, Bi, s);
      if (st != TSR_OK) return st;
    }
  }
  if (fc.empty()) return TSR_OK;
  if (few) return relight_fused((int)fc.size(), fc.data(), n_edit, fg.data(), l, fb.data(), s);
  // more edits: the light-contracted basis images of every copy, then one combine
  Scratch sc;
  st = sc.alloc(sizeof(float) * z_total, s);
  if (st != TSR_OK) return st;
  std::vector<float *> zi(fc.size());
  float *zp = static_cast<float *>(sc.p);
  for (size_t i = 0; i < fc.size(); ++i) {
    zi[i] = zp;
    zp += K * (size_t)fn[i];
  }
  st = relight_basis_images_many((int)fc.size(), fc.data(), l, zi.data(), s);
  if (st != TSR_OK) return st;
  return relight_combine_many((int)fc.size(), zi.data(), fn.data(), (int)K, (int)V, fg.data(), fb.data(), s);
}

extern "C" tsr_status tsr_relight_backward(const tsr_compressed *c, int n_edit, const float *g, const float *l,
                                           const float *dLdB, float *dg, float *dl, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(c && g && l && dLdB && dg && dl, "tsr_relight_backward: NULL argument");
  TSR_CHECK_ARG(n_edit >= 1 && n_edit <= (1 << 20), "tsr_relight_backward: n_edit=%d out of range", n_edit);
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(c->device, "tsr_relight_backward");
  if (st != TSR_OK) return st;
  return relight_backward(c, n_edit, g, l, dLdB, dg, dl, as_stream(stream));
}

extern "C" tsr_status tsr_batch_plan_create(const tsr_basis *basis, int n_mesh, const int64_t *offsets, int J,
                                            tsr_precision prec, tsr_batch_plan **out) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(basis && offsets && out, "tsr_batch_plan_create: NULL argument");
  TSR_CHECK_ARG(n_mesh >= 1 && n_mesh <= 65536, "tsr_batch_plan_create: n_mesh=%d out of range", n_mesh);
  TSR_CHECK_ARG(J >= 1 && J <= 32, "tsr_batch_plan_create: J=%d outside [1, 32]", J);
  TSR_CHECK_ARG(offsets[0] == 0, "tsr_batch_plan_create: offsets[0] must be 0");
  for (int b = 0; b < n_mesh; ++b)
    TSR_CHECK_ARG(offsets[b + 1] - offsets[b] >= 12 && offsets[b + 1] - offsets[b] <= (1 << 24),
                  "tsr_batch_plan_create: mesh %d has %lld vertices", b, (long long)(offsets[b + 1] - offsets[b]));
  TSR_CHECK_ARG(prec == TSR_BF16 || prec == TSR_FP32, "tsr_batch_plan_create: precision %d unsupported", (int)prec);
  *out = nullptr;
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(basis->device, "tsr_batch_plan_create");
  if (st != TSR_OK) return st;
  return batch_plan_create(basis, n_mesh, offsets, J, (int)prec, out);
}

extern "C" tsr_status tsr_precompute_transfer_plan(const tsr_batch_plan *plan, const float *pos, const float *area,
                                                   const float *T, float *M, tsr_stream stream) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(plan && pos && area && T && M, "tsr_precompute_transfer_plan: NULL argument");
  TSR_CHECK_ARG(aligned(pos, 16), "tsr_precompute_transfer_plan: misaligned pos");
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(plan->device, "tsr_precompute_transfer_plan");
  if (st != TSR_OK) return st;
  return batch_plan_run(plan, pos, area, T, M, as_stream(stream));
}

extern "C" tsr_status tsr_batch_plan_autotune(tsr_batch_plan *plan, const float *pos, const float *area,
                                              const float *T, float *M, tsr_stream stream, float *best_ms) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(plan && pos && area && T && M, "tsr_batch_plan_autotune: NULL argument");
  tsr_status st = require_device();
  if (st == TSR_OK) st = require_same_device(plan->device, "tsr_batch_plan_autotune");
  if (st != TSR_OK) return st;
  return batch_plan_autotune(plan, pos, area, T, M, as_stream(stream), best_ms);
}

extern "C" tsr_status tsr_batch_plan_info(const tsr_batch_plan *plan, int *n_units, int *generator, int *param) {
  TSR_API_ENTRY();
  TSR_CHECK_ARG(plan, "tsr_batch_plan_info: NULL plan");
  const int gen = (plan->gen == 0 && plan->basis->cheb_ok) ? 0 : 1;
  if (n_units) *n_units = plan->n_units;
  if (generator) *generator = gen;
  if (param) *param = gen == 0 ? plan->conc : plan->kb;
  return TSR_OK;
}

extern "C" void tsr_batch_plan_destroy(tsr_batch_plan *plan) {
  if (!plan) return;
  cudaFree(plan->tables);
  delete plan;
}
