// Library-owned objects behind the opaque handles of tsr.h.
#pragma once
#include <vector>

#include "tsr_internal.cuh"

// Radial basis f_k on the grid r_m = r_max m / (n_r - 1) plus the lookup tables
// the transfer kernels read.  Row n_r of each table is all zero: kernels send
// pairs beyond the cutoff there instead of branching.
struct tsr_basis {
  int device = -1;
  int K = 0, n_r = 0, KP = 0;   // KP: K rounded up to a multiple of 4
  double r_max = 0.0;
  double *f64 = nullptr;        // [K][n_r]
  float2 *tab32 = nullptr;      // [n_r + 1][KP]  {f_k(r_m), f_k(r_m+1) - f_k(r_m)}
  uint32_t *tab16 = nullptr;    // [n_r + 1][KP]  bf16x2 {lo: value, hi: slope}
  // Far field of the BF16 transfer: for r_near <= r <= r_max,
  //   f_k(r) ~= sum_p cheb[k][p] W_p(r),  W_p = sigma_p T_p(x) / r^2,
  // x = x_alpha log2(r^2) + x_beta in [-1, 1] (linear in log r), sigma_p = (-1)^(p(p-1)/2).
  float *cheb = nullptr;        // [K][TSR_CHEB_P] (+ the fit-check scratch)
  double r_near = 0.0;
  float x_alpha = 0.f, x_beta = 0.f;
  double cheb_err = 0.0;        // max_k relative error of the TSR_CHEB_BF16-term series on [r_near, r_max]
  bool cheb_ok = false;         // cheb_err <= TSR_CHEB_MAX_ERR: the BF16 transfer uses the series
};
#define TSR_CHEB_P 16          // Chebyshev coefficients kept per basis
#define TSR_CHEB_BF16 12       // terms the BF16 far field generates
#define TSR_CHEB_NODES 256     // Chebyshev nodes of the projection
#define TSR_CHEB_MAX_ERR 2e-3  // largest accepted relative error of the truncated series

// Compressed wavelet transfer: CSR over wavelet rows w in [0, 10 P^2 + 2).
struct tsr_compressed {
  int device = -1;
  int K = 0, J = 0, nu = 0, P = 0, n_rows = 0;
  int n_keep = 0;               // per (k, j) under the top-p rule; -1 under the energy rule
  int keep_rule = 0;            // 0: top-p fraction, 1: energy threshold
  int wavelet = 0;              // 0: orthonormal Haar over the Morton order, 1: CDF 9/7 2D pyramid
  int64_t nnz = 0;
  int64_t *row_ptr = nullptr;   // [n_rows + 1]
  uint16_t *col = nullptr;      // [nnz]  k*J + j
  float *val = nullptr;         // [nnz]
  // The same entries by column, used by the reverse mode: column kj holds its
  // n_keep + 2 entries (ascending wavelet row) at [col_ptr[kj], col_ptr[kj+1]).
  int32_t *cidx = nullptr;      // [nnz] wavelet rows
  float *cval = nullptr;        // [nnz]
  int64_t *col_ptr = nullptr;   // [K*J + 1]
};

// Batched-transfer plan: unit and mesh tables on the device (built once, outside
// any stream capture) and the chosen tile configuration.
struct tsr_batch_plan {
  int device = -1;
  const tsr_basis *basis = nullptr;
  int n_mesh = 0, J = 0, total_steps = 0, n_units = 0;
  long long total = 0;
  int prec = 1;                 // tsr_precision
  int gen = 0;                  // BF16 generator: 0 far-field series, 1 table
  int conc = 0;                 // series: steps in flight (0: default)
  int kb = 0;                   // table: bases per CTA group (0: default for K)
  std::vector<int64_t> offsets; // host copy
  void *tables = nullptr;       // device: units | voff | N | soff
  int4 *d_units = nullptr;
  long long *d_voff = nullptr;
  int *d_N = nullptr, *d_soff = nullptr;
};

namespace tsr {
// Exact FP32 near field of the BF16 transfer (near.cu): pairs with r^2 < r_e^2 of
// their mesh.  near_setup computes r_e^2 per mesh (rn2, read by the far-field
// kernels too) and the Morton-sorted copies; near_apply adds the near sums to M.
// The scratch lives in `buf` until the NearField goes out of scope (stream-ordered).
struct NearField {
  Scratch buf;
  int n_mesh = 1, J = 0, JP = 0, n_tiles = 0, n_chunks = 0;
  long long total = 0, np = 0;
  const long long *voff = nullptr;   // [n_mesh + 1] device (NULL: one mesh)
  float *rn2 = nullptr;              // [n_mesh] r_e^2 per mesh
  int *perm = nullptr;               // sorted position -> vertex
  float *pos_s = nullptr;            // [3][np] sorted positions
  float *tq = nullptr;               // [np][JP] sorted A_i T[j][i] (FP32)
  int *mesh_s = nullptr;             // [np] mesh of each sorted vertex (-1: padding)
  float *tile_box = nullptr, *chunk_box = nullptr;
};
tsr_status near_setup(NearField &nf, const tsr_basis *b, int n_mesh, const long long *d_voff, long long total,
                      const float *pos, long long stride, const float *area, const float *T, int J, cudaStream_t s);
tsr_status near_apply(const NearField &nf, const tsr_basis *b, float *M, long long stride, cudaStream_t s);

tsr_status batch_plan_create(const tsr_basis *b, int n_mesh, const int64_t *offsets, int J, int prec,
                             tsr_batch_plan **out);
tsr_status batch_plan_run(const tsr_batch_plan *p, const float *pos, const float *area, const float *T, float *M,
                          cudaStream_t s);
tsr_status batch_plan_autotune(tsr_batch_plan *p, const float *pos, const float *area, const float *T, float *M,
                               cudaStream_t s, float *best_ms);
tsr_status basis_build_tables(tsr_basis *b, cudaStream_t s);
tsr_status transfer_fp32(const tsr_basis *b, int N, const float *pos, const float *area, const float *T,
                         int J, float *M, cudaStream_t s, long long stride = 0);
tsr_status transfer_tc(const tsr_basis *b, int N, const float *pos, const float *area, const float *T,
                       int J, bool split, float *M, cudaStream_t s);
tsr_status transfer_tc_batched(const tsr_basis *b, int n_mesh, const int64_t *offsets, const float *pos,
                               const float *area, const float *T, int J, float *M, cudaStream_t s);
tsr_status transfer_fp32_batched(const tsr_basis *b, int n_mesh, const int64_t *offsets, const float *pos,
                                 const float *area, const float *T, int J, float *M, cudaStream_t s);
tsr_status haar_forward(const float *X, int rows, int nu, float *Xw, cudaStream_t s);
// The same with input rows ldx apart (ldx >= 10 nu^2 + 2), e.g. one mesh of a batched M.
tsr_status haar_forward_ld(const float *X, long long ldx, int rows, int nu, float *Xw, cudaStream_t s);
// seg: optional caller buffer for the run approximations of charts of more than 1,024
// Morton positions (haar_inverse_seg_floats(rows, nu) floats); NULL takes stream-ordered scratch.
tsr_status haar_inverse(const float *Xw, int rows, int nu, float *X, cudaStream_t s, float *seg = nullptr);
size_t haar_inverse_seg_floats(int rows, int nu);
tsr_status cdf97_forward(const float *X, int rows, int nu, float *Xw, cudaStream_t s);
tsr_status cdf97_inverse(const float *Xw, int rows, int nu, float *X, cudaStream_t s);
tsr_status cdf97_inverse_transpose(const float *X, int rows, int nu, float *Xw, cudaStream_t s);
// The spatial transform of wavelet 0 (Haar) or 1 (CDF 9/7): analysis, synthesis, and the
// transpose of the synthesis (for the orthonormal Haar, the analysis).
tsr_status fresnel_output(int E, const double *eta, int N, const float *cos_o, const float *B, float *Bout,
                          cudaStream_t s);
tsr_status fresnel_output_backward(int E, const double *eta, int N, const float *cos_o, const float *B,
                                   const float *dBout, float *dB, float *deta, cudaStream_t s);
tsr_status sh_transfer(int N, const float *normals, int J, double eta, float *T, cudaStream_t s);
tsr_status visibility_transfer(int N, const float *pos, const float *normals, int F, const int *tris, int J, int S,
                               double eta, float eps, float *T, cudaStream_t s);
tsr_status spatial_forward(int wavelet, const float *X, int rows, int nu, float *Xw, cudaStream_t s);
tsr_status spatial_inverse(int wavelet, const float *Xw, int rows, int nu, float *X, cudaStream_t s,
                           float *seg = nullptr);
tsr_status spatial_inverse_transpose(int wavelet, const float *X, int rows, int nu, float *Xw, cudaStream_t s);
tsr_status wavelet_compress(const float *Mw, int K, int J, int nu, double p, tsr_compressed **out,
                            cudaStream_t s);
tsr_status wavelet_compress_into(const float *Mw, tsr_compressed *c, cudaStream_t s);
// Step 2 of n meshes whose columns of M start at M + offsets[b] (row stride offsets[n]): fill
// existing top-p Haar handles, or create and fill them.  One launch per stage and 32 meshes.
tsr_status haar_recompress_many(int n, const int64_t *offsets, const float *M, tsr_compressed *const *c,
                                cudaStream_t s);
tsr_status haar_compress_many(int n, const int64_t *offsets, const float *M, int K, int J, double p,
                              tsr_compressed **out, cudaStream_t s);
tsr_status wavelet_compress_energy(const float *Mw, int K, int J, int nu, double energy, tsr_compressed **out,
                                   cudaStream_t s);
tsr_status relight(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B,
                   cudaStream_t s);
tsr_status relight_backward(const tsr_compressed *c, int n_edit, const float *g, const float *l,
                            const float *dLdB, float *dg, float *dl, cudaStream_t s);
// Floats of caller-provided scratch relight_with_scratch needs: the intermediates Y and Z
// (K (10 P^2 + 2 + N)) or b^w, plus the inverse Haar's run approximations.
size_t relight_scratch_floats(const tsr_compressed *c);
// Steps 4-5 for one or two edits with the product and the inverse Haar fused, over
// n compressed transfers (Haar, P <= 128, same K and J) in one launch per 32.
bool relight_fusable(const tsr_compressed *c, int n_edit);
tsr_status relight_fused(int n, const tsr_compressed *const *c, int n_edit, const float *const *gi, const float *l,
                         float *const *Bi, cudaStream_t s);
// The factorised relight over n copies (Haar, P <= 128, same K and J; any number of
// edits): the light-contracted basis images Z_i ([K][N_i]) in one fused pass per 32
// copies, then B_i[v] = sum_k g_i[v][k] Z_i[k] in one combine launch per 32 copies.
bool relight_fusable_basis(const tsr_compressed *c);
tsr_status relight_basis_images_many(int n, const tsr_compressed *const *c, const float *l, float *const *Zi,
                                     cudaStream_t s);
tsr_status relight_combine_many(int n, const float *const *Zi, const int *Ni, int K, int V, const float *const *gi,
                                float *const *Bi, cudaStream_t s);
tsr_status relight_with_scratch(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B,
                                float *scratch, cudaStream_t s);
}  // namespace tsr
