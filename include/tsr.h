/*
 * tsr.h -- C ABI of the GB300 translucent subsurface-transfer library (libtsr.so).
 *
 * The library computes the data-parallel path of "Real-time Rendering and
 * Editing of Scattering Effects for Translucent Objects" (Wang, Hua, Huo, Bao):
 *
 *   basis     f_k(r)        PCA of sampled dipole R_d            (Section 2.2, Eq. 4-5)
 *   project   g_k(theta)    projection of R_d onto f_k            (Section 2.2; rendering Step 3)
 *   transfer  M[k,j,o]    = sum_i A_i f_k(|x_o - x_i|) T[j,i]     (Section 3, Eq. 6-7; precompute Step 1)
 *   compress  wavelet of M over the surface charts + keep rule   (Section 3.2, Eq. 9-10; precompute Step 2)
 *   relight   B[e,c,o]    = W^-1 sum_kj g_k l_j M^w[k,j,.]        (Section 4, rendering Steps 3-5)
 *   adjoint   of relight and of the projection (for fitting materials)
 *
 * Conventions (all calls):
 *   - Every function is extern "C" and returns tsr_status (0 on success).  On
 *     failure tsr_last_error() returns a message for the calling thread.
 *   - Array arguments are DEVICE pointers owned by the caller unless stated
 *     otherwise; the library never frees them.  Layouts are row-major with the
 *     dimensions written in brackets, the last one contiguous.
 *   - Opaque handles (tsr_basis, tsr_compressed) own device memory that the
 *     library allocates at creation and frees in the matching _destroy call.
 *   - Calls that take a tsr_stream enqueue work on that CUDA stream
 *     (a cudaStream_t; NULL = legacy default stream) and return without
 *     waiting, unless the comment says the call synchronises.
 *   - Scratch memory some calls need is allocated stream-ordered
 *     (cudaMallocAsync / cudaFreeAsync) on the caller's stream.
 *   - Errors: TSR_ERR_INVALID_ARG for a bad size, a NULL or misaligned
 *     pointer; TSR_ERR_UNSUPPORTED when no sm_103 device is current or a size
 *     is beyond the compiled limits; TSR_ERR_CUDA for a CUDA runtime error;
 *     TSR_ERR_TIMEOUT when a kernel's bounded wait gave up (the kernel then
 *     returned early and its outputs are undefined); TSR_ERR_OOM when an
 *     allocation failed.  There is no CPU fallback.
 *
 * Limits: 1 <= K <= 16 basis functions, 1 <= J <= 32 light coefficients,
 * n_r = 16..4096 radius samples, 12 <= N vertices.  Compression and relight
 * need the chart layout N = 10 nu^2 + 2, 1 <= nu <= 256.
 */
#ifndef TSR_H
#define TSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int tsr_status;
#define TSR_OK 0
#define TSR_ERR_INVALID_ARG (-1)
#define TSR_ERR_CUDA (-2)
#define TSR_ERR_OOM (-3)
#define TSR_ERR_TIMEOUT (-4)
#define TSR_ERR_UNSUPPORTED (-5)

/* A CUDA stream handle (binary-compatible with cudaStream_t). */
typedef struct CUstream_st *tsr_stream;

/* Arithmetic of the transfer contraction. */
typedef enum {
  TSR_FP32 = 0,   /* CUDA-core FP32 products, FP32 compensated accumulation        */
  TSR_BF16 = 1,   /* tcgen05 tensor cores: BF16 f_k and T', FP32 accumulation in TMEM */
  TSR_BF16X3 = 2  /* split BF16: hi*hi + hi*lo + lo*hi tensor-core products, FP32 accumulation */
} tsr_precision;

typedef struct tsr_basis tsr_basis;
typedef struct tsr_compressed tsr_compressed;

/* Thread-local message of the last failed call ("" if none). */
const char *tsr_last_error(void);

/* Library ABI version (major*100 + minor). */
int tsr_version(void);

/* Number of kernel launches the library has made in this process (all
 * threads and devices); a diagnostic for counting launches in a region. */
uint64_t tsr_kernel_launches(void);

/* Device timing of the transfer's tensor-core kernel, for measurement: while
 * enabled (enable = 1), every launch of that kernel is bracketed by two CUDA
 * events on its stream.  tsr_kernel_timing_read synchronises on the recorded
 * events, returns the sum of their elapsed times (ms) and their number, and
 * releases them.  Enable it only outside stream capture. */
tsr_status tsr_kernel_timing(int enable);
tsr_status tsr_kernel_timing_read(double *total_ms, int *launches);

/* Diagnostic of the failure path: launches one block that waits, with at most
 * `limit` (1..1e6) polls, on an mbarrier phase that nothing completes.  The
 * wait gives up, the kernel records a timeout in the device status word and
 * returns; the following tsr_stream_status reports TSR_ERR_TIMEOUT and the
 * context stays usable.  The same bounded waits guard every pipeline barrier
 * of the transfer kernels. */
tsr_status tsr_selftest_bounded_wait(unsigned limit, tsr_stream stream);

/* Synchronises the stream, then reports whether any library kernel since the
 * last check gave up a bounded wait (TSR_ERR_TIMEOUT) or flagged an
 * out-of-range access (TSR_ERR_CUDA); also returns the stream's own CUDA
 * error, if any.  The device status word is cleared. */
tsr_status tsr_stream_status(tsr_stream stream);

/* Host-side fault injection, for testing a caller's error handling without
 * faulting a GPU (the paper has no counterpart).  The next n occurrences of a
 * kind fail as if the underlying call had failed (n = 0 clears; process-wide):
 *   TSR_FAULT_ALLOC   (1): stream-ordered scratch allocations -> TSR_ERR_OOM;
 *   TSR_FAULT_CUDA    (2): checked CUDA runtime calls (launch checks, copies,
 *                          allocations) -> TSR_ERR_CUDA; the call itself ran;
 *   TSR_FAULT_TIMEOUT (3): tsr_stream_status -> TSR_ERR_TIMEOUT, as if a kernel's
 *                          bounded wait had run out.
 * An injected failure leaves the call's outputs undefined, as a real one would.
 * TSR_ERR_INVALID_ARG for an unknown kind or n outside [0, 2^20]. */
#define TSR_FAULT_ALLOC 1
#define TSR_FAULT_CUDA 2
#define TSR_FAULT_TIMEOUT 3
tsr_status tsr_fault_inject(int kind, int n);

/* ------------------------------------------------------------------------
 * Basis (Section 2.2, Eq. 5).
 *
 * tsr_fit_pca_basis: samples the dipole R_d of Eq. 4 for n_mat materials
 * (sigma_a[s], sigma_s[s] in 1/mm, common index eta) at n_r radii
 * r_m = r_max * m / (n_r - 1) (mm), forms R[s][m], computes its singular
 * value decomposition R = U S V^T in FP64 on the device (one-sided Jacobi) and
 * keeps the first K right singular vectors as the radial basis f_k (each
 * flipped so that its largest-magnitude sample is positive).
 *   sigma_a, sigma_s : device [n_mat] FP64, > 0.  2 <= n_mat <= 1024.
 *   eta              : 1.0 <= eta <= 2.0 (the F_dr fit of Section 2.1).
 *   sing_vals        : device [min(n_mat, n_r)] FP64 out, descending; may be NULL.
 *   out              : receives a new handle (destroy with tsr_basis_destroy).
 * The call synchronises the stream (it is a one-time set-up step).
 *
 * tsr_basis_create: builds a handle from a caller table f[K][n_r] (FP64,
 * HOST pointer) sampled on the same grid, e.g. a stored basis.
 *
 * tsr_basis_table: copies f[K][n_r] (FP64) to a device buffer.
 * tsr_basis_info: K, n_r and r_max of a handle (host out-pointers, any may be NULL).
 * tsr_basis_far_series: the far-field series the BF16 transfer evaluates
 *   instead of the table (Section 3, Eq. 6-7; see tsr_precompute_transfer):
 *   *rel_err = max_k max over r in [r_max / 16, r_max] of
 *   |sum_{p<12} c_kp T_p(x(r)) - r^2 f_k(r)| / max_r |r^2 f_k(r)|, computed on the
 *   device when the handle was made; *used = 1 when rel_err <= 2e-3 (the BF16
 *   transfer then uses the series, else the table).  Out-pointers may be NULL.
 * ---------------------------------------------------------------------- */
tsr_status tsr_fit_pca_basis(int n_mat, const double *sigma_a, const double *sigma_s, double eta,
                             int n_r, double r_max, int K, double *sing_vals, tsr_basis **out,
                             tsr_stream stream);
tsr_status tsr_basis_create(int K, int n_r, double r_max, const double *f_host, tsr_basis **out);
tsr_status tsr_basis_table(const tsr_basis *basis, double *f, tsr_stream stream);
tsr_status tsr_basis_info(const tsr_basis *basis, int *K, int *n_r, double *r_max);
tsr_status tsr_basis_far_series(const tsr_basis *basis, double *rel_err, int *used);
void tsr_basis_destroy(tsr_basis *basis);

/* ------------------------------------------------------------------------
 * Material projection (Section 2.2 "projected onto the basis"; rendering
 * Step 3):  g[e][c][k] = sum_m f_k(r_m) R_d(r_m; sigma_a[e][c], sigma_s[e][c], eta[e])
 * in FP64, for n edits and the 3 colour channels c.
 *   sigma_a, sigma_s : device [n][3] FP64 (1/mm, > 0);  eta: device [n] FP64 in [1, 2].
 *   g                : device [n][3][K] FP64 out.
 *   g32              : device [n][3][K] FP32 out (same values rounded); may be NULL.
 *   dg               : device [n][3][K][3] FP64 out, the Jacobian
 *                      (dg/dsigma_a, dg/dsigma_s, dg/deta) from the analytic
 *                      derivative of Eq. 4; may be NULL.
 *
 * tsr_project_material_backward: vector-Jacobian product of the projection.
 *   dLdg : device [n][3][K] FP32;  dsigma_a, dsigma_s: device [n][3] FP32 out;
 *   deta : device [n] FP32 out.  Exactly overwrites the outputs.
 * ---------------------------------------------------------------------- */
tsr_status tsr_project_material(const tsr_basis *basis, int n, const double *sigma_a,
                                const double *sigma_s, const double *eta, double *g, float *g32,
                                double *dg, tsr_stream stream);
tsr_status tsr_project_material_backward(const tsr_basis *basis, int n, const double *sigma_a,
                                         const double *sigma_s, const double *eta, const float *dLdg,
                                         float *dsigma_a, float *dsigma_s, float *deta,
                                         tsr_stream stream);

/* ------------------------------------------------------------------------
 * Transfer (Section 3, Eq. 6-7; precompute Step 1):
 *   M[k][j][o] = sum_{i<N} A_i f_k(|x_o - x_i|) T[j][i]
 * with f_k piecewise linear on the basis grid and zero where the FP32
 * squared distance fl(fl(fl(dx^2)+fl(dy^2))+fl(dz^2)) exceeds r_max^2
 * (dx = fl(x_o - x_i)); the self pair i = o is included.
 *   pos  : device [3][N] FP32 (x, then y, then z; mm), 16-byte aligned.
 *   area : device [N] FP32 (mm^2).
 *   T    : device [J][N] FP32.
 *   M    : device [K][J][N] FP32 out (overwritten).
 *   prec : TSR_FP32, TSR_BF16 or TSR_BF16X3.
 * Precisions:
 *   TSR_FP32   CUDA cores, FP32 table of f_k, Kahan-compensated sums.
 *   TSR_BF16   tensor cores (BF16 x BF16 -> FP32) for the far pairs, those with
 *              r^2 >= r_e^2, r_e = max(r_max / 16, 2 h), h^2 = sum(A)/N; the near
 *              pairs r^2 < r_e^2 (the self pair among them) are summed exactly in
 *              FP32 and added.  The far kernel values come from the 12-term
 *              series f_k(r) = sum_p c_kp T_p(x) / r^2 (x linear in log r on
 *              [r_max / 16, r_max]) when tsr_basis_far_series reports it accurate,
 *              else from the BF16 table.
 *   TSR_BF16X3 split BF16 (hi + lo of both operands, three products) for every
 *              pair from the table, the self pair replaced in FP32.
 * Scratch: a pre-tiled copy of (x_i, A_i T[.,i]), about N*(2*J_pad*2+12) bytes,
 * and for TSR_BF16 the Morton-sorted copy of the inputs the near field reads,
 * about N*(4*J_pad+40) bytes (stream-ordered, freed by the call).
 * Errors: TSR_ERR_INVALID_ARG for NULL or misaligned pointers or N, J out of
 * range; TSR_ERR_OOM when scratch cannot be allocated; nothing is launched then.
 * ---------------------------------------------------------------------- */
tsr_status tsr_precompute_transfer(const tsr_basis *basis, int N, const float *pos, const float *area,
                                   const float *T, int J, tsr_precision prec, float *M,
                                   tsr_stream stream);

/* Batched transfer over n_mesh independent meshes of uneven size (Eq. 6-7 per
 * mesh; pairs never cross meshes).  All arrays are concatenated over the meshes:
 *   offsets : HOST [n_mesh + 1] int64 vertex offsets (offsets[0] = 0; 12 <= each mesh <= 2^24).
 *   pos     : device [3][total] FP32;  area: device [total];  T: device [J][total];
 *   M       : device [K][J][total] FP32 out.  Only TSR_BF16 and TSR_FP32.
 * TSR_BF16 runs one persistent launch over the (mesh, 128-row tile) units in
 * longest-first order; TSR_FP32 runs one launch per mesh.
 *
 * tsr_precompute_transfer_batched synchronises the stream (it builds and frees
 * a plan).  For repeated or graph-captured use, build a plan once:
 *   tsr_batch_plan_create   uploads the unit and mesh tables (synchronous);
 *   tsr_batch_plan_autotune times each generator configuration of the BF16
 *                           transfer (the far-field series with three or two
 *                           16-i steps in flight, and one at J <= 16; the table
 *                           with 4, 8, 12 or 16 bases
 *                           per CTA group) on the caller's data, keeps the
 *                           fastest, returns its time in *best_ms (synchronises;
 *                           outside any capture);
 *   tsr_precompute_transfer_plan enqueues the transfer only (kernels and
 *                           stream-ordered scratch), so it may be captured in a
 *                           CUDA graph;
 *   tsr_batch_plan_info     units, the chosen generator (0: far-field series,
 *                           1: table) and its parameter (steps in flight, or
 *                           bases per group; 0 = default);
 *   tsr_batch_plan_destroy. */
tsr_status tsr_precompute_transfer_batched(const tsr_basis *basis, int n_mesh, const int64_t *offsets,
                                           const float *pos, const float *area, const float *T, int J,
                                           tsr_precision prec, float *M, tsr_stream stream);
typedef struct tsr_batch_plan tsr_batch_plan;
tsr_status tsr_batch_plan_create(const tsr_basis *basis, int n_mesh, const int64_t *offsets, int J,
                                 tsr_precision prec, tsr_batch_plan **out);
tsr_status tsr_batch_plan_autotune(tsr_batch_plan *plan, const float *pos, const float *area, const float *T,
                                   float *M, tsr_stream stream, float *best_ms);
tsr_status tsr_precompute_transfer_plan(const tsr_batch_plan *plan, const float *pos, const float *area,
                                        const float *T, float *M, tsr_stream stream);
tsr_status tsr_batch_plan_info(const tsr_batch_plan *plan, int *n_units, int *generator, int *param);
void tsr_batch_plan_destroy(tsr_batch_plan *plan);

/* ------------------------------------------------------------------------
 * Spatial wavelet (Section 3.2, Eq. 9-10).  Vertex data of the chart mesh
 * (N = 10 nu^2 + 2; chart d row r col c has id d nu^2 + r nu + c, poles last)
 * is put in Morton order per chart, zero-padded to P x P (P = 2^ceil(log2 nu)),
 * and transformed by the orthonormal 1D Haar (output order: scaling, then
 * details coarse to fine).  The wavelet layout is [10 P^2 + 2]: chart d at
 * [d P^2, (d+1) P^2), the two pole values last (passed through).
 *
 * tsr_haar_forward:  X [rows][N] FP32 -> Xw [rows][10 P^2 + 2] FP32.
 * tsr_haar_inverse:  Xw [rows][10 P^2 + 2] -> X [rows][N] (padding dropped).
 * ---------------------------------------------------------------------- */
tsr_status tsr_haar_forward(const float *X, int rows, int nu, float *Xw, tsr_stream stream);
tsr_status tsr_haar_inverse(const float *Xw, int rows, int nu, float *X, tsr_stream stream);

/* ------------------------------------------------------------------------
 * Compression (precompute Step 2, Section 3.2).
 * tsr_wavelet_compress: from wavelet coefficients Mw [K][J][10 P^2 + 2] keeps,
 * per (k, j), the n_keep = floor(p * 10 P^2 + 0.5) (clamped to [1, 10 P^2])
 * chart coefficients of largest |value| (ties: lower index) plus both poles,
 * and packs them as a CSR matrix over wavelet rows w (entries: column
 * kj = k*J + j as uint16, value FP32, columns ascending within a row).
 * tsr_haar_compress = tsr_haar_forward of M followed by tsr_wavelet_compress.
 * The packed size is known in advance (K*J*(n_keep + 2) entries), so the
 * handle's arrays are allocated at creation (cudaMalloc) and filled on the
 * stream without synchronising.
 * tsr_haar_recompress re-runs tsr_haar_compress for a new M [K][J][N] into an
 * existing handle (same K, J, nu and keep rule): no device allocation other
 * than stream-ordered scratch, so it suits a per-frame or per-step loop.
 * ---------------------------------------------------------------------- */
tsr_status tsr_wavelet_compress(const float *Mw, int K, int J, int nu, double p, tsr_compressed **out,
                                tsr_stream stream);
tsr_status tsr_haar_compress(const float *M, int K, int J, int nu, double p, tsr_compressed **out,
                             tsr_stream stream);
tsr_status tsr_haar_recompress(const float *M, tsr_compressed *c, tsr_stream stream);
/* Step 2 (Section 3, Eq. 9-10) for every mesh of a batched transfer: M is the
 * device [K][J][total] output of tsr_precompute_transfer_batched (mesh b's
 * values at columns offsets[b] .. offsets[b+1]-1 of every (k, j) row, read in
 * place with row stride total); offsets: HOST [n_mesh + 1] int64, each mesh
 * 10 nu^2 + 2 vertices (nu <= 128).  Per mesh: the Haar analysis of its rows and
 * the top-fraction selection of tsr_haar_compress (the same kernels' work, so each
 * handle is bit-identical to compressing its mesh alone), in one launch per stage
 * (Haar, top levels, selection, row counts, scan, packing) and group of 32 meshes
 * (stream-ordered scratch of the group: about 5 K J (10 P^2 + 2) bytes per mesh).  All
 * handles share K and J.
 *   tsr_haar_compress_batched   creates the n_mesh handles in out (HOST array;
 *                               allocates device memory, synchronises); on error
 *                               none is left (out[b] = NULL).
 *   tsr_haar_recompress_batched refills them for a new M (Haar top-fraction
 *                               handles whose nu matches each mesh); stream-ordered
 *                               scratch only, so it may be captured in a CUDA graph.
 * TSR_ERR_INVALID_ARG for NULL pointers, a mesh size not of the chart form, or a
 * handle that does not fit its mesh. */
tsr_status tsr_haar_compress_batched(int n_mesh, const int64_t *offsets, const float *M, int K, int J, double p,
                                     tsr_compressed **out, tsr_stream stream);
tsr_status tsr_haar_recompress_batched(int n_mesh, const int64_t *offsets, const float *M,
                                       tsr_compressed *const *c, tsr_stream stream);
/* The paper's Step-2 wavelet (Section 5, "Daubechies 9/7"): the CDF 9/7
 * biorthogonal pair by lifting (whole-sample symmetric extension, low band DC
 * gain sqrt 2), as the separable 2D Mallat pyramid of each chart's P x P image
 * (row-major, pixel (r, c) = vertex d nu^2 + r nu + c, zero padding), every level
 * transforming the rows, then the columns, of the low-low band down to 1 x 1;
 * chart d's coefficients at [d P^2, (d+1) P^2), the poles last.  Same shapes as
 * tsr_haar_forward / tsr_haar_inverse.  tsr_cdf97_inverse_transpose applies the
 * transpose of the synthesis (the reverse mode of the relight; for this
 * biorthogonal pair it differs from the analysis). */
tsr_status tsr_cdf97_forward(const float *X, int rows, int nu, float *Xw, tsr_stream stream);
tsr_status tsr_cdf97_inverse(const float *Xw, int rows, int nu, float *X, tsr_stream stream);
tsr_status tsr_cdf97_inverse_transpose(const float *X, int rows, int nu, float *Xw, tsr_stream stream);

#define TSR_WAVELET_HAAR 0
#define TSR_WAVELET_CDF97 1
#define TSR_KEEP_TOP_FRACTION 0
#define TSR_KEEP_ENERGY 1
/* Step 2 with either spatial wavelet and either keep rule: tsr_haar_compress is
 * (TSR_WAVELET_HAAR, TSR_KEEP_TOP_FRACTION, p), tsr_haar_compress_energy is
 * (TSR_WAVELET_HAAR, TSR_KEEP_ENERGY, energy).  The handle remembers its wavelet:
 * tsr_relight and tsr_relight_backward invert (and transpose) the right one, and
 * tsr_haar_recompress re-applies it (top-fraction handles only). */
tsr_status tsr_compress(const float *M, int K, int J, int nu, int wavelet, int rule, double param,
                        tsr_compressed **out, tsr_stream stream);

/* Step 2 with the paper's energy threshold (Section 3, precompute Step 2: "the
 * reserved energy exceeds the threshold"; 95-98 % in its results): per (k, j)
 * the smallest n >= 1 such that the n largest |c| of the chart coefficients
 * (ties: lower index) hold at least `energy` of the row's energy sum c^2 (FP64);
 * both poles always kept and not counted.  energy in (0, 1].  The number kept
 * varies per (k, j); the call reads those counts back (one synchronisation of
 * `stream`) to size the handle.  tsr_haar_recompress does not apply to such a
 * handle (TSR_ERR_UNSUPPORTED). */
tsr_status tsr_haar_compress_energy(const float *M, int K, int J, int nu, double energy, tsr_compressed **out,
                                    tsr_stream stream);
/* Sizes of a compressed transfer (host out-pointers, any may be NULL). */
tsr_status tsr_compressed_info(const tsr_compressed *c, int *K, int *J, int *nu, int64_t *nnz,
                               int *n_rows);
/* Copies the CSR arrays to caller device buffers: row_ptr [n_rows+1] int64,
 * col [nnz] uint16, val [nnz] FP32. */
tsr_status tsr_compressed_export(const tsr_compressed *c, int64_t *row_ptr, uint16_t *col, float *val,
                                 tsr_stream stream);
void tsr_compressed_destroy(tsr_compressed *c);

/* Checkpoint and resume of the precompute's result (the paper has no
 * counterpart): tsr_compressed_save writes the handle to a file (synchronous
 * device-to-host copies; little-endian binary: an 8-byte magic "TSRCMP01", the
 * int32 fields K, J, nu, P, n_rows, n_keep, keep rule, wavelet, the int64 nnz,
 * then row_ptr, col, val, the column lists and col_ptr); tsr_compressed_load
 * reads one back into a new handle on the current device, equal to the saved one
 * for every call.  TSR_ERR_INVALID_ARG, with nothing allocated, for a file that
 * cannot be opened, is not such a file, is truncated, or whose header, pointers
 * or indices are out of range (all checked on the host before any device work). */
tsr_status tsr_compressed_save(const tsr_compressed *c, const char *path);
tsr_status tsr_compressed_load(const char *path, tsr_compressed **out);

/* ------------------------------------------------------------------------
 * Fresnel transmittance factors of Eq. 3 and Eq. 6,
 *   S = (1/pi) F_t(eta, w_i) R_d F_t(eta, w_o),
 * F_t(eta, mu) = 1 - (r_s^2 + r_p^2)/2, the exact unpolarised dielectric Fresnel
 * reflectance for a direction at cosine mu > 0 outside (0 for mu <= 0).
 * tsr_fresnel_output: Bout[e][c][o] = (1/pi) F_t(eta[e], cos_o[o]) B[e][c][o]
 *   (eta: device [n_edit] FP64; cos_o: device [N] FP32, the caller's n_o . w_o per
 *   output vertex; B, Bout: device [n_edit][3][N] FP32, may alias).
 * tsr_fresnel_output_backward: dB = (1/pi) F_t dBout and
 *   deta[e] = sum_{c,o} dBout B (1/pi) dF_t/deta (device [n_edit] FP32, overwritten).
 * tsr_sh_transfer: the unshadowed SH irradiance transfer with the incident F_t
 *   folded in, T[j][i] = A_l(eta) Y_lm(n_i) (real orthonormal SH, j = l^2 + l + m,
 *   no Condon-Shortley phase), A_l(eta) = 2 pi int_0^1 F_t(eta, mu) mu P_l(mu) dmu
 *   (Funk-Hecke; eta = 1 gives the clamped cosine pi, 2pi/3, pi/4, 0, -pi/24).
 *   normals: device [3][N] FP32 unit vectors; J in {1, 4, 9, 16, 25}; eta in
 *   [1, 2]; T: device [J][N] FP32 out.
 * ---------------------------------------------------------------------- */
tsr_status tsr_fresnel_output(int n_edit, const double *eta, int N, const float *cos_o, const float *B, float *Bout,
                              tsr_stream stream);
tsr_status tsr_fresnel_output_backward(int n_edit, const double *eta, int N, const float *cos_o, const float *B,
                                       const float *dBout, float *dB, float *deta, tsr_stream stream);
tsr_status tsr_sh_transfer(int N, const float *normals, int J, double eta, float *T, tsr_stream stream);

/* Self-shadowed SH irradiance transfer (E of Eq. 6 with the visibility of the
 * transfer, E11-E14) for displaced meshes:
 *   T[j][i] = (pi / S) sum_s Y_j(w_s) V(x_i, w_s) [F_t(eta, mu_s)],
 * w_s the S cosine-weighted Hammersley directions (u1 = (s + 1/2)/S, u2 = the
 * bit-reversed s; r = sqrt u1, phi = 2 pi u2, mu = sqrt(1 - u1)) in the frame of n_i
 * (Duff et al. 2017), rays from x_i + eps n_i, V = 0 if a ray hits any triangle
 * (FP32 Moller-Trumbore, t > 1e-4).  A linear BVH is built on the device per call.
 *   pos, normals: device [3][N] FP32; tris: device [F][3] int32 vertex indices;
 *   J in {1, 4, 9, 16, 25}; S in [1, 65536]; eta = 0 (no Fresnel factor) or in
 *   [1, 2]; T: device [J][N] FP32 out. */
tsr_status tsr_visibility_transfer(int N, const float *pos, const float *normals, int F, const int32_t *tris, int J,
                                   int S, double eta, float eps, float *T, tsr_stream stream);

/* ------------------------------------------------------------------------
 * Relight / material edit (Section 4, rendering Steps 3-5):
 *   b^w[e][c][w] = sum_{(kj,v) in row w} v * g[e][c][k] * l[j]
 *   B[e][c][.]   = W^-1 b^w[e][c][.]         (inverse Haar per chart)
 *   g : device [n_edit][3][K] FP32;  l: device [J] FP32 (one light for all edits);
 *   B : device [n_edit][3][N] FP32 out.
 * For n_edit > 2 it is evaluated with the light contracted first (the same B
 * by linearity):
 *   Y[k][w] = sum_j S[w][kj] l[j],  Z[k] = W^-1 Y[k],  B[e][c] = sum_k g[e][c][k] Z[k],
 * so the kept coefficients are read once per call, whatever n_edit; for one or
 * two edits as written (one pass over S for their 3 or 6 vectors; under the
 * Haar (every chart the library accepts) the product and the inverse Haar run fused per chart run
 * without scratch).
 * Scratch: max(K*(10 P^2 + 2 + N), 6*(10 P^2 + 2)) FP32.
 *
 * tsr_relight_backward: reverse mode for an upstream gradient dLdB
 * [n_edit][3][N] (r^w = W dLdB, dc = S^T r^w, dg = sum_j l_j dc, dl = sum g dc),
 * evaluated as
 *   dg[e][c][k] = <dLdB[e][c], Z[k]>,
 *   dl[j] = sum_k sum_w S[w][kj] (W Q[k])[w],  Q[k] = sum_{e,c} g[e][c][k] dLdB[e][c].
 *   dg : device [n_edit][3][K] FP32 out;  dl: device [J] FP32 out (overwritten).
 * ---------------------------------------------------------------------- */
tsr_status tsr_relight(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B,
                       tsr_stream stream);
tsr_status tsr_relight_backward(const tsr_compressed *c, int n_edit, const float *g, const float *l,
                                const float *dLdB, float *dg, float *dl, tsr_stream stream);

/* ------------------------------------------------------------------------
 * tsr_relight_many: Steps 4-5 (Section 4) for n_copy compressed transfers at
 * once -- the objects of a scene, or the pieces of a frame too large for one
 * mesh -- each relit under its own edits and one shared light.
 *   c      : HOST array [n_copy] of handles (0 <= n_copy <= 65536), all with
 *            the same K and J, on the current device;
 *   n_edit : edits per copy (0 <= n_edit <= 2^20);
 *   g      : device [n_copy][n_edit][3][K] FP32;  l: device [J] FP32;
 *   B      : device FP32 out, the copies' [n_edit][3][N_i] blocks back to back
 *            (copy i starts at n_edit * 3 * (N_0 + ... + N_{i-1}), N_i = 10 nu_i^2 + 2).
 * Result per copy: tsr_relight of that copy (FP32 sums in another order for
 * more than two edits).  Copies under the orthonormal Haar go through fused
 * kernels, 32 copies per launch: with one or two edits b^w = S c and the inverse
 * Haar per chart run in shared memory (no scratch); with more, the
 * light-contracted basis images Z[k] = W^-1 (S (e_k x l)) of every copy in one
 * such pass, then B = sum_k g_k Z[k] for all copies and edits in one launch
 * (stream-ordered scratch K (N_0 + ... ) floats).  CDF 9/7 copies run
 * tsr_relight copy by copy.
 * Errors: TSR_ERR_INVALID_ARG for NULL or misaligned pointers, a NULL handle or
 * handles whose K or J differ from the first one's; nothing is launched then.
 * ---------------------------------------------------------------------- */
tsr_status tsr_relight_many(int n_copy, const tsr_compressed *const *c, int n_edit, const float *g, const float *l,
                            float *B, tsr_stream stream);

/* ------------------------------------------------------------------------
 * tsr_relight_noalloc: tsr_relight for callers that cannot allocate device
 * memory (a host that owns every device allocation and forbids new ones after
 * start-up, or a frame loop that may not issue an allocation call).  The paper
 * has no counterpart; this is a property of the library, not of the method.
 * Same arguments, layouts and result as tsr_relight.  Its intermediate buffer
 * comes from a fixed 32 MiB array of device memory that the library reserves on
 * every GPU where it is loaded (held until the process exits), so the call
 * itself allocates nothing (the array also holds the run approximations that
 * the inverse Haar of charts larger than 32 x 32 needs).
 *   - Limit: the scratch above <= 8,388,608 floats, else TSR_ERR_INVALID_ARG
 *     (the largest case the library accepts, K = 16 on nu = 128, needs 5.2 Mi;
 *     the number of edits does not enter).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls on a device share the one array: calls whose kernels overlap
 *     on the GPU (other streams, other threads) race and give wrong results.
 *     Serialise them, e.g. on one stream.
 * ---------------------------------------------------------------------- */
tsr_status tsr_relight_noalloc(const tsr_compressed *c, int n_edit, const float *g, const float *l, float *B,
                               tsr_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* TSR_H */
