// Section 4, rendering Steps 4-5 for one or two edits, fused: the sparse product
// b^w = S c and the inverse Haar B = w_1^{-1} b^w in one kernel, over one or many
// compressed transfers (the objects of a scene, or the copies that make up a
// large frame) in one launch.
//
// The inverse Haar of a chart (Section 3.2, Eq. 9-10) splits into independent
// runs of RF_SEG Morton positions once the approximation of each run is known,
// and that approximation depends only on the chart's scaling coefficient and the
// one detail per coarse level on the run's path to the root.  So a block owns a
// (copy, chart, run): it computes b^w for the 1 + log2(runs per chart) path rows
// and the RF_SEG - 1 detail rows of its run into shared memory, then each output
// value is synthesised by walking down the tree from the chart's scaling
// coefficient, and scattered to its vertex.  b^w never reaches global memory and
// the kept coefficients are read once (the few path rows are re-read from L2 by
// the runs of a chart).
//
// Fixed-order arithmetic (results do not depend on scheduling): a row's sum is
// formed by one 8-lane group, lane sub adding the entries of its groups of 4
// (sub, sub + 8, ...) in order, the 8 partial sums meeting in xor-shuffles 4, 2,
// 1; each synthesis step is (a + d) / sqrt2 or (a - d) / sqrt2, as in the
// level-by-level inverse.
//
// With g = identity the same kernel yields the light-contracted basis images
// Z[k] = w_1^{-1} (S (e_k x l)) (K "vectors"); the relight of many edits on many
// copies is then those images plus relight_combine_many_kernel, B = sum_k g_k Z[k].
#include <algorithm>
#include <atomic>

#include "handles.cuh"

namespace tsr {

constexpr int RF_THREADS = 256;
constexpr int RF_LPR = 8;                                  // lanes per wavelet row
constexpr int RF_SEG = 1024;                               // Morton positions per run
constexpr int RF_MAX_LGN = 4;                              // up to 16 runs per chart (P <= 128, the library's nu <= 128)
constexpr int RF_MAX_TOP = 1 + RF_MAX_LGN;                 // path rows
constexpr int RF_MAX_ROWS = RF_MAX_TOP + RF_SEG - 1 + 2;   // + run details + the two poles
constexpr int RF_MAXC = 32;                                // copies per launch (kernel parameter space)

struct RelightCopy {
  const int64_t *row_ptr;
  const uint16_t *col;
  const float *val;
  const float *g;   // [VV][K]
  float *B;         // [VV][10 nu^2 + 2]
  int nu, lgP;      // chart side P = 2^lgP
  int item0;        // first work item (chart-run) of this copy
};

struct RelightBatch {
  RelightCopy c[RF_MAXC];
  int n;
  int nv;   // output rows written per copy (the kernel's VV, or K in basis-image mode)
};

__device__ __forceinline__ unsigned rf_compact(unsigned x) {   // even bits of x, packed
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  x = (x | (x >> 8)) & 0x0000FFFFu;
  return x;
}
__device__ __forceinline__ unsigned rf_spread(unsigned x) {    // inverse of rf_compact
  x &= 0x0000FFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// b^w of local row q into its place: path rows and poles in `top`, run details in x.
template <int VV>
__device__ __forceinline__ void rf_store(float (*x)[RF_SEG], float (*top)[RF_MAX_TOP + 2], int q, int T, int R, int v,
                                         float b) {
  if (q < T)
    top[v][q] = b;
  else if (q < R)
    x[v][q - T + 1] = b;
  else
    top[v][RF_MAX_TOP + q - R] = b;
}

// Row of the c table holding column kj: bits 3-4 of kj flip bits 0-1, so the
// columns kj, kj + 4, ..., kj + 28 that the 8 lanes of a group read together (they
// walk groups of 4 entries) fall in different 16-byte bank groups.  A bijection on
// each aligned block of 32 columns.
__device__ __forceinline__ int rf_crow(int kj) { return kj ^ ((kj >> 3) & 3); }

// c_v[kj] for one entry, VV of them from the padded row (float4 loads); one FMA
// per vector and entry.
template <int VV>
__device__ __forceinline__ void rf_fma(const float4 *cs4, int kj, float a, float (&acc)[VV]) {
  constexpr int VQ = (VV + 3) / 4;
  kj = rf_crow(kj);
#pragma unroll
  for (int h = 0; h < VQ; ++h) {
    const float4 c = cs4[kj * VQ + h];
    const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (4 * h + e < VV) acc[4 * h + e] = fmaf(a, cv[e], acc[4 * h + e]);
  }
}

template <int VV>
__global__ void __launch_bounds__(RF_THREADS, VV <= 6 ? 5 : 2) relight_fused_kernel(const __grid_constant__ RelightBatch bt, int K,
                                                                  int J, const float *__restrict__ l) {
  constexpr int VQ = (VV + 3) / 4;   // float4s per c row
  constexpr bool XDYN = VV > 6;      // x in dynamic shared memory (above 24 KB)
  // Non-empty rows of the block: {first entry - e0, q << 16 | entries}.
  __shared__ int2 lst[RF_MAX_ROWS];
  __shared__ __align__(16) float xs[XDYN ? 1 : VV][RF_SEG];
  __shared__ float top[VV][RF_MAX_TOP + 2];   // path rows, then the poles
  __shared__ int n_rows_ne;
  // dynamic: [x: VV][RF_SEG] floats when XDYN, then the c table
  // [K J rounded up to 32][VQ] float4: c_v[kj] = g_v[k] l[j] at row rf_crow(kj)
  extern __shared__ float4 dyn4[];
  float (*x)[RF_SEG] = XDYN ? reinterpret_cast<float (*)[RF_SEG]>(dyn4) : xs;
  float4 *cs4 = dyn4 + (XDYN ? VV * RF_SEG / 4 : 0);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int ci = 0;
  while (ci + 1 < bt.n && bt.c[ci + 1].item0 <= (int)blockIdx.x) ++ci;
  const RelightCopy &cp = bt.c[ci];
  const int nu = cp.nu, lgP = cp.lgP;
  const int lgP2 = 2 * lgP, P2 = 1 << lgP2;
  const int lgL = min(lgP2, 10), L = 1 << lgL;
  const int lgn = lgP2 - lgL;   // log2(runs per chart)
  const int local = (int)blockIdx.x - cp.item0;
  const int d = local >> lgn, s = local & ((1 << lgn) - 1);
  const int T = 1 + lgn;        // path rows
  const int R = T + L - 1;
  const bool poles = (d == 0 && s == 0);
  const int R_tot = R + (poles ? 2 : 0);
  const int64_t wbase = (int64_t)d * P2;
  const float *__restrict__ val = cp.val;
  const uint16_t *__restrict__ col = cp.col;
  const int64_t *__restrict__ row_ptr = cp.row_ptr;
  const int64_t e0 = row_ptr[wbase];   // entries of the block's rows lie in [e0, e0 + 2^31 - 4)

  // Empty rows contribute zeros.
  for (int q = tid; q < VV * RF_SEG / 4; q += RF_THREADS)
    reinterpret_cast<float4 *>(&x[0][0])[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (tid < VV * (RF_MAX_TOP + 2)) (&top[0][0])[tid] = 0.0f;
  if (tid == 0) n_rows_ne = 0;
  const int KJ = K * J;
  for (int q = tid; q < KJ; q += RF_THREADS) {
    const int k = q / J;
    const float lj = l[q - k * J];
    float c[4 * VQ];
#pragma unroll
    for (int v = 0; v < 4 * VQ; ++v)   // basis-image mode (no g): c_v[kj] = l[j] for v = k, else 0
      c[v] = v < VV ? (cp.g ? cp.g[v * K + k] : (v == k ? 1.0f : 0.0f)) * lj : 0.0f;
#pragma unroll
    for (int h = 0; h < VQ; ++h)
      cs4[rf_crow(q) * VQ + h] = make_float4(c[4 * h], c[4 * h + 1], c[4 * h + 2], c[4 * h + 3]);
  }
  __syncthreads();

  // The non-empty rows (warp-aggregated appends: each warp appends its 32 consecutive
  // rows in order, so rows of similar length sit together; the order does not change
  // any sum, each row being reduced by one lane group in a fixed order).
  constexpr int SQ = (RF_MAX_ROWS + RF_THREADS - 1) / RF_THREADS;
  int64_t pa[SQ], pb[SQ];
#pragma unroll
  for (int i = 0; i < SQ; ++i) {   // every row pointer of the thread's rows in flight at once
    const int q = warp * 32 + RF_THREADS * i + lane;
    pa[i] = pb[i] = 0;
    if (q < R_tot) {
      int64_t w;
      if (q == 0) {
        w = wbase;
      } else if (q < T) {
        const int lv = q - 1;   // level with 2^lv approximations
        w = wbase + (1 << lv) + (s >> (lgn - lv));
      } else if (q < R) {
        const int qq = q - T + 1;   // position n + t of the run's local layout
        const int nn = 1 << (31 - __clz(qq));
        w = wbase + ((int64_t)nn << lgn) + (int64_t)s * nn + (qq - nn);
      } else {
        w = 10 * (int64_t)P2 + (q - R);
      }
      pa[i] = __ldg(row_ptr + w);
      pb[i] = __ldg(row_ptr + w + 1);
    }
  }
#pragma unroll
  for (int i = 0; i < SQ; ++i) {
    const int q = warp * 32 + RF_THREADS * i + lane;
    const int n = (int)(pb[i] - pa[i]);
    const unsigned mk = __ballot_sync(0xffffffffu, n > 0);
    int base = 0;
    if (lane == 0 && mk) base = atomicAdd(&n_rows_ne, __popc(mk));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (n > 0) lst[base + __popc(mk & ((1u << lane) - 1u))] = make_int2((int)(pa[i] - e0), (q << 16) | n);
  }
  __syncthreads();

  // b^w of the non-empty rows.  Row lengths are very uneven: up to K J entries at
  // the coarse levels, where nearly every coefficient is kept, a few dozen or none
  // at the fine ones.  Entries are read as aligned groups of 4 (a float4 of values
  // and 4 u16 column indices; the arrays are padded to whole groups), entries of a
  // group outside the row masked.  An 8-lane group takes a row (four rows per warp):
  // lane sub takes the row's groups sub, sub + 8, sub + 16, ... in order, two in
  // flight per pass, and the 8 partial sums meet in a 3-step xor tree.
  {
    constexpr int GQ = 2;   // groups of 4 entries in flight per lane
    const int NR = n_rows_ne;
    // groups counted from the aligned group holding entry e0 (32-bit offsets)
    const float4 *__restrict__ val4 = reinterpret_cast<const float4 *>(val) + (e0 >> 2);
    const uint2 *__restrict__ col4 = reinterpret_cast<const uint2 *>(col) + (e0 >> 2);
    const int e0m = (int)(e0 & 3);
    const int sub = lane & (RF_LPR - 1), grp = lane >> 3;
    for (int hb = warp * 4; hb < NR; hb += (RF_THREADS / 32) * 4) {
      const int h = hb + grp;
      const int2 r = h < NR ? lst[h] : make_int2(0, 0);
      const int n = r.y & 0xFFFF;
      const int rb = r.x + e0m, re = rb + n;
      const int qb = rb >> 2;
      const int nq = n > 0 ? ((re + 3) >> 2) - qb : 0;
      const int head = rb & 3, tail = re & 3;
      float acc[VV];
#pragma unroll
      for (int v = 0; v < VV; ++v) acc[v] = 0.0f;
      for (int i0 = 0; i0 < nq; i0 += GQ * RF_LPR) {
        float4 a[GQ];
        uint2 kk[GQ];
#pragma unroll
        for (int i = 0; i < GQ; ++i) {
          const int Q = qb + min(i0 + sub + RF_LPR * i, nq - 1);
          a[i] = __ldg(val4 + Q);
          kk[i] = __ldg(col4 + Q);
        }
#pragma unroll
        for (int i = 0; i < GQ; ++i) {
          const int qi = i0 + sub + RF_LPR * i;
          if (qi < nq) {
            const float av[4] = {a[i].x, a[i].y, a[i].z, a[i].w};
            const int kv[4] = {(int)(kk[i].x & 0xFFFFu), (int)(kk[i].x >> 16), (int)(kk[i].y & 0xFFFFu),
                               (int)(kk[i].y >> 16)};
            const int lo = qi == 0 ? head : 0;
            const int hi = (qi == nq - 1 && tail) ? tail : 4;
            if (lo == 0 && hi == 4) {
#pragma unroll
              for (int b = 0; b < 4; ++b) rf_fma<VV>(cs4, kv[b], av[b], acc);
            } else {
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                const bool in = b >= lo && b < hi;
                rf_fma<VV>(cs4, in ? kv[b] : 0, in ? av[b] : 0.0f, acc);
              }
            }
          }
        }
      }
#pragma unroll
      for (int v = 0; v < VV; ++v)
#pragma unroll
        for (int o = RF_LPR / 2; o > 0; o >>= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
      if (sub == 0 && h < NR)
#pragma unroll
        for (int v = 0; v < VV; ++v) rf_store<VV>(x, top, r.y >> 16, T, R, v, acc[v]);
    }
  }
  __syncthreads();

  // Synthesis by walking down the tree: an item (v, t) produces the G = min(4, L)
  // consecutive Morton positions G t .. G t + G - 1 of the run.  It starts from the
  // chart's scaling coefficient, descends the chart's coarse path to the run and the
  // run's levels to the ancestor of its positions, then expands the last log2(G)
  // levels in registers.  Each value is formed exactly as in the level-by-level
  // synthesis, ((a + d) / sqrt2 or (a - d) / sqrt2 from its parent and the
  // parent's detail), and details are only read, so the walks need no barriers.
  const float rs2 = 0.70710678118654752440f;
  const int lgG = min(lgL, 2), G = 1 << lgG;
  const int lgI = lgL - lgG;   // log2(items per vector)
  const unsigned m0 = (unsigned)s << lgL;
  const int r0 = (int)rf_compact(m0 >> 1), c0 = (int)rf_compact(m0);
  const int N = 10 * nu * nu + 2;
  float *__restrict__ B = cp.B;
  const int nv = bt.nv;
  for (int it = tid; it < (nv << lgI); it += RF_THREADS) {
    const int v = it >> lgI, t = it & ((1 << lgI) - 1);
    float a = top[v][0];
    for (int lv = 0; lv < lgn; ++lv) {
      const float dd = top[v][1 + lv];
      a = ((s >> (lgn - 1 - lv)) & 1) ? (a - dd) * rs2 : (a + dd) * rs2;
    }
    for (int ln = 0; ln < lgI; ++ln) {   // approximation index t >> (lgI - ln) at level 2^ln
      const int pidx = t >> (lgI - ln);
      const float dd = x[v][(1 << ln) + pidx];
      a = ((t >> (lgI - ln - 1)) & 1) ? (a - dd) * rs2 : (a + dd) * rs2;
    }
    float out[4] = {a, 0.0f, 0.0f, 0.0f};
    if (lgG == 2) {
      const int n1 = 1 << lgI, n2 = 2 << lgI;
      const float d1 = x[v][n1 + t];
      const float aL = (a + d1) * rs2, aR = (a - d1) * rs2;   // positions 2t, 2t + 1 of level n2
      const float dL = x[v][n2 + 2 * t], dR = x[v][n2 + 2 * t + 1];
      out[0] = (aL + dL) * rs2;
      out[1] = (aL - dL) * rs2;
      out[2] = (aR + dR) * rs2;
      out[3] = (aR - dR) * rs2;
    }
    const unsigned mb = (unsigned)t << lgG;   // first Morton position of the item in the run
    const int rr0 = (int)rf_compact(mb >> 1), cc0 = (int)rf_compact(mb);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (b >= G) break;
      const int r = r0 + rr0 + (b >> 1), c = c0 + cc0 + (b & 1);
      if (r < nu && c < nu) B[(size_t)v * N + (size_t)d * nu * nu + (size_t)r * nu + c] = out[b];
    }
  }
  if (poles && tid < nv) {
    B[(size_t)tid * N + 10 * (size_t)nu * nu] = top[tid][RF_MAX_TOP];
    B[(size_t)tid * N + 10 * (size_t)nu * nu + 1] = top[tid][RF_MAX_TOP + 1];
  }
}

bool relight_fusable(const tsr_compressed *c, int n_edit) {
  return c->wavelet == 0 && n_edit >= 1 && n_edit <= 2 && relight_fusable_basis(c);
}

bool relight_fusable_basis(const tsr_compressed *c) {
  return c->wavelet == 0 && c->P <= (1 << (RF_MAX_LGN / 2 + 5)) && c->nnz < (1ll << 31);
}

// Dynamic shared memory of relight_fused_kernel<VV>: x (VV > 6) and the c table.
template <int VV>
static size_t fused_smem(int K, int J) {
  constexpr int VQ = (VV + 3) / 4;
  return (VV > 6 ? sizeof(float) * VV * RF_SEG : 0) + sizeof(float4) * (size_t)((K * J + 31) & ~31) * VQ;
}

// Launches relight_fused_kernel<VV> over the copies, RF_MAXC per launch.  g: per-copy
// [nv][K] pointers, or all null for the basis images (nv = K rows: c_k[kj] = l[j] for
// the entries of basis k).
template <int VV>
static tsr_status launch_fused(int n, const tsr_compressed *const *c, int nv, const float *const *gi, const float *l,
                               float *const *Bi, cudaStream_t s) {
  const int K = c[0]->K, J = c[0]->J;
  const size_t smem = fused_smem<VV>(K, J);
  {   // dynamic shared memory up to the largest case (K = 16, J = 32), set once per device
    static std::atomic<bool> attr_set[64];   // the call is idempotent: threads racing here set the same value
    int dev = 0;
    TSR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
      TSR_CUDA(cudaFuncSetAttribute(relight_fused_kernel<VV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)fused_smem<VV>(16, 32)));
      if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
    }
  }
  for (int b0 = 0; b0 < n; b0 += RF_MAXC) {
    RelightBatch bt{};
    bt.n = std::min(RF_MAXC, n - b0);
    bt.nv = nv;
    int items = 0;
    for (int i = 0; i < bt.n; ++i) {
      const tsr_compressed *h = c[b0 + i];
      RelightCopy &cp = bt.c[i];
      cp.row_ptr = h->row_ptr;
      cp.col = h->col;
      cp.val = h->val;
      cp.g = gi ? gi[b0 + i] : nullptr;
      cp.B = Bi[b0 + i];
      cp.nu = h->nu;
      cp.lgP = ilog2(h->P);
      cp.item0 = items;
      items += 10 * std::max(1, (h->P * h->P) / RF_SEG);
    }
    relight_fused_kernel<VV><<<items, RF_THREADS, smem, s>>>(bt, K, J, l);
    ::tsr::count_launch();
    TSR_CUDA(cudaGetLastError());
  }
  return TSR_OK;
}

// Copies must all be fusable for n_edit and share K and J; copy i reads g from gi[i]
// ([n_edit][3][K]) and writes B to Bi[i] ([n_edit][3][N_i]).
tsr_status relight_fused(int n, const tsr_compressed *const *c, int n_edit, const float *const *gi, const float *l,
                         float *const *Bi, cudaStream_t s) {
  if (n <= 0) return TSR_OK;
  return n_edit == 1 ? launch_fused<3>(n, c, 3, gi, l, Bi, s) : launch_fused<6>(n, c, 6, gi, l, Bi, s);
}

// Z_i[k] = w_1^{-1} (S_i (e_k x l)) for every copy (Zi[i]: [K][N_i]), one fused pass
// per 32 copies: the light-contracted basis images of the factorised relight.
tsr_status relight_basis_images_many(int n, const tsr_compressed *const *c, const float *l, float *const *Zi,
                                     cudaStream_t s) {
  if (n <= 0) return TSR_OK;
  const int K = c[0]->K;
  if (K <= 3) return launch_fused<3>(n, c, K, nullptr, l, Zi, s);
  if (K <= 6) return launch_fused<6>(n, c, K, nullptr, l, Zi, s);
  if (K <= 12) return launch_fused<12>(n, c, K, nullptr, l, Zi, s);
  return launch_fused<16>(n, c, K, nullptr, l, Zi, s);
}

// ---------------------------------------------------------------- combine, many copies
// B_i[v][o] = sum_k g_i[v][k] Z_i[k][o] for every copy i: a block per (512 vertices of
// one copy, RC_VB vectors), the K values of Z of its vertex held in registers, the
// vectors' g in shared memory as float4 rows of KT = K rounded up to 4 (zero padded,
// so the loop has no per-basis test; the padding adds fmaf(0, 0, b) = b).  Same
// arithmetic as relight_combine_kernel.
constexpr int RC_VB = 32;
constexpr int RC_VERTS = 512;   // vertices per block (two per thread; four measured slower: registers)
struct CombineCopy {
  const float *Z;   // [K][N]
  const float *g;   // [V][K]
  float *B;         // [V][N]
  int N;
  int blk0;         // first vertex block of the copy
};
struct CombineBatch {
  CombineCopy c[RF_MAXC];
  int n, K, V;
};

template <int KT>
__global__ void __launch_bounds__(256) relight_combine_many_kernel(const __grid_constant__ CombineBatch cb) {
  __shared__ float4 gs[RC_VB * KT / 4];
  int ci = 0;
  while (ci + 1 < cb.n && cb.c[ci + 1].blk0 <= (int)blockIdx.x) ++ci;
  const CombineCopy &cp = cb.c[ci];
  const int K = cb.K, V = cb.V, N = cp.N;
  const int v0 = blockIdx.y * RC_VB;
  float *gsf = reinterpret_cast<float *>(gs);
  for (int q = threadIdx.x; q < RC_VB * KT; q += blockDim.x) {
    const int vv = q / KT, k = q - vv * KT;
    gsf[q] = (v0 + vv < V && k < K) ? cp.g[(size_t)(v0 + vv) * K + k] : 0.0f;
  }
  __syncthreads();
  // two vertices per thread (o and o + 256): each g row read from shared memory serves both
  const int o = ((int)blockIdx.x - cp.blk0) * RC_VERTS + threadIdx.x;
  if (o >= N) return;
  const bool two = o + 256 < N;
  float z[2][KT];
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    z[0][k] = (k < K) ? __ldg(cp.Z + (size_t)k * N + o) : 0.0f;
    z[1][k] = (k < K && two) ? __ldg(cp.Z + (size_t)k * N + o + 256) : 0.0f;
  }
  const int vn = min(RC_VB, V - v0);
  float *__restrict__ B = cp.B + (size_t)v0 * N + o;
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
    B[(size_t)vv * N] = b0;
    if (two) B[(size_t)vv * N + 256] = b1;
  }
}

template <int KT>
static tsr_status launch_combine_many(int n, const float *const *Zi, const int *Ni, int K, int V,
                                      const float *const *gi, float *const *Bi, cudaStream_t s) {
  for (int b0 = 0; b0 < n; b0 += RF_MAXC) {
    CombineBatch cb{};
    cb.n = std::min(RF_MAXC, n - b0);
    cb.K = K;
    cb.V = V;
    int blocks = 0;
    for (int i = 0; i < cb.n; ++i) {
      CombineCopy &cp = cb.c[i];
      cp.Z = Zi[b0 + i];
      cp.g = gi[b0 + i];
      cp.B = Bi[b0 + i];
      cp.N = Ni[b0 + i];
      cp.blk0 = blocks;
      blocks += (cp.N + RC_VERTS - 1) / RC_VERTS;
    }
    relight_combine_many_kernel<KT><<<dim3(blocks, (V + RC_VB - 1) / RC_VB), 256, 0, s>>>(cb);
    ::tsr::count_launch();
    TSR_CUDA(cudaGetLastError());
  }
  return TSR_OK;
}

tsr_status relight_combine_many(int n, const float *const *Zi, const int *Ni, int K, int V, const float *const *gi,
                                float *const *Bi, cudaStream_t s) {
  if (K <= 4) return launch_combine_many<4>(n, Zi, Ni, K, V, gi, Bi, s);
  if (K <= 8) return launch_combine_many<8>(n, Zi, Ni, K, V, gi, Bi, s);
  if (K <= 12) return launch_combine_many<12>(n, Zi, Ni, K, V, gi, Bi, s);
  return launch_combine_many<16>(n, Zi, Ni, K, V, gi, Bi, s);
}

}  // namespace tsr
