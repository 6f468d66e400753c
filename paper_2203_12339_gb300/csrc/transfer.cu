// Section 3, Eq. 6-7 (precompute Step 1): the transfer
//     M[k][j][o] = sum_i A_i f_k(|x_o - x_i|) T[j][i]
// generated and contracted on the fly, so the N x N kernel matrix never
// reaches HBM.
//
//  * transfer_fp32: CUDA-core FP32 path.  A block owns 32 output rows; each
//    thread owns one row o and two bases, evaluates f_k(r) from the table and
//    accumulates all J products per pair, with the partial sum of each 64-i
//    tile added into a Kahan-compensated total.
//  * transfer_tc:   tensor-core path (tcgen05).  A block owns 128 output rows
//    (the UMMA M = 128) and a group of KB bases.  Per 16-i step, 256 threads
//    evaluate F_k[o, i] = f_k(r_oi) (BF16, or hi/lo BF16 for the split
//    variant) into shared memory in the canonical K-major layout, while the
//    Tensor Memory Accelerator streams the matching tile of
//    T'[j][i] = A_i T[j][i] (pre-tiled BF16 records that also carry the x_i).
//    One thread issues tcgen05.mma with FP32 accumulators for all KB bases in
//    tensor memory (KB x J_pad columns); the epilogue reads TMEM back with
//    tcgen05.ld and writes M.
//
// Pair geometry (both paths): dx = fl(x_o - x_i) etc. and
// r2 = fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)) without contraction; pairs with
// r2 > fl(r_max^2) are cut off (f_k = 0).  Otherwise r = sqrt(r2),
// x = r / dr, m = min(floor(x), n_r - 2), t = x - m and
// f_k(r) = v_k[m] + t s_k[m] (s_k = f_k[m+1] - f_k[m]).
#include <algorithm>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>
#include <vector>

#include "handles.cuh"

namespace tsr {

__device__ __forceinline__ float pair_r2(float xo, float yo, float zo, float xi, float yi, float zi) {
  const float dx = __fsub_rn(xo, xi), dy = __fsub_rn(yo, yi), dz = __fsub_rn(zo, zi);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ============================================================================ FP32 SIMT
constexpr int F32_BO = 32;   // output rows per block
constexpr int F32_BI = 64;   // i per shared-memory tile

// T'[i][jp] = A_i T[j][i] (FP32, zero for j >= J or i >= N), rows padded to a multiple of F32_BI.
__global__ void pretile_fp32_kernel(const float *__restrict__ area, const float *__restrict__ T, int N, int J,
                                    int JP, int n_pad, float *__restrict__ Tp) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_pad * JP) return;
  const int i = idx / JP, j = idx % JP;
  Tp[idx] = (i < N && j < J) ? area[i] * T[(size_t)j * N + i] : 0.0f;
}

template <int JP>
__global__ void __launch_bounds__(256, 1)
    transfer_fp32_kernel(const float *__restrict__ pos, int N, const float *__restrict__ Tp,
                         const float4 *__restrict__ tab, int KG, int n_r, float inv_dr, float r2max, int K,
                         int J, float *__restrict__ M, int n_tiles) {
  __shared__ __align__(16) float sT[F32_BI * JP];
  __shared__ float sx[F32_BI], sy[F32_BI], sz[F32_BI];
  const int kg = threadIdx.x % KG;
  const int ol = threadIdx.x / KG;
  const float *px = pos, *py = pos + N, *pz = pos + 2 * (size_t)N;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int o = tile * F32_BO + ol;
    const bool o_ok = o < N;
    const float xo = o_ok ? px[o] : 0.0f, yo = o_ok ? py[o] : 0.0f, zo = o_ok ? pz[o] : 0.0f;
    float acc0[JP], acc1[JP], c0[JP], c1[JP];
#pragma unroll
    for (int j = 0; j < JP; ++j) acc0[j] = acc1[j] = c0[j] = c1[j] = 0.0f;
    for (int i0 = 0; i0 < N; i0 += F32_BI) {
      __syncthreads();
      const float4 *src = reinterpret_cast<const float4 *>(Tp + (size_t)i0 * JP);
      for (int q = threadIdx.x; q < F32_BI * JP / 4; q += blockDim.x) reinterpret_cast<float4 *>(sT)[q] = src[q];
      for (int q = threadIdx.x; q < F32_BI; q += blockDim.x) {
        const int i = i0 + q;
        sx[q] = i < N ? px[i] : 0.0f;
        sy[q] = i < N ? py[i] : 0.0f;
        sz[q] = i < N ? pz[i] : 0.0f;
      }
      __syncthreads();
      float p0[JP], p1[JP];
#pragma unroll
      for (int j = 0; j < JP; ++j) p0[j] = p1[j] = 0.0f;
#pragma unroll 2
      for (int ii = 0; ii < F32_BI; ++ii) {
        const float r2 = pair_r2(xo, yo, zo, sx[ii], sy[ii], sz[ii]);
        const float x = __fsqrt_rn(r2) * inv_dr;
        const int m = max(0, min(static_cast<int>(x), n_r - 2));
        const float t = x - static_cast<float>(m);
        const int row = (r2 <= r2max) ? m : n_r;
        const float4 tb = __ldg(tab + (size_t)row * KG + kg);
        const float F0 = fmaf(t, tb.y, tb.x), F1 = fmaf(t, tb.w, tb.z);
        const float *tv = sT + ii * JP;
#pragma unroll
        for (int j = 0; j < JP; ++j) {
          p0[j] = fmaf(F0, tv[j], p0[j]);
          p1[j] = fmaf(F1, tv[j], p1[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < JP; ++j) {   // Kahan: total += tile partial
        float y = p0[j] - c0[j];
        float s = acc0[j] + y;
        c0[j] = (s - acc0[j]) - y;
        acc0[j] = s;
        y = p1[j] - c1[j];
        s = acc1[j] + y;
        c1[j] = (s - acc1[j]) - y;
        acc1[j] = s;
      }
    }
    if (o_ok) {
      const int k0 = 2 * kg, k1 = 2 * kg + 1;
#pragma unroll
      for (int j = 0; j < JP; ++j) {
        if (j < J) {
          if (k0 < K) M[((size_t)k0 * J + j) * N + o] = acc0[j];
          if (k1 < K) M[((size_t)k1 * J + j) * N + o] = acc1[j];
        }
      }
    }
  }
}

template <int JP>
static cudaError_t launch_fp32(int grid, int threads, cudaStream_t s, const float *pos, int N, const float *Tp,
                               const float4 *tab, int KG, int n_r, float inv_dr, float r2max, int K, int J,
                               float *M, int n_tiles) {
  transfer_fp32_kernel<JP><<<grid, threads, 0, s>>>(pos, N, Tp, tab, KG, n_r, inv_dr, r2max, K, J, M, n_tiles);
  return cudaGetLastError();
}

tsr_status transfer_fp32(const tsr_basis *b, int N, const float *pos, const float *area, const float *T, int J,
                         float *M, cudaStream_t s) {
  const int JP = (J + 3) & ~3;
  const int n_pad = (N + F32_BI - 1) / F32_BI * F32_BI;
  Scratch tp;
  tsr_status st = tp.alloc(sizeof(float) * (size_t)n_pad * JP, s);
  if (st != TSR_OK) return st;
  float *Tp = static_cast<float *>(tp.p);
  pretile_fp32_kernel<<<(n_pad * JP + 255) / 256, 256, 0, s>>>(area, T, N, J, JP, n_pad, Tp);
  TSR_CUDA(cudaGetLastError());
  const int KG = b->KP / 2;
  const int threads = F32_BO * KG;
  const int n_tiles = (N + F32_BO - 1) / F32_BO;
  const int grid = std::min(n_tiles, num_sms());
  const float inv_dr = static_cast<float>((b->n_r - 1) / b->r_max);
  const float r2max = static_cast<float>(b->r_max * b->r_max);
  const float4 *tab = reinterpret_cast<const float4 *>(b->tab32);
  cudaError_t e;
  switch (JP) {
#define F32_CASE(JPV) \
  case JPV: e = launch_fp32<JPV>(grid, threads, s, pos, N, Tp, tab, KG, b->n_r, inv_dr, r2max, b->K, J, M, n_tiles); break;
    F32_CASE(4) F32_CASE(8) F32_CASE(12) F32_CASE(16) F32_CASE(20) F32_CASE(24) F32_CASE(28) F32_CASE(32)
#undef F32_CASE
    default:
      set_error("transfer_fp32: J=%d unsupported", J);
      return TSR_ERR_UNSUPPORTED;
  }
  TSR_CUDA(e);
  return TSR_OK;
}

// ============================================================================ tcgen05 path
// Record of one 16-i step in global memory (and, after TMA, in shared memory):
//   [0, JP*32)            T'_hi tile, canonical K-major no-swizzle layout:
//                         core matrix (h = i/8, jg = j/8) at h*JP*16 + jg*128,
//                         row j%8 at +16*(j%8), element i%8 at +2*(i%8)
//   [JP*32, 2*JP*32)      T'_lo tile (split variant only)
//   next 192 bytes        x[16], y[16], z[16] (FP32) of the 16 i
//   padded to a multiple of 128 bytes (the TMA box row).
__host__ __device__ constexpr int rec_bytes(int JP, bool split) {
  return ((JP * 32 * (split ? 2 : 1) + 192) + 127) / 128 * 128;
}

__global__ void pretile_tc_kernel(const float *__restrict__ pos, const float *__restrict__ area,
                                  const float *__restrict__ T, int N, int J, int JP, int split, int REC,
                                  int n_steps, uint8_t *__restrict__ rec) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // (step, ii)
  if (idx >= n_steps * 16) return;
  const int step = idx / 16, ii = idx % 16;
  const int i = step * 16 + ii;
  const bool ok = i < N;
  uint8_t *r = rec + (size_t)step * REC;
  const float a = ok ? area[i] : 0.0f;
  const int h = ii / 8, e = ii % 8;
  for (int j = 0; j < JP; ++j) {
    const float v = (ok && j < J) ? a * T[(size_t)j * N + i] : 0.0f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const size_t off = (size_t)h * JP * 16 + (size_t)j * 16 + e * 2;
    *reinterpret_cast<__nv_bfloat16 *>(r + off) = hi;
    if (split) {
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      *reinterpret_cast<__nv_bfloat16 *>(r + JP * 32 + off) = lo;
    }
  }
  float *p = reinterpret_cast<float *>(r + JP * 32 * (split ? 2 : 1));
  p[ii] = ok ? pos[i] : 0.0f;
  p[16 + ii] = ok ? pos[N + i] : 0.0f;
  p[32 + ii] = ok ? pos[2 * (size_t)N + i] : 0.0f;
}

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version (sm_100 family)
  return d;                 // base offset 0, layout SWIZZLE_NONE
}

__host__ __device__ constexpr uint32_t umma_idesc_bf16(int N) {
  return (1u << 4)                       // D: F32
         | (1u << 7)                     // A: BF16
         | (1u << 10)                    // B: BF16
         | ((uint32_t)(N >> 3) << 17)    // N
         | ((uint32_t)(128 >> 4) << 24); // M = 128; A, B K-major
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t bf16x2_fma(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// ---------------------------------------------------------------- the kernel
struct TcArgs {
  int N;             // vertices (rows o and columns i)
  int n_steps;       // 16-i steps (records), a multiple of KS
  int n_r;           // radius samples
  float inv_dr, r2max;
  int K, J;
  int n_otiles, n_kgroups, n_items;
  int n_split;       // each tile's i-range is cut into n_split units (wave balance)
  float *P;          // [n_split-1][K][J][N] partial sums of units 1.. (NULL if n_split == 1)
  const float *pos;  // [3][N] (rows o)
  const float *area; // [N]      (self pair, FP32 epilogue)
  const float *T;    // [J][N]   (self pair, FP32 epilogue)
  const uint32_t *tab16;   // [n_r + 1][KP] bf16x2
  const float2 *tab32;     // [n_r + 1][KP]
  int KP;
  int seg_stages;    // stages per accumulation segment (TMEM flushed to M after each)
  float *M;          // [K][J][N]
  unsigned *status;
};

template <int KB, int JP, bool SPLIT, int NS, int KS>
struct TcCfg {
  static constexpr int NR = NS + 2;                        // record stages (TMA runs 2 stages ahead)
  static constexpr int LOOKAHEAD = 2;
  static constexpr int REC = rec_bytes(JP, SPLIT);
  static constexpr int A_TILE = 128 * 16 * 2;              // one (base, 16-i step) BF16 tile
  static constexpr int A_STAGE = KS * KB * (SPLIT ? 2 : 1) * A_TILE;
  static constexpr int REC_STAGE = KS * REC;
  static constexpr int TAB_ELEM = SPLIT ? 8 : 4;
  static constexpr int U = KB * TAB_ELEM / 16;             // 16-byte units per table row
  static constexpr int NGEN = 512;                         // generator threads (warps 0-15)
  static constexpr int NTHREADS = NGEN + 32;               // + one control warp (TMA + MMA issue)
  static constexpr int TMEM_COLS = (KB * JP <= 32) ? 32 : (KB * JP <= 64) ? 64 : (KB * JP <= 128) ? 128
                                 : (KB * JP <= 256) ? 256 : 512;
  static size_t smem_bytes(int n_r) {
    return 1024 + (size_t)NS * A_STAGE + (size_t)NR * REC_STAGE + (size_t)(n_r + 1) * KB * TAB_ELEM + 256;
  }
};

// Table rows are U 16-byte units; rotating the units of row m by m/2 (U = 4) or
// m/4 (U = 2) spreads the rows read by one warp over all eight bank groups.
template <int U>
__device__ __forceinline__ int tab_unit(int m, int u) {
  if (U == 4) return m * 4 + ((u + (m >> 1)) & 3);
  if (U == 2) return m * 2 + ((u + (m >> 2)) & 1);
  return m * U + u;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up as soon as another thread raised the abort flag.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  for (uint32_t it = 0; it < TSR_WAIT_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

template <int KB, int JP, bool SPLIT, int NS, int KS>
__global__ void __launch_bounds__(TcCfg<KB, JP, SPLIT, NS, KS>::NTHREADS, 1)
    transfer_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs args) {
  using C = TcCfg<KB, JP, SPLIT, NS, KS>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // align by pointer arithmetic on the shared array (keeps the shared address space: LDS/STS, not generic)
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *sA = smem;                                   // NS * A_STAGE
  uint8_t *sRec = sA + (size_t)NS * C::A_STAGE;         // NR * REC_STAGE
  uint8_t *sTab = sRec + (size_t)C::NR * C::REC_STAGE;  // (n_r+1) * KB * TAB_ELEM
  uint64_t *bar = reinterpret_cast<uint64_t *>(sTab + (size_t)(args.n_r + 1) * KB * C::TAB_ELEM);
  uint64_t *bar_tma = bar;                        // [NR] records landed
  uint64_t *bar_full = bar + C::NR;               // [NS] A stage written by all generators
  uint64_t *bar_mma = bar + C::NR + NS;           // [NS] MMAs of a stage completed
  uint64_t *bar_tfree = bar + C::NR + 2 * NS;     // [1]  epilogue finished reading TMEM
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar + C::NR + 2 * NS + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
  volatile long *tma_done = reinterpret_cast<volatile long *>(tmem_holder + 2);   // stages whose records generators saw

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // Items: (k-group, 128-row tile).  Each CTA keeps one k-group, so its table
  // slice is loaded once: CTA b takes group b % G and tiles b / G, b / G + grid / G, ...
  const int G = args.n_kgroups;
  const int kgroup = blockIdx.x % G;
  const int k0 = kgroup * KB;
  // Units: (tile, split).  Unit u covers tile u / S and stages [sp*SPT/S, (sp+1)*SPT/S) of it.
  const int S = args.n_split;
  const int SPT = args.n_steps / KS;   // stages of a whole tile
  const int unit_first = blockIdx.x / G, unit_step = gridDim.x / G;
  const int n_units = args.n_otiles * S;
  long total_stages = 0;
  for (int u = unit_first; u < n_units; u += unit_step) {
    const int sp = u % S;
    total_stages += (long)((sp + 1) * SPT / S - sp * SPT / S);
  }
  const int seg_stages = args.seg_stages;

  if (tid == 0) {
    for (int q = 0; q < C::NR; ++q) mbar_init(&bar_tma[q], 1);
    for (int q = 0; q < NS; ++q) {
      mbar_init(&bar_full[q], C::NGEN);
      mbar_init(&bar_mma[q], 1);
    }
    mbar_init(bar_tfree, C::NGEN);
    *abort_flag = 0;
    *tma_done = 0;
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  // this group's table slice (zero beyond K), rows swizzled by tab_unit
  {
    const int n_units = (args.n_r + 1) * C::U;
    for (int q = tid; q < n_units; q += blockDim.x) {
      const int m = q / C::U, u = q % C::U;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      if (!SPLIT) {
        uint32_t e4[4] = {0u, 0u, 0u, 0u};   // {lo: v_k, hi: s_k} per base
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = k0 + u * 4 + e;
          if (k < args.K) e4[e] = args.tab16[(size_t)m * args.KP + k];
        }
        w[0] = __byte_perm(e4[0], e4[1], 0x5410);   // {v_k, v_k+1}
        w[1] = __byte_perm(e4[2], e4[3], 0x5410);   // {v_k+2, v_k+3}
        w[2] = __byte_perm(e4[0], e4[1], 0x7632);   // {s_k, s_k+1}
        w[3] = __byte_perm(e4[2], e4[3], 0x7632);   // {s_k+2, s_k+3}
      } else {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k = k0 + u * 2 + e;
          if (k < args.K) {
            const float2 f = args.tab32[(size_t)m * args.KP + k];
            w[2 * e] = __float_as_uint(f.x);
            w[2 * e + 1] = __float_as_uint(f.y);
          }
        }
      }
      v = make_uint4(w[0], w[1], w[2], w[3]);
      reinterpret_cast<uint4 *>(sTab)[tab_unit<C::U>(m, u)] = v;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const int rows_per_stage = C::REC_STAGE / 128;

  if (warp == C::NGEN / 32) {
    // ------------------------------------------------------------ control warp
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_bf16(JP);
      const uint32_t sA_u32 = smem_u32(sA);
      long issued = 0;
      // TMA cursor: unit tu, absolute stage ts within the tile (runs LOOKAHEAD stages ahead)
      int tu = unit_first, ts = 0, te = 0;
      if (tu < n_units) {
        ts = (tu % S) * SPT / S;
        te = (tu % S + 1) * SPT / S;
      }
      auto issue_tma = [&](long q) {
        const int slot = (int)(q % C::NR);
        mbar_arrive_expect_tx(&bar_tma[slot], C::REC_STAGE);
        tma_load_2d(sRec + (size_t)slot * C::REC_STAGE, &tmap, &bar_tma[slot], 0, ts * rows_per_stage);
        if (++ts == te) {   // next unit of this CTA
          tu += unit_step;
          if (tu < n_units) {
            ts = (tu % S) * SPT / S;
            te = (tu % S + 1) * SPT / S;
          }
        }
      };
      for (; issued < C::LOOKAHEAD && issued < total_stages; ++issued) issue_tma(issued);
      long g = 0;
      int seg_no = 0;   // accumulation segments issued so far
      for (int u = unit_first; u < n_units && !*abort_flag; u += unit_step) {
        const int sb = (u % S) * SPT / S, se = (u % S + 1) * SPT / S;
        for (int sidx = sb; sidx < se && !*abort_flag; ++sidx, ++g) {
          const bool seg_start = ((sidx - sb) % seg_stages) == 0;
          // TMA of stage g + LOOKAHEAD reuses the slot of stage g - NS: wait for its MMAs
          if (issued < total_stages && issued <= g + C::LOOKAHEAD) {
            const long prev = issued - C::NR;
            if (prev >= 0 && !wait_or_abort(&bar_mma[prev % NS], (uint32_t)((prev / NS) & 1), abort_flag)) break;
            issue_tma(issued);
            ++issued;
          }
          const int sa = (int)(g % NS);
          if (!wait_or_abort(&bar_full[sa], (uint32_t)((g / NS) & 1), abort_flag)) break;
          // the epilogue of the previous segment must have read TMEM before it is overwritten
          if (seg_start && seg_no > 0 && !wait_or_abort(bar_tfree, (uint32_t)((seg_no - 1) & 1), abort_flag)) break;
          if (seg_start) ++seg_no;
          tc_fence_after();
          const uint32_t rec_u32 = smem_u32(sRec + (size_t)(g % C::NR) * C::REC_STAGE);
#pragma unroll 1
          for (int ks = 0; ks < KS; ++ks) {
            const uint32_t b_hi = rec_u32 + ks * C::REC;
            const uint64_t dbh = umma_desc(b_hi, JP * 16, 128);
            const uint64_t dbl = umma_desc(b_hi + JP * 32, JP * 16, 128);
            const uint32_t a_step =
                sA_u32 + (uint32_t)(sa * C::A_STAGE) + (uint32_t)(ks * KB * (SPLIT ? 2 : 1) * C::A_TILE);
            const uint32_t first = (seg_start && ks == 0) ? 0u : 1u;
#pragma unroll 1
            for (int kb = 0; kb < KB; ++kb) {
              const uint32_t d = tmem_base + (uint32_t)(kb * JP);
              if (!SPLIT) {
                umma_bf16(d, umma_desc(a_step + kb * C::A_TILE, 128, 256), dbh, idesc, first);
              } else {
                const uint64_t dah = umma_desc(a_step + (2 * kb) * C::A_TILE, 128, 256);
                const uint64_t dal = umma_desc(a_step + (2 * kb + 1) * C::A_TILE, 128, 256);
                umma_bf16(d, dah, dbh, idesc, first);
                umma_bf16(d, dah, dbl, idesc, 1u);
                umma_bf16(d, dal, dbh, idesc, 1u);
              }
            }
          }
          umma_commit(&bar_mma[sa]);
        }
      }
      if (*abort_flag) {   // let copies already issued land before the CTA exits
        for (long q = *tma_done; q < issued; ++q) {
          for (uint32_t it = 0; it < TSR_WAIT_LIMIT; ++it)
            if (mbar_try_wait(&bar_tma[q % C::NR], (uint32_t)((q / C::NR) & 1))) break;
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ generator warps
    // Thread (orow, h4): output row orow of the tile, i = 4*h4 .. 4*h4+3 of every 16-i step.
    // A warp covers 16 rows x two neighbouring i-quarters, so its 8-byte stores fill
    // two whole 128-byte core matrices (2 shared-memory wavefronts per store).
    const int orow = (warp & 7) * 16 + (lane & 7) + ((lane >> 4) << 3);
    const int h4 = (warp >> 3) * 2 + ((lane >> 3) & 1);
    const uint32_t a_row_off =
        (uint32_t)((orow >> 3) * 256 + (h4 >> 1) * 128 + (orow & 7) * 16 + (h4 & 1) * 8);
    const uint32_t sA_u32 = smem_u32(sA);
    const float r2max = args.r2max, inv_dr = args.inv_dr;
    const int n_r = args.n_r;
    long g = 0;
    for (int u = unit_first; u < n_units; u += unit_step) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const int t = u / S, sp = u % S;
      const int sb = sp * SPT / S, se = (sp + 1) * SPT / S;
      float *Mdst = (sp == 0) ? args.M : args.P + (size_t)(sp - 1) * args.K * args.J * args.N;
      const int o = t * 128 + orow;
      const bool o_ok = o < args.N;
      const float xo = o_ok ? args.pos[o] : 0.f;
      const float yo = o_ok ? args.pos[args.N + o] : 0.f;
      const float zo = o_ok ? args.pos[2 * (size_t)args.N + o] : 0.f;
      bool ok = true;
      for (int sidx = sb; sidx < se; ++sidx, ++g) {
        const int sa = (int)(g % NS);
        const int sr = (int)(g % C::NR);
        bool w_ok = true;
        if (g >= NS) w_ok = wait_or_abort(&bar_mma[sa], (uint32_t)(((g / NS) - 1) & 1), abort_flag);
        if (w_ok) w_ok = wait_or_abort(&bar_tma[sr], (uint32_t)((g / C::NR) & 1), abort_flag);
        if (__any_sync(0xffffffffu, !w_ok)) {
          ok = false;
          break;
        }
        if (tid == 0) *tma_done = g + 1;
        const uint8_t *rec_stage = sRec + (size_t)sr * C::REC_STAGE;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          const float *rp = reinterpret_cast<const float *>(rec_stage + ks * C::REC + JP * 32 * (SPLIT ? 2 : 1));
          const float4 xs = *reinterpret_cast<const float4 *>(rp + h4 * 4);
          const float4 ys = *reinterpret_cast<const float4 *>(rp + 16 + h4 * 4);
          const float4 zs = *reinterpret_cast<const float4 *>(rp + 32 + h4 * 4);
          const float xa[4] = {xs.x, xs.y, xs.z, xs.w}, ya[4] = {ys.x, ys.y, ys.z, ys.w},
                      za[4] = {zs.x, zs.y, zs.z, zs.w};
          // Padded i (beyond N) carry T' = 0 and finite positions, so they add nothing;
          // the self pair i = o is corrected to FP32 in the epilogue.
          int row[4];
          float tq[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float dx = xo - xa[u], dy = yo - ya[u], dz = zo - za[u];
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            bool inside = r2 <= r2max;
            if (fabsf(r2 - r2max) <= 1e-3f * r2max)   // near the cutoff: decide on the exact FP32 r^2
              inside = pair_r2(xo, yo, zo, xa[u], ya[u], za[u]) <= r2max;
            const float x = r2 * rsqrtf(fmaxf(r2, 1e-30f)) * inv_dr;
            // m = floor(x) (round-to-nearest of x - 1/2 at 1.5 * 2^23), t = x - m
            const float yv = (x - 0.5f) + 12582912.0f;
            const int m = __float_as_int(yv) - 0x4B400000;
            tq[u] = x - (yv - 12582912.0f);
            row[u] = inside ? m : n_r;
          }
          const uint32_t a_step =
              sA_u32 + (uint32_t)(sa * C::A_STAGE) + (uint32_t)(ks * KB * (SPLIT ? 2 : 1) * C::A_TILE);
          if (!SPLIT) {
            // unit kb4 of a table row: {v_4kb4..+1, v_+2..+3, s_4kb4..+1, s_+2..+3} (bf16 pairs)
            uint32_t t2[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) t2[u] = pack_bf16x2(tq[u], tq[u]);
            const uint4 *tab4 = reinterpret_cast<const uint4 *>(sTab);
#pragma unroll
            for (int kb4 = 0; kb4 < KB / 4; ++kb4) {
              uint4 w[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) w[u] = tab4[tab_unit<C::U>(row[u], kb4)];
              uint32_t F01[4], F23[4];   // {F_k, F_k+1} of pair u
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                F01[u] = bf16x2_fma(t2[u], w[u].z, w[u].x);
                F23[u] = bf16x2_fma(t2[u], w[u].w, w[u].y);
              }
              const uint32_t base = a_step + (uint32_t)(kb4 * 4 * C::A_TILE) + a_row_off;
              st_shared_v2(base, __byte_perm(F01[0], F01[1], 0x5410), __byte_perm(F01[2], F01[3], 0x5410));
              st_shared_v2(base + C::A_TILE, __byte_perm(F01[0], F01[1], 0x7632), __byte_perm(F01[2], F01[3], 0x7632));
              st_shared_v2(base + 2 * C::A_TILE, __byte_perm(F23[0], F23[1], 0x5410), __byte_perm(F23[2], F23[3], 0x5410));
              st_shared_v2(base + 3 * C::A_TILE, __byte_perm(F23[0], F23[1], 0x7632), __byte_perm(F23[2], F23[3], 0x7632));
            }
          } else {
            const float4 *tab4 = reinterpret_cast<const float4 *>(sTab);   // {v_k, s_k, v_k+1, s_k+1}
#pragma unroll
            for (int kb2 = 0; kb2 < KB / 2; ++kb2) {
              float F0[4], F1[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float4 w = tab4[tab_unit<C::U>(row[u], kb2)];
                F0[u] = fmaf(tq[u], w.y, w.x);
                F1[u] = fmaf(tq[u], w.w, w.z);
              }
#pragma unroll
              for (int b = 0; b < 2; ++b) {
                const float *F = b ? F1 : F0;
                const uint32_t hi01 = pack_bf16x2(F[0], F[1]), hi23 = pack_bf16x2(F[2], F[3]);
                const uint32_t lo01 = pack_bf16x2(F[0] - __uint_as_float(hi01 << 16),
                                                  F[1] - __uint_as_float(hi01 & 0xFFFF0000u));
                const uint32_t lo23 = pack_bf16x2(F[2] - __uint_as_float(hi23 << 16),
                                                  F[3] - __uint_as_float(hi23 & 0xFFFF0000u));
                const int kb = kb2 * 2 + b;
                st_shared_v2(a_step + (uint32_t)((2 * kb) * C::A_TILE) + a_row_off, hi01, hi23);
                st_shared_v2(a_step + (uint32_t)((2 * kb + 1) * C::A_TILE) + a_row_off, lo01, lo23);
              }
            }
          }
        }
        fence_proxy_async_smem();
        mbar_arrive(&bar_full[sa]);
        if ((sidx - sb + 1) % seg_stages != 0 && sidx + 1 != se) continue;
        // End of an accumulation segment: TMEM -> registers -> M.  The tensor-core
        // FP32 accumulator is flushed every seg_stages steps and summed into M with
        // round-to-nearest adds.  The first segment also replaces the self pair's
        // BF16 product (exact in FP32) by f_k(0) A_o T[j][o] in FP32.
        const int seg_in_item = (sidx - sb) / seg_stages;
        const long last = g;
        const bool e_ok = wait_or_abort(&bar_mma[last % NS], (uint32_t)((last / NS) & 1), abort_flag);
        if (__any_sync(0xffffffffu, !e_ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int quarter = warp & 3, wq = warp >> 2;
        const int oe = t * 128 + quarter * 32 + lane;
        const bool oe_ok = oe < args.N;
        const float a_o = oe_ok ? args.area[oe] : 0.f;
        for (int kb = wq; kb < KB; kb += C::NGEN / 128) {
          const int k = k0 + kb;
          const float f0 = (k < args.K) ? args.tab32[k].x : 0.f;   // f_k(0), FP32
          const float f0h = __bfloat162float(__float2bfloat16_rn(f0));
          const float f0l = __bfloat162float(__float2bfloat16_rn(f0 - f0h));
#pragma unroll
          for (int jc = 0; jc < JP; jc += 16) {
            uint32_t r[16];
            tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(kb * JP + jc), r);
            tmem_ld_wait();
            if (k < args.K && oe_ok) {
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const int j = jc + q;
                if (j < args.J) {
                  float *dst = Mdst + ((size_t)k * args.J + j) * args.N + oe;
                  if (seg_in_item == 0 && sp == 0) {
                    const float tp = a_o * args.T[(size_t)j * args.N + oe];
                    const float th = __bfloat162float(__float2bfloat16_rn(tp));
                    float tc_self;
                    if (!SPLIT) {
                      tc_self = __bfloat162float(__ushort_as_bfloat16((unsigned short)(args.tab16[k] & 0xFFFFu))) * th;
                    } else {
                      const float tl = __bfloat162float(__float2bfloat16_rn(tp - th));
                      tc_self = f0h * th + f0h * tl + f0l * th;
                    }
                    *dst = __uint_as_float(r[q]) + (f0 * tp - tc_self);
                  } else if (seg_in_item == 0) {
                    *dst = __uint_as_float(r[q]);
                  } else {
                    *dst = *dst + __uint_as_float(r[q]);
                  }
                }
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(bar_tfree);
      }
      if (!ok) break;
    }
  }

  __syncthreads();
  if (tid == 0 && *abort_flag) report_device_error(args.status, DEV_ERR_TIMEOUT);
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
}

// M += sum of the partial sums of units 1 .. S-1 (fixed order: deterministic)
__global__ void add_partials_kernel(float *__restrict__ M, const float *__restrict__ P, int n_part, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float acc = M[i];
    for (int q = 0; q < n_part; ++q) acc += P[(size_t)q * n + i];
    M[i] = acc;
  }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

struct TcChoice {
  int KB, NS, KS;
};

template <int KB, int JP, bool SPLIT, int NS, int KS>
static tsr_status launch_tc(const TcArgs &a0, const uint8_t *rec, cudaStream_t s) {
  using C = TcCfg<KB, JP, SPLIT, NS, KS>;
  TcArgs a = a0;
  a.seg_stages = std::max(1, 4096 / (16 * KS));   // flush the tensor-core accumulator every 4,096 i
  a.n_kgroups = (a.K + KB - 1) / KB;
  a.n_items = a.n_otiles * a.n_kgroups;
  const size_t smem = C::smem_bytes(a.n_r);
  if (smem > 232448) {
    set_error("transfer_tc: shared memory %zu bytes exceeds the per-block limit (n_r too large)", smem);
    return TSR_ERR_UNSUPPORTED;
  }
  auto encode = get_encode();
  if (!encode) {
    set_error("transfer_tc: cuTensorMapEncodeTiled unavailable");
    return TSR_ERR_CUDA;
  }
  CUtensorMap tmap;
  const cuuint64_t rows_total = (cuuint64_t)a.n_steps * C::REC / 128;
  const cuuint64_t gdim[2] = {32, rows_total};
  const cuuint64_t gstride[1] = {128};
  const cuuint32_t box[2] = {32, (cuuint32_t)(C::REC_STAGE / 128)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult cr = encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint8_t *>(rec), gdim, gstride, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    set_error("transfer_tc: cuTensorMapEncodeTiled failed (%d)", (int)cr);
    return TSR_ERR_CUDA;
  }
  auto kern = transfer_tc_kernel<KB, JP, SPLIT, NS, KS>;
  TSR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // Every CTA keeps one k-group: the grid is a multiple of the group count.  Each
  // tile's i-range is cut into S units so that the last wave is nearly full.
  const int G = a.n_kgroups;
  const int sms = num_sms();
  const int SPT = a.n_steps / KS;
  int best_S = 1;
  double best_cost = 1e30;
  for (int S = 1; S <= 4 && S <= SPT; ++S) {
    const long units = (long)a.n_otiles * S * G;
    int grid = (int)std::min<long>(units, sms);
    grid = std::max(G, grid / G * G);
    const long per_cta = (units / G + grid / G - 1) / (grid / G);        // units on the busiest CTA
    const double cost = (double)per_cta / S * (1.0 + 0.03 * (S - 1));    // in whole-tile units
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best_S = S;
    }
  }
  a.n_split = best_S;
  const long units = (long)a.n_otiles * best_S * G;
  int grid = (int)std::min<long>(units, sms);
  grid = std::max(G, grid / G * G);
  Scratch part;
  const size_t mn = (size_t)a.K * a.J * a.N;
  a.P = nullptr;
  if (best_S > 1) {
    tsr_status st = part.alloc(sizeof(float) * mn * (best_S - 1), s);
    if (st != TSR_OK) return st;
    a.P = static_cast<float *>(part.p);
  }
  kern<<<grid, C::NTHREADS, smem, s>>>(tmap, a);
  TSR_CUDA(cudaGetLastError());
  if (best_S > 1) {
    add_partials_kernel<<<4 * sms, 256, 0, s>>>(a.M, a.P, best_S - 1, mn);
    TSR_CUDA(cudaGetLastError());
  }
  return TSR_OK;
}

// Configuration per (K, J_pad, split): bases per item, pipeline stages, steps per stage.
static tsr_status dispatch_tc(const TcArgs &a, int JP, bool split, const uint8_t *rec, cudaStream_t s) {
  const int K = a.K;
  if (!split) {
    if (JP == 16) {
      if (K <= 4) return launch_tc<4, 16, false, 4, 2>(a, rec, s);
      if (K <= 8) return launch_tc<8, 16, false, 4, 1>(a, rec, s);
      if (K <= 12) return launch_tc<12, 16, false, 3, 1>(a, rec, s);
      return launch_tc<16, 16, false, 2, 1>(a, rec, s);
    } else {
      if (K <= 4) return launch_tc<4, 32, false, 4, 2>(a, rec, s);
      if (K <= 8) return launch_tc<8, 32, false, 4, 1>(a, rec, s);
      if (K <= 12) return launch_tc<12, 32, false, 3, 1>(a, rec, s);
      return launch_tc<16, 32, false, 2, 1>(a, rec, s);
    }
  } else {
    if (JP == 16) {
      if (K <= 4) return launch_tc<4, 16, true, 4, 1>(a, rec, s);
      return launch_tc<8, 16, true, 2, 1>(a, rec, s);
    } else {
      if (K <= 4) return launch_tc<4, 32, true, 4, 1>(a, rec, s);
      return launch_tc<8, 32, true, 2, 1>(a, rec, s);
    }
  }
}

tsr_status transfer_tc(const tsr_basis *b, int N, const float *pos, const float *area, const float *T, int J,
                       bool split, float *M, cudaStream_t s) {
  const int JP = J <= 16 ? 16 : 32;
  const int KS_MAX = 2;
  const int n_steps = ((N + 15) / 16 + KS_MAX - 1) / KS_MAX * KS_MAX;
  const int REC = rec_bytes(JP, split);
  Scratch rs;
  tsr_status st = rs.alloc((size_t)n_steps * REC, s);
  if (st != TSR_OK) return st;
  uint8_t *rec = static_cast<uint8_t *>(rs.p);
  TSR_CUDA(cudaMemsetAsync(rec, 0, (size_t)n_steps * REC, s));
  pretile_tc_kernel<<<(n_steps * 16 + 255) / 256, 256, 0, s>>>(pos, area, T, N, J, JP, split ? 1 : 0, REC, n_steps,
                                                                rec);
  TSR_CUDA(cudaGetLastError());
  TcArgs a{};
  a.N = N;
  a.n_steps = n_steps;
  a.n_r = b->n_r;
  a.inv_dr = static_cast<float>((b->n_r - 1) / b->r_max);
  a.r2max = static_cast<float>(b->r_max * b->r_max);
  a.K = b->K;
  a.J = J;
  a.n_otiles = (N + 127) / 128;
  a.pos = pos;
  a.area = area;
  a.T = T;
  a.tab16 = b->tab16;
  a.tab32 = b->tab32;
  a.KP = b->KP;
  a.M = M;
  a.status = device_status_ptr();
  return dispatch_tc(a, JP, split, rec, s);
}

// Batched transfer over independent meshes: one launch per mesh, in order.
tsr_status transfer_fp32_batched(const tsr_basis *b, int n_mesh, const int64_t *offsets, const float *pos,
                                 const float *area, const float *T, int J, float *M, cudaStream_t s) {
  (void)b; (void)n_mesh; (void)offsets; (void)pos; (void)area; (void)T; (void)J; (void)M; (void)s;
  set_error("batched FP32 transfer not built yet");
  return TSR_ERR_UNSUPPORTED;
}
tsr_status transfer_tc_batched(const tsr_basis *b, int n_mesh, const int64_t *offsets, const float *pos,
                               const float *area, const float *T, int J, float *M, cudaStream_t s) {
  (void)b; (void)n_mesh; (void)offsets; (void)pos; (void)area; (void)T; (void)J; (void)M; (void)s;
  set_error("batched BF16 transfer not built yet");
  return TSR_ERR_UNSUPPORTED;
}

}  // namespace tsr
