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
//    (the UMMA M = 128).  Per 16-i step, 512 generator threads write the A
//    operand (128 rows x 16 i, BF16) into tensor memory or shared memory, while
//    the Tensor Memory Accelerator streams the matching tile of
//    T'[j][i] = A_i T[j][i] (pre-tiled BF16 records that also carry the x_i), and
//    one warp issues tcgen05.mma with FP32 accumulators in tensor memory; the
//    epilogue reads TMEM back with tcgen05.ld and writes M.  Two generators:
//      - BF16 (default): the far field r >= r_e from the scaled Chebyshev series
//        of the basis (f_k(r) = sum_p c_kp W_p(r), W_p = sigma_p T_p(x) / r^2, 12
//        terms), the W_p evaluated in registers by a packed BF16 recurrence, the
//        accumulators holding G[p][j] = sum_i W_p T'[j][i] and the epilogue
//        forming M[k][j] = sum_p c_kp G[p][j]; the near field r < r_e is added
//        exactly in FP32 by near.cu;
//      - table (split BF16, and bases whose series is not accurate): F_k from
//        the shared-memory table of {value, slope} per radius sample.
//
// Pair geometry (every path): dx = fl(x_o - x_i) etc. and
// r2 = fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)) without contraction; pairs with
// r2 > fl(r_max^2) are cut off (f_k = 0).  Otherwise r = sqrt(r2),
// x = r / dr, m = min(floor(x), n_r - 2), t = x - m and
// f_k(r) = v_k[m] + t s_k[m] (s_k = f_k[m+1] - f_k[m]).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>
#include <string>
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
__global__ void pretile_fp32_kernel(const float *__restrict__ area, const float *__restrict__ T, int N, long long stride,
                                    int J, int JP, int n_pad, float *__restrict__ Tp) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_pad * JP) return;
  const int i = idx / JP, j = idx % JP;
  Tp[idx] = (i < N && j < J) ? area[i] * T[(size_t)j * stride + i] : 0.0f;
}

template <int JP>
__global__ void __launch_bounds__(256, 1)
    transfer_fp32_kernel(const float *__restrict__ pos, int N, long long stride, const float *__restrict__ Tp,
                         const float4 *__restrict__ tab, int KG, int n_r, float inv_dr, float r2max, int K,
                         int J, float *__restrict__ M, int n_tiles) {
  __shared__ __align__(16) float sT[F32_BI * JP];
  __shared__ float sx[F32_BI], sy[F32_BI], sz[F32_BI];
  const int kg = threadIdx.x % KG;
  const int ol = threadIdx.x / KG;
  const float *px = pos, *py = pos + stride, *pz = pos + 2 * stride;
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
          if (k0 < K) M[((size_t)k0 * J + j) * stride + o] = acc0[j];
          if (k1 < K) M[((size_t)k1 * J + j) * stride + o] = acc1[j];
        }
      }
    }
  }
}

template <int JP>
static cudaError_t launch_fp32(int grid, int threads, cudaStream_t s, const float *pos, int N, long long stride,
                               const float *Tp, const float4 *tab, int KG, int n_r, float inv_dr, float r2max, int K,
                               int J, float *M, int n_tiles) {
  transfer_fp32_kernel<JP><<<grid, threads, 0, s>>>(pos, N, stride, Tp, tab, KG, n_r, inv_dr, r2max, K, J, M, n_tiles); ::tsr::count_launch();
  return cudaGetLastError();
}

tsr_status transfer_fp32(const tsr_basis *b, int N, const float *pos, const float *area, const float *T, int J,
                         float *M, cudaStream_t s, long long stride) {
  if (stride <= 0) stride = N;
  const int JP = (J + 3) & ~3;
  const int n_pad = (N + F32_BI - 1) / F32_BI * F32_BI;
  Scratch tp;
  tsr_status st = tp.alloc(sizeof(float) * (size_t)n_pad * JP, s);
  if (st != TSR_OK) return st;
  float *Tp = static_cast<float *>(tp.p);
  pretile_fp32_kernel<<<(n_pad * JP + 255) / 256, 256, 0, s>>>(area, T, N, stride, J, JP, n_pad, Tp); ::tsr::count_launch();
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
  case JPV: e = launch_fp32<JPV>(grid, threads, s, pos, N, stride, Tp, tab, KG, b->n_r, inv_dr, r2max, b->K, J, M, n_tiles); break;
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

// Writes entry ii of record `step` for vertex i of a mesh whose arrays start at
// vertex 0 of `pos`/`area`/`T` with row stride `stride` (ok = false: padding).
__device__ __forceinline__ void pretile_entry(const float *__restrict__ pos, const float *__restrict__ area,
                                              const float *__restrict__ T, long long stride, int J, int JP, int split,
                                              int REC, int step, int ii, int i, bool ok, uint8_t *__restrict__ rec) {
  uint8_t *r = rec + (size_t)step * REC;
  const float a = ok ? area[i] : 0.0f;
  const int h = ii / 8, e = ii % 8;
  for (int j = 0; j < JP; ++j) {
    const float v = (ok && j < J) ? a * T[(size_t)j * stride + i] : 0.0f;
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
  p[16 + ii] = ok ? pos[stride + i] : 0.0f;
  p[32 + ii] = ok ? pos[2 * stride + i] : 0.0f;
}

__global__ void pretile_tc_kernel(const float *__restrict__ pos, const float *__restrict__ area,
                                  const float *__restrict__ T, int N, int J, int JP, int split, int REC,
                                  int n_steps, uint8_t *__restrict__ rec) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // (step, ii)
  if (idx >= n_steps * 16) return;
  const int step = idx / 16, ii = idx % 16;
  const int i = step * 16 + ii;
  pretile_entry(pos, area, T, N, J, JP, split, REC, step, ii, i, i < N, rec);
}

// Records of concatenated meshes: mesh b owns records [mesh_soff[b], mesh_soff[b+1]).
__global__ void pretile_tc_batched_kernel(const float *__restrict__ pos, const float *__restrict__ area,
                                          const float *__restrict__ T, long long stride, int J, int JP, int split,
                                          int REC, int n_steps, const int *__restrict__ mesh_soff, int n_mesh,
                                          const int *__restrict__ mesh_N, const long long *__restrict__ mesh_voff,
                                          uint8_t *__restrict__ rec) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_steps * 16) return;
  const int step = idx / 16, ii = idx % 16;
  int lo = 0, hi = n_mesh;   // mesh_soff[lo] <= step < mesh_soff[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (mesh_soff[mid] <= step) lo = mid; else hi = mid;
  }
  const int i = (step - mesh_soff[lo]) * 16 + ii;
  const long long v = mesh_voff[lo];
  pretile_entry(pos + v, area + v, T + v, stride, J, JP, split, REC, step, ii, i, i < mesh_N[lo], rec);
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



// Warp-collective forms: every lane of the warp executes them with the same
// operands, and the lane chosen by elect.sync issues the instruction.
__device__ __forceinline__ void umma_bf16_elect(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                                uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_bf16_ta_elect(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                                   uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// Four MMAs of consecutive columns groups (accumulators d0 + c JP, A tiles a0 + 8 c, c < 4)
// under one elect.sync, all with the same B tile and accumulate flag.
template <int JP>
__device__ __forceinline__ void umma4_ta(uint32_t d0, uint32_t a0, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\t.reg .b32 d, a;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t"
      "add.u32 d, %0, %5;\n\tadd.u32 a, %1, 8;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [d], [a], %2, %3, p;\n\t"
      "add.u32 d, %0, %6;\n\tadd.u32 a, %1, 16;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [d], [a], %2, %3, p;\n\t"
      "add.u32 d, %0, %7;\n\tadd.u32 a, %1, 24;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [d], [a], %2, %3, p;\n\t}" ::"r"(d0),
      "r"(a0), "l"(b), "r"(idesc), "r"(acc), "n"(JP), "n"(2 * JP), "n"(3 * JP)
      : "memory");
}
__device__ __forceinline__ void umma_commit_elect(uint64_t *bar) {
  asm volatile(
      "{\n\t.reg .pred e;\n\t"
      "elect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_st2(uint32_t taddr, uint32_t a, uint32_t b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }


__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
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

// hi/lo BF16 split of four consecutive-i values; hi tile at addr, lo tile at addr + lo_off
__device__ __forceinline__ void store_split4(uint32_t addr, uint32_t lo_off, float f0, float f1, float f2, float f3) {
  const __nv_bfloat162 h01 = __floats2bfloat162_rn(f0, f1), h23 = __floats2bfloat162_rn(f2, f3);
  const float2 g01 = __bfloat1622float2(h01), g23 = __bfloat1622float2(h23);
  const __nv_bfloat162 l01 = __floats2bfloat162_rn(f0 - g01.x, f1 - g01.y), l23 = __floats2bfloat162_rn(f2 - g23.x, f3 - g23.y);
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(*reinterpret_cast<const uint32_t *>(&h01)),
               "r"(*reinterpret_cast<const uint32_t *>(&h23))
               : "memory");
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr + lo_off), "r"(*reinterpret_cast<const uint32_t *>(&l01)),
               "r"(*reinterpret_cast<const uint32_t *>(&l23))
               : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// ---------------------------------------------------------------- the kernel
// One pipeline, three generators of the A operand (128 output rows x 16 i per step):
//  * MODE_NEAR:      A[o][i] = f_k(r_oi), k in the CTA's group of CB bases, from the
//    shared-memory table, written to shared memory (canonical K-major layout);
//  * MODE_NEAR_TMEM: the same values written to tensor memory (tcgen05.st); the
//    MMA reads A from TMEM.  Warp w owns TMEM lanes (rows) 32 (w mod 4) .. +31 and
//    i-quarter w / 4 of every step;
//  * MODE_CHEB:      A[o][i] = W_p(r_oi), p < CB = 12, the scaled Chebyshev terms of
//    the far field, in tensor memory; the accumulators hold
//    G[p][j] = sum_i W_p(r_oi) T'[j][i] and the epilogue forms M[k][j] = sum_p c_kp G[p][j].
//    The warps form CONC = NS groups, one per A slot (group g takes the steps s with
//    s mod CONC = g and visits only those), so that steps are written while the tensor
//    core consumes earlier ones: one group of 16 warps with 4 i per thread, or two or
//    three groups of 8 warps with 8 i per thread (three: 24 generator warps at 72
//    registers, the default);
//  * MODE_CHEB_S:    the same terms written to shared memory (canonical K-major layout, one
//    16-byte store per term and thread) for the MMA to read from there, so that tensor
//    memory holds only the accumulators (at J_pad = 32, 12 x 32 accumulator columns);
//  * MODE_CHEB_H:    hybrid: the first PT terms of a step in the tensor-memory columns
//    left beside the accumulators, the other CB - PT in shared memory, so that the
//    shared-memory data path carries only part of the A traffic (written once by the
//    generators, read once by the MMAs); the default at J_pad = 32.
// Table modes take the pairs with rn2 <= r^2 <= r_max^2 (rn2 = 0 when no separate
// near field is added: the self pair is then replaced in FP32 by the epilogue);
// the series modes take the same far pairs, whose near complement near.cu adds in FP32.
enum { MODE_NEAR = 0, MODE_CHEB = 1, MODE_NEAR_TMEM = 2, MODE_CHEB_S = 3, MODE_CHEB_H = 4 };
__host__ __device__ constexpr bool is_series(int mode) {
  return mode == MODE_CHEB || mode == MODE_CHEB_S || mode == MODE_CHEB_H;
}
// Terms per A slot that the hybrid layout keeps in tensor memory: what the 512 columns hold
// beside CB x JP accumulators for NS slots of 8 columns per term.
__host__ __device__ constexpr int hybrid_terms(int CB, int JP, int NS) {
  return (512 - CB * JP) / (8 * NS) < CB ? (512 - CB * JP) / (8 * NS) : CB;
}

struct TcArgs {
  int N;             // vertices (rows o and columns i)
  int n_steps;       // 16-i records
  int n_r;           // radius samples
  float inv_dr, r2max;
  const float *rn2;  // [n_mesh] near radius^2 of each mesh (NULL: 0, every pair in this pass)
  int self_fix;      // table modes: the epilogue replaces the self pair's BF16 product by FP32
  int K, J, KP;
  int n_otiles, n_groups, n_split;
  const float *pos;  // [3][N] (rows o)
  const float *area; // [N]      (self pair, FP32 epilogue)
  const float *T;    // [J][N]   (self pair, FP32 epilogue)
  const uint32_t *tab16;   // [n_r + 1][KP] bf16x2
  const float2 *tab32;     // [n_r + 1][KP]
  const float *cheb;       // [K][PCH]
  int PCH;
  float x_alpha, x_beta;
  int seg_stages;    // stages per accumulation segment (TMEM flushed after each)
  int accumulate;    // destination 0 (M) is accumulated into instead of overwritten
  float *M;          // [K][J][N]
  float *P;          // [n_dest - 1][K][J][N] partial sums (NULL if one destination)
  // Stream-K split (streamk_P > 0, one mesh, no near lists): CTA p of its group takes
  // the stages [p T / P, (p+1) T / P) of the tile-major stage space (T = n_otiles n_steps).
  // The piece of a tile that starts at its first stage writes M; a piece that starts
  // inside a tile (only the first piece of a CTA) writes the CTA's slot, which a fix-up
  // kernel adds to M in CTA order.
  int streamk_P;
  float *slots;      // [G][P][K][J][128]
  unsigned *status;
  // Batched meshes (units != NULL): arrays are concatenated along the vertex axis
  // with row stride `stride`; unit u = (mesh, tile, split, splits of that mesh).
  const int4 *units;
  int n_units_total;
  const int *mesh_N;
  const long long *mesh_voff;   // first vertex of each mesh
  const int *mesh_soff;         // first record of each mesh
  long long stride;             // total vertices (= N for one mesh)
};

// Everything a CTA needs to know about one unit of work.
struct Unit {
  int t, sp, sb, se;   // tile, split, stage range [sb, se)
  int mesh;            // mesh of the unit (0: one mesh)
  int Nb;              // vertices of the unit's mesh
  long long voff;      // first vertex of the mesh
  int soff;            // first record of the mesh
};

template <int MODE, int CB, int JP, bool SPLIT, int NS>
struct TcCfg {
  static constexpr int LOOKAHEAD = 8;                      // records in flight ahead of the generators
  static constexpr int CONC = is_series(MODE) ? NS : 1;   // generator groups (steps in flight)
  static constexpr int NR = NS + LOOKAHEAD;                // record slots
  static constexpr int REC = rec_bytes(JP, SPLIT);
  static constexpr bool ATMEM = (MODE == MODE_NEAR_TMEM || MODE == MODE_CHEB);
  static constexpr bool HYB = MODE == MODE_CHEB_H;
  static constexpr int PT = HYB ? hybrid_terms(CB, JP, NS) : (ATMEM ? CB : 0);   // A terms in TMEM
  static constexpr bool TABLE = (MODE == MODE_NEAR || MODE == MODE_NEAR_TMEM);
  static constexpr int A_TILE = 128 * 16 * 2;              // one (column, 16-i step) BF16 tile
  static constexpr int A_STAGE = ATMEM ? 0 : (CB - PT) * (SPLIT ? 2 : 1) * A_TILE;
  static constexpr int REC_STAGE = REC;
  static constexpr int TAB_ELEM = TABLE ? (SPLIT ? 8 : 4) : 0;
  static constexpr int U = TABLE ? CB * TAB_ELEM / 16 : 1;   // 16-byte units per table row
  // generator threads: 16 warps, or for the series modes with NS >= 2 one group of 8 warps per A slot
  static constexpr int NGEN = (is_series(MODE) && NS >= 2) ? 256 * NS : 512;
  static constexpr int NTHREADS = NGEN + 64;               // + the MMA-issue warp and the TMA warp
  static_assert(NTHREADS <= 1024, "at most 1024 threads per block");
  static constexpr int ACC_COLS = CB * JP;                 // FP32 accumulators
  static constexpr int A_COLS = PT * 8;                    // A tiles of one stage in TMEM (16 BF16 per row = 8 columns)
  static constexpr int USED_COLS = ACC_COLS + NS * A_COLS;
  static constexpr int TMEM_COLS = (USED_COLS <= 32) ? 32 : (USED_COLS <= 64) ? 64 : (USED_COLS <= 128) ? 128
                                 : (USED_COLS <= 256) ? 256 : 512;
  static_assert(USED_COLS <= 512, "tensor memory holds 512 columns");
  static size_t smem_bytes(int n_r, int K) {
    return 1024 + (size_t)NS * A_STAGE + (size_t)NR * REC_STAGE + (size_t)(n_r + 1) * CB * TAB_ELEM +
           (is_series(MODE) ? (size_t)K * CB * sizeof(float) : 0) + 512;
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


__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One run of W consecutive 32-bit TMEM columns of this thread's lane (W = 2 or 4).
template <int W>
__device__ __forceinline__ void tmem_st_run(uint32_t taddr, const uint32_t (&v)[W]) {
  if constexpr (W == 2) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(v[0]), "r"(v[1]) : "memory");
  } else {
    static_assert(W == 4, "runs of 2 or 4 columns");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
  }
}

__device__ __forceinline__ float fast_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Two FP32 lanes per instruction (add/sub/mul/fma .rn.f32x2): each lane rounds exactly as
// the scalar instruction, so results are bit-identical to the scalar code.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Decodes unit u.  One mesh: u = tile * S + split, stages over all records (or
// over the tile's near-chunk list); batched: the unit table.
__device__ __forceinline__ Unit decode_unit(int u, int S, int SPT, int N, const int4 *units, const int *mesh_N,
                                            const long long *mesh_voff, const int *mesh_soff) {
  Unit r;
  if (units) {
    const int4 d = units[u];
    r.t = d.y;
    r.sp = d.z;
    r.mesh = d.x;
    r.Nb = mesh_N[d.x];
    r.voff = mesh_voff[d.x];
    r.soff = mesh_soff[d.x];
    const int spt = (r.Nb + 15) / 16;
    r.sb = d.z * spt / d.w;
    r.se = (d.z + 1) * spt / d.w;
    return r;
  }
  r.t = u / S;
  r.sp = u % S;
  r.mesh = 0;
  r.Nb = N;
  r.voff = 0;
  r.soff = 0;
  r.sb = r.sp * SPT / S;
  r.se = (r.sp + 1) * SPT / S;
  return r;
}

template <int MODE, int CB, int JP, bool SPLIT, int NS>
__global__ void __launch_bounds__(TcCfg<MODE, CB, JP, SPLIT, NS>::NTHREADS, 1)
    transfer_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs args) {
  using C = TcCfg<MODE, CB, JP, SPLIT, NS>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // align by pointer arithmetic on the shared array (keeps the shared address space: LDS/STS, not generic)
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *sA = smem;                                   // NS * A_STAGE
  uint8_t *sRec = sA + (size_t)NS * C::A_STAGE;         // NR * REC_STAGE
  uint8_t *sTab = sRec + (size_t)C::NR * C::REC_STAGE;  // (n_r+1) * CB * TAB_ELEM   (MODE_NEAR)
  float *sC = reinterpret_cast<float *>(sTab + (size_t)(args.n_r + 1) * CB * C::TAB_ELEM);   // [K][CB] (MODE_CHEB)
  uint64_t *bar = reinterpret_cast<uint64_t *>(
      reinterpret_cast<uint8_t *>(sC) + (is_series(MODE) ? (((size_t)args.K * CB * 4 + 15) / 16) * 16 : 0));
  uint64_t *bar_tma = bar;                        // [NR] records landed
  uint64_t *bar_full = bar + C::NR;               // [NS] A stage written by its generator group
  uint64_t *bar_mma = bar + C::NR + NS;           // [NS] MMAs of a stage completed
  uint64_t *bar_tfree = bar + C::NR + 2 * NS;     // [1]  epilogue finished reading TMEM
  uint64_t *bar_seg = bar + C::NR + 2 * NS + 1;   // [1]  MMAs of an accumulation segment completed (MODE_CHEB)
  uint64_t *bar_rfree = bar + C::NR + 2 * NS + 2; // [NR] MMAs that read a record slot completed
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar + 2 * C::NR + 2 * NS + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  // Each CTA keeps one column group (bases or Chebyshev columns): CTA b takes
  // group b % G and units b / G, b / G + grid / G, ... of that group.
  const int G = args.n_groups;
  const int group = blockIdx.x % G;
  const int c0 = group * CB;        // first basis (table modes) or Chebyshev column (MODE_CHEB)
  const int S = args.n_split;
  const int SPT = args.n_steps;     // stages of a whole tile (one 16-i record per stage)
  const int SKP = args.streamk_P;
  const int cta_in_group = blockIdx.x / G;
  long long sk0 = 0, sk1 = 0;   // stream-K stage range of this CTA
  int sk_t0 = 0;                // its first tile
  int unit_first, unit_step, n_units;
  if (SKP > 0) {
    const long long T_st = (long long)args.n_otiles * SPT;
    sk0 = T_st * cta_in_group / SKP;
    sk1 = T_st * (cta_in_group + 1) / SKP;
    sk_t0 = (int)(sk0 / SPT);
    unit_first = 0;
    unit_step = 1;
    n_units = sk1 > sk0 ? (int)((sk1 - 1) / SPT) - sk_t0 + 1 : 0;
  } else {
    unit_first = cta_in_group;
    unit_step = gridDim.x / G;
    n_units = args.units ? args.n_units_total : args.n_otiles * S;
  }
  const int4 *const units = args.units;
  const int *const mesh_N = args.mesh_N;
  const long long *const mesh_voff = args.mesh_voff;
  const int *const mesh_soff = args.mesh_soff;
  const long long stride = args.stride;
  // stream-K: piece u of this CTA's stage range (sp = 1: starts inside its tile -> slot)
  auto streamk_unit = [&](int u) {
    Unit r;
    r.t = sk_t0 + u;
    const long long base = (long long)r.t * SPT;
    r.sb = (int)((sk0 > base ? sk0 : base) - base);
    r.se = (int)((sk1 < base + SPT ? sk1 : base + SPT) - base);
    r.sp = r.sb > 0 ? 1 : 0;
    r.mesh = 0;
    r.Nb = args.N;
    r.voff = 0;
    r.soff = 0;
    return r;
  };
#define TSR_UNIT(u) \
  (SKP > 0 ? streamk_unit(u) : decode_unit((u), S, SPT, args.N, units, mesh_N, mesh_voff, mesh_soff))
  const int seg_stages = args.seg_stages;
  const size_t KJN = (size_t)args.K * args.J * (size_t)stride;

  if (tid == 0) {
    for (int q = 0; q < C::NR; ++q) mbar_init(&bar_tma[q], 1);
    for (int q = 0; q < NS; ++q) {
      mbar_init(&bar_full[q], C::NGEN / C::CONC);
      mbar_init(&bar_mma[q], 1);
    }
    mbar_init(bar_tfree, C::NGEN);
    mbar_init(bar_seg, 1);
    for (int q = 0; q < C::NR; ++q) mbar_init(&bar_rfree[q], 1);
    *abort_flag = 0;
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  if (C::TABLE) {
    // this group's table slice (zero beyond K), rows swizzled by tab_unit
    const int n_units_tab = (args.n_r + 1) * C::U;
    for (int q = tid; q < n_units_tab; q += blockDim.x) {
      const int m = q / C::U, u = q % C::U;
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      if (!SPLIT) {
        uint32_t e4[4] = {0u, 0u, 0u, 0u};   // {lo: v_k, hi: s_k} per base
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = c0 + u * 4 + e;
          if (k < args.K) e4[e] = args.tab16[(size_t)m * args.KP + k];
        }
        w[0] = __byte_perm(e4[0], e4[1], 0x5410);   // {v_k, v_k+1}
        w[1] = __byte_perm(e4[2], e4[3], 0x5410);   // {v_k+2, v_k+3}
        w[2] = __byte_perm(e4[0], e4[1], 0x7632);   // {s_k, s_k+1}
        w[3] = __byte_perm(e4[2], e4[3], 0x7632);   // {s_k+2, s_k+3}
      } else {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k = c0 + u * 2 + e;
          if (k < args.K) {
            const float2 f = args.tab32[(size_t)m * args.KP + k];
            w[2 * e] = __float_as_uint(f.x);
            w[2 * e + 1] = __float_as_uint(f.y);
          }
        }
      }
      reinterpret_cast<uint4 *>(sTab)[tab_unit<C::U>(m, u)] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    for (int q = tid; q < args.K * CB; q += blockDim.x) {
      const int k = q / CB, p = c0 + q % CB;
      sC[q] = (p < args.PCH) ? args.cheb[k * args.PCH + p] : 0.f;
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

  if (warp == C::NGEN / 32 + 1) {
    // ------------------------------------------------------------ TMA warp
    // Streams the records of this CTA's stages in order into the NR record slots; a slot
    // is refilled once the MMAs that read its previous record have completed (bar_rfree).
    long issued = 0;
    int slot = 0;
    uint32_t ph = 0u;   // use parity of the slot
    bool run = true;
    for (int u = unit_first; u < n_units && run; u += unit_step) {
      const Unit un = TSR_UNIT(u);
      for (int q = un.sb; q < un.se; ++q) {
        if (issued >= C::NR && !__all_sync(0xffffffffu, wait_or_abort(&bar_rfree[slot], ph ^ 1u, abort_flag))) {
          run = false;
          break;
        }
        if (lane == 0) {
          mbar_arrive_expect_tx(&bar_tma[slot], C::REC_STAGE);
          tma_load_2d(sRec + (size_t)slot * C::REC_STAGE, &tmap, &bar_tma[slot], 0, (un.soff + q) * rows_per_stage);
        }
        __syncwarp();
        ++issued;
        if (++slot == C::NR) {
          slot = 0;
          ph ^= 1u;
        }
      }
    }
    __syncwarp();
    if (lane == 0 && *abort_flag) {   // let the copies still in flight land before the CTA exits
      for (long q = issued > C::NR ? issued - C::NR : 0; q < issued; ++q) {
        for (uint32_t it = 0; it < TSR_WAIT_LIMIT; ++it)
          if (mbar_try_wait(&bar_tma[q % C::NR], (uint32_t)((q / C::NR) & 1))) break;
      }
    }
    __syncwarp();
  } else if (warp == C::NGEN / 32) {
    // ------------------------------------------------------------ MMA warp
    // All 32 lanes run the loop on warp-uniform state, so the MMA operands stay in
    // uniform registers; one elected lane issues each group of MMAs and each commit.
    const uint32_t idesc = umma_idesc_bf16(JP);
    const uint64_t desc_a0 = umma_desc(smem_u32(sA), 128, 256);             // A: K-major, 8x16B core matrices
    const uint64_t desc_b0 = umma_desc(smem_u32(sRec), JP * 16, 128);       // B: T' tile of a record
    auto wait_warp = [&](uint64_t *b, uint32_t parity) {
      return __all_sync(0xffffffffu, wait_or_abort(b, parity, abort_flag));
    };
    int sa = 0, sr = 0;
    uint32_t pa = 0u;
    int seg_no = 0;   // accumulation segments issued so far
    bool run = true;
    for (int u = unit_first; u < n_units && run; u += unit_step) {
      const Unit un = TSR_UNIT(u);
      const int sb = un.sb, se = un.se;
      int seg_pos = 0;
      for (int sidx = sb; sidx < se; ++sidx) {
        const bool seg_start = seg_pos == 0;
        if (++seg_pos == seg_stages) seg_pos = 0;
        const bool seg_end = seg_pos == 0 || sidx + 1 == se;
        // the A tile of this stage is written (its record landed before that)
        if (!wait_warp(&bar_full[sa], pa)) {
          run = false;
          break;
        }
        // the epilogue of the previous segment must have read TMEM before it is overwritten
        if (seg_start && seg_no > 0 && !wait_warp(bar_tfree, (uint32_t)((seg_no - 1) & 1))) {
          run = false;
          break;
        }
        if (seg_start) ++seg_no;
        tc_fence_after();
        // descriptors: start-address field (addr >> 4) advanced by offsets from the base ones
        const uint64_t dbh = desc_b0 + (uint64_t)((sr * C::REC_STAGE) >> 4);
        const uint64_t dbl = dbh + (uint64_t)((JP * 32) >> 4);
        const uint64_t da = desc_a0 + (uint64_t)((sa * C::A_STAGE) >> 4);
        const uint32_t first = seg_start ? 0u : 1u;
        if constexpr (C::ATMEM) {
          const uint32_t a0 = tmem_base + (uint32_t)(C::ACC_COLS + sa * C::A_COLS);
#pragma unroll
          for (int cb = 0; cb < CB; cb += 4) umma4_ta<JP>(tmem_base + (uint32_t)(cb * JP), a0 + (uint32_t)(cb * 8), dbh, idesc, first);
        } else if constexpr (C::HYB) {
          const uint32_t a0 = tmem_base + (uint32_t)(C::ACC_COLS + sa * C::A_COLS);
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) {
            const uint32_t d = tmem_base + (uint32_t)(cb * JP);
            if (cb < C::PT) umma_bf16_ta_elect(d, a0 + (uint32_t)(cb * 8), dbh, idesc, first);
            else umma_bf16_elect(d, da + (uint64_t)(((cb - C::PT) * C::A_TILE) >> 4), dbh, idesc, first);
          }
        } else {
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) {
            const uint32_t d = tmem_base + (uint32_t)(cb * JP);
            if (!SPLIT) {
              umma_bf16_elect(d, da + (uint64_t)((cb * C::A_TILE) >> 4), dbh, idesc, first);
            } else {
              const uint64_t dah = da + (uint64_t)(((2 * cb) * C::A_TILE) >> 4);
              const uint64_t dal = da + (uint64_t)(((2 * cb + 1) * C::A_TILE) >> 4);
              umma_bf16_elect(d, dah, dbh, idesc, first);
              umma_bf16_elect(d, dah, dbl, idesc, 1u);
              umma_bf16_elect(d, dal, dbh, idesc, 1u);
            }
          }
        }
        umma_commit_elect(&bar_mma[sa]);     // the A slot may be rewritten
        umma_commit_elect(&bar_rfree[sr]);   // the record slot may be refilled
        if (is_series(MODE) && seg_end) umma_commit_elect(bar_seg);   // the segment's accumulators are final
        if (++sa == NS) {
          sa = 0;
          pa ^= 1u;
        }
        if (++sr == C::NR) sr = 0;
      }
    }
    __syncwarp();
  } else if constexpr (is_series(MODE)) {
    // ------------------------------------------------------------ generator warps, far-field series
    // Warp w: TMEM lane quarter w mod 4 (rows 32 (w mod 4) + lane), group w / GW (the
    // steps s with s mod CONC = group), run (w mod GW) / 4 of IPT consecutive i of the step.
    // One group: 16 warps, 4 i per thread; two or three groups: 8 warps each, 8 i per thread.
    constexpr int CONC = C::CONC, GW = CONC >= 2 ? 8 : 16, IPT = 64 / GW, NWD = IPT / 2;
    constexpr bool SMEM_A = MODE == MODE_CHEB_S, HYB = C::HYB;
    constexpr int PT = C::PT;
    static_assert(!(SMEM_A || HYB) || NWD == 4, "shared-memory A: 8 i per thread (two or three generator groups)");
    const int quarter = warp & 3, grp = warp / GW, ih = (warp % GW) >> 2;
    const int orow = quarter * 32 + lane;
    const uint32_t a_tmem_row =
        tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(C::ACC_COLS + ih * NWD);
    // shared-memory A: the thread's row and 8-i K chunk in the canonical K-major layout (8 x 16 B
    // core matrices, K chunks 128 B apart, 8-row groups 256 B apart), one 16-byte store per term
    const uint32_t a_smem_row =
        smem_u32(sA) + (uint32_t)((orow >> 3) * 256 + ih * 128 + (orow & 7) * 16);
    const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
    const float r2max = args.r2max, xa_alpha = args.x_alpha, xa_beta = args.x_beta;
    const uint64_t alpha2 = f2_pack(xa_alpha, xa_alpha), beta2 = f2_pack(xa_beta, xa_beta);
    // Ring state of this group's steps (steps grp, grp + CONC, ...): A slot sa (phase pa),
    // record slot sr (phase pr); `own` counts down to this group's next step.
    int sa = grp % NS, sr = grp % C::NR, own = grp;
    uint32_t pa = 0u, pr = 0u;
    bool first_use = true;   // the A slot has not been used yet
    int seg_done = 0;        // accumulation segments finished by this CTA
    for (int u = unit_first; u < n_units; u += unit_step) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const Unit un = TSR_UNIT(u);
      const int t = un.t, sp = un.sp, sb = un.sb, se = un.se, Nb = un.Nb;
      if (sb == se) continue;
      const int d_idx = sp;
      const bool to_M = SKP > 0 ? sp == 0 : d_idx == 0;
      float *dbase;
      long long dld;
      if (SKP > 0 && sp != 0) {
        dbase = args.slots + (size_t)(group * SKP + cta_in_group) * args.K * args.J * 128;
        dld = 128;
      } else {
        dbase = ((d_idx == 0) ? args.M : args.P + (size_t)(d_idx - 1) * KJN) + un.voff + (size_t)t * 128;
        dld = stride;
      }
      const bool dst_accumulates = to_M && args.accumulate;
      const int o = t * 128 + orow;
      const bool o_ok = o < Nb;
      const float *pos_m = args.pos + un.voff;
      const float xo = o_ok ? pos_m[o] : 0.f;
      const float yo = o_ok ? pos_m[stride + o] : 0.f;
      const float zo = o_ok ? pos_m[2 * stride + o] : 0.f;
      const uint64_t xo2 = f2_pack(xo, xo), yo2 = f2_pack(yo, yo), zo2 = f2_pack(zo, zo);
      const float rlo2 = args.rn2 ? args.rn2[un.mesh] : 0.f;   // below: the exact near field
      bool ok = true;
      int seg_count = 0;
      for (int s0 = sb; s0 < se; s0 += seg_stages) {
        // accumulation segment [s0, s0 + n_seg): this group's steps s0 + own, s0 + own + CONC, ...
        const int n_seg = min(se - s0, seg_stages);
        int q = own;
        for (; q < n_seg; q += CONC) {
          if (__any_sync(0xffffffffu, !wait_or_abort(&bar_tma[sr], pr, abort_flag))) {
            ok = false;
            break;
          }
          const float *rp = reinterpret_cast<const float *>(sRec + (size_t)sr * C::REC_STAGE + JP * 32);
          // W_0 = s, W_1 = x s, W_p = (-1)^(p-1) 2x W_{p-1} + W_{p-2}, s = 1/r^2 (0 outside the far
          // field), two consecutive i per packed BF16 word: the word layout of the A operand in TMEM.
          uint32_t w0[NWD], w1[NWD], mp[NWD], mn[NWD];
#pragma unroll
          for (int h = 0; h < NWD; h += 2) {
            const float4 xs = *reinterpret_cast<const float4 *>(rp + ih * IPT + 2 * h);
            const float4 ys = *reinterpret_cast<const float4 *>(rp + 16 + ih * IPT + 2 * h);
            const float4 zs = *reinterpret_cast<const float4 *>(rp + 32 + ih * IPT + 2 * h);
            const float xa[4] = {xs.x, xs.y, xs.z, xs.w}, ya[4] = {ys.x, ys.y, ys.z, ys.w},
                        za[4] = {zs.x, zs.y, zs.z, zs.w};
            float sv[4], xsv[4], x2v[4];
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {   // two i per packed instruction, as pair_r2 rounds
              const int q0 = 2 * e2;
              const uint64_t dx = f2_sub(xo2, f2_pack(xa[q0], xa[q0 + 1]));
              const uint64_t dy = f2_sub(yo2, f2_pack(ya[q0], ya[q0 + 1]));
              const uint64_t dz = f2_sub(zo2, f2_pack(za[q0], za[q0 + 1]));
              float r2[2];
              f2_unpack(f2_add(f2_add(f2_mul(dx, dx), f2_mul(dy, dy)), f2_mul(dz, dz)), r2[0], r2[1]);
              bool far[2];
              float lg[2], rc[2];
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                far[e] = r2[e] >= rlo2 && r2[e] <= r2max;
                // lg2 and rcp run on every pair (no branch); a pair outside the far field
                // gets s = 0, which zeroes all of its terms whatever x is
                const float rf = far[e] ? r2[e] : 1.f;
                lg[e] = fast_lg2(rf);
                rc[e] = rcp_approx(rf);
              }
              const uint64_t x = f2_fma(alpha2, f2_pack(lg[0], lg[1]), beta2);
              const uint64_t s2 = f2_pack(far[0] ? rc[0] : 0.f, far[1] ? rc[1] : 0.f);
              f2_unpack(s2, sv[q0], sv[q0 + 1]);
              f2_unpack(f2_mul(x, s2), xsv[q0], xsv[q0 + 1]);
              f2_unpack(f2_add(x, x), x2v[q0], x2v[q0 + 1]);
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              mp[h + e] = pack_bf16x2(x2v[2 * e], x2v[2 * e + 1]);
              mn[h + e] = mp[h + e] ^ 0x80008000u;
              w0[h + e] = pack_bf16x2(sv[2 * e], sv[2 * e + 1]);
              w1[h + e] = pack_bf16x2(xsv[2 * e], xsv[2 * e + 1]);
            }
          }
          const uint32_t a_slot = a_tmem_row + (uint32_t)(sa * C::A_COLS);
          if constexpr (HYB) {
            // terms p < PT to tensor memory, the others to shared memory, as the recurrence
            // produces them (the slot's previous MMAs completed CONC steps back)
            if (!first_use && __any_sync(0xffffffffu, !wait_or_abort(&bar_mma[sa], pa ^ 1u, abort_flag))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_st = a_smem_row + (uint32_t)(sa * C::A_STAGE) - (uint32_t)(PT * C::A_TILE);
            auto put = [&](int p, const uint32_t (&w)[NWD]) {
              if (p < PT) tmem_st_run<NWD>(a_slot + (uint32_t)(p * 8), w);
              else st_shared_v4(a_st + (uint32_t)(p * C::A_TILE), w[0], w[1], w[2], w[3]);
            };
            put(0, w0);
            put(1, w1);
#pragma unroll
            for (int p = 2; p < CB; ++p) {
              uint32_t w2[NWD];
#pragma unroll
              for (int h = 0; h < NWD; ++h) w2[h] = bf16x2_fma((p & 1) ? mp[h] : mn[h], w1[h], w0[h]);
              put(p, w2);
#pragma unroll
              for (int h = 0; h < NWD; ++h) {
                w0[h] = w1[h];
                w1[h] = w2[h];
              }
            }
          } else if constexpr (SMEM_A) {
            // the slot's previous MMAs (CONC steps back) completed long ago: wait, then store
            // the terms as the recurrence produces them
            if (!first_use && __any_sync(0xffffffffu, !wait_or_abort(&bar_mma[sa], pa ^ 1u, abort_flag))) {
              ok = false;
              break;
            }
            const uint32_t a_st = a_smem_row + (uint32_t)(sa * C::A_STAGE);
            st_shared_v4(a_st, w0[0], w0[1], w0[2], w0[3]);
            st_shared_v4(a_st + C::A_TILE, w1[0], w1[1], w1[2], w1[3]);
#pragma unroll
            for (int p = 2; p < CB; ++p) {
              uint32_t w2[NWD];
#pragma unroll
              for (int h = 0; h < NWD; ++h) w2[h] = bf16x2_fma((p & 1) ? mp[h] : mn[h], w1[h], w0[h]);
              st_shared_v4(a_st + (uint32_t)(p * C::A_TILE), w2[0], w2[1], w2[2], w2[3]);
#pragma unroll
              for (int h = 0; h < NWD; ++h) {
                w0[h] = w1[h];
                w1[h] = w2[h];
              }
            }
          } else if constexpr (NS >= 2) {
            // the slot's previous MMAs (CONC steps back) completed long ago: wait, then stream
            // the terms to TMEM as the recurrence produces them (few live registers)
            if (!first_use && __any_sync(0xffffffffu, !wait_or_abort(&bar_mma[sa], pa ^ 1u, abort_flag))) {
              ok = false;
              break;
            }
            tc_fence_after();
            tmem_st_run<NWD>(a_slot, w0);
            tmem_st_run<NWD>(a_slot + 8u, w1);
#pragma unroll
            for (int p = 2; p < CB; ++p) {
              uint32_t w2[NWD];
#pragma unroll
              for (int h = 0; h < NWD; ++h) w2[h] = bf16x2_fma((p & 1) ? mp[h] : mn[h], w1[h], w0[h]);
              tmem_st_run<NWD>(a_slot + (uint32_t)(p * 8), w2);
#pragma unroll
              for (int h = 0; h < NWD; ++h) {
                w0[h] = w1[h];
                w1[h] = w2[h];
              }
            }
          } else {
            // one A slot: the previous step's MMAs may still be running, so every term is
            // formed in registers before the wait
            uint32_t feat[CB][NWD];
#pragma unroll
            for (int h = 0; h < NWD; ++h) {
              feat[0][h] = w0[h];
              feat[1][h] = w1[h];
            }
#pragma unroll
            for (int p = 2; p < CB; ++p)
#pragma unroll
              for (int h = 0; h < NWD; ++h) feat[p][h] = bf16x2_fma((p & 1) ? mp[h] : mn[h], feat[p - 1][h], feat[p - 2][h]);
            if (!first_use && __any_sync(0xffffffffu, !wait_or_abort(&bar_mma[sa], pa ^ 1u, abort_flag))) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int p = 0; p < CB; ++p) tmem_st_run<NWD>(a_slot + (uint32_t)(p * 8), feat[p]);
          }
          if constexpr (HYB) {
            fence_proxy_async_smem();   // the shared-memory stores, before the tensor core reads them
            tmem_st_wait();
            tc_fence_before();
          } else if constexpr (SMEM_A) {
            fence_proxy_async_smem();   // the stores, before the tensor core reads them
          } else {
            tmem_st_wait();
            tc_fence_before();
          }
          mbar_arrive(&bar_full[sa]);
          // advance this group's ring by CONC steps
          sa += CONC;
          if (sa >= NS) {
            sa -= NS;
            pa ^= 1u;
            first_use = false;
          }
          sr += CONC;
          if (sr >= C::NR) {
            sr -= C::NR;
            pr ^= 1u;
          }
        }
        if (!ok) break;
        own = q - n_seg;   // steps of the next segment before this group's next one
        // End of an accumulation segment (every warp): M[k][j] (+)= sum_p c_kp G[p][j] for
        // 2 k x 8 j per item, G read from TMEM two terms at a time.
        const bool first_seg = seg_count == 0;
        ++seg_count;
        const bool e_ok = wait_or_abort(bar_seg, (uint32_t)(seg_done & 1), abort_flag);
        ++seg_done;
        if (__any_sync(0xffffffffu, !e_ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int wq = warp >> 2;   // 4 warps share a lane quarter
        const int oe = t * 128 + quarter * 32 + lane;
        const bool oe_ok = oe < Nb;
        const int n_kc = (args.K + 1) / 2;
        for (int item = wq; item < n_kc * (JP / 8); item += C::NGEN / 128) {
          const int kc = item / (JP / 8), jc = (item % (JP / 8)) * 8;
          const int ka = kc * 2, kb = kc * 2 + 1;
          float acc0[8], acc1[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) acc0[q] = acc1[q] = 0.f;
#pragma unroll
          for (int cb0 = 0; cb0 < CB; cb0 += 2) {
            uint32_t r[2][8];
#pragma unroll
            for (int v = 0; v < 2; ++v) tmem_ld8(lane_base + (uint32_t)((cb0 + v) * JP + jc), r[v]);
            tmem_ld_wait();
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              const float ca = sC[ka * CB + cb0 + v];
              const float cbv = (kb < args.K) ? sC[kb * CB + cb0 + v] : 0.f;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                acc0[q] = fmaf(ca, __uint_as_float(r[v][q]), acc0[q]);
                acc1[q] = fmaf(cbv, __uint_as_float(r[v][q]), acc1[q]);
              }
            }
          }
          if (oe_ok) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int j = jc + q;
              if (j < args.J) {
                float *da = dbase + ((size_t)ka * args.J + j) * dld + (oe - t * 128);
                *da = (first_seg && !dst_accumulates) ? acc0[q] : *da + acc0[q];
                if (kb < args.K) {
                  float *db = dbase + ((size_t)kb * args.J + j) * dld + (oe - t * 128);
                  *db = (first_seg && !dst_accumulates) ? acc1[q] : *db + acc1[q];
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
  } else {
    // ------------------------------------------------------------ generator warps, table
    // Thread (orow, h4): output row orow of the tile, i = 4*h4 .. 4*h4+3 of every 16-i step.
    // A warp covers 16 rows x two neighbouring i-quarters, so its 8-byte stores fill
    // two whole 128-byte core matrices (2 shared-memory wavefronts per store).
    const int orow = C::ATMEM ? (warp & 3) * 32 + lane : (warp & 7) * 16 + (lane & 7) + ((lane >> 4) << 3);
    const int h4 = C::ATMEM ? (warp >> 2) : (warp >> 3) * 2 + ((lane >> 3) & 1);
    const uint32_t a_tmem_row = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(C::ACC_COLS + 2 * h4);
    const uint32_t a_row_off =
        (uint32_t)((orow >> 3) * 256 + (h4 >> 1) * 128 + (orow & 7) * 16 + (h4 & 1) * 8);
    const uint32_t sA_u32 = smem_u32(sA);
    const float r2max = args.r2max, inv_dr2 = args.inv_dr * args.inv_dr;
    const int n_r = args.n_r;
    long g = 0;
    // ring state (advanced once per stage): A slot sa with phase bit pa = (g / NS) & 1,
    // record slot sr with phase bit pr = (g / NR) & 1
    int sa = 0, sr = 0;
    uint32_t pa = 0u, pr = 0u;
    for (int u = unit_first; u < n_units; u += unit_step) {
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
      const Unit un = TSR_UNIT(u);
      const int t = un.t, sp = un.sp, sb = un.sb, se = un.se, Nb = un.Nb;
      if (sb == se) continue;
      const int d_idx = sp;   // destination (equal splits)
      // destination base shifted to the unit's mesh (rows voff .. voff + Nb - 1)
      // destination of this unit: element (k, j, row r of the tile) at dbase + (k J + j) dld + r
      const bool to_M = SKP > 0 ? sp == 0 : d_idx == 0;
      float *dbase;
      long long dld;
      if (SKP > 0 && sp != 0) {
        dbase = args.slots + (size_t)(group * SKP + cta_in_group) * args.K * args.J * 128;
        dld = 128;
      } else {
        dbase = ((d_idx == 0) ? args.M : args.P + (size_t)(d_idx - 1) * KJN) + un.voff + (size_t)t * 128;
        dld = stride;
      }
      const bool dst_accumulates = to_M && args.accumulate;
      const int o = t * 128 + orow;
      const bool o_ok = o < Nb;
      const float *pos_m = args.pos + un.voff;
      const float xo = o_ok ? pos_m[o] : 0.f;
      const float yo = o_ok ? pos_m[stride + o] : 0.f;
      const float zo = o_ok ? pos_m[2 * stride + o] : 0.f;
      const float rlo2 = args.rn2 ? args.rn2[un.mesh] : 0.f;   // pairs below it: the separate near field
      bool ok = true;
      int seg_pos = 0, seg_count = 0;   // position in / index of the accumulation segment
      for (int sidx = sb; sidx < se; ++sidx) {
        bool w_ok = true;
        if (g >= NS) w_ok = wait_or_abort(&bar_mma[sa], pa ^ 1u, abort_flag);
        if (w_ok) w_ok = wait_or_abort(&bar_tma[sr], pr, abort_flag);
        if (__any_sync(0xffffffffu, !w_ok)) {
          ok = false;
          break;
        }
        if (C::ATMEM) tc_fence_after();    // the MMAs that read this A slot have completed
        const uint8_t *rec_stage = sRec + (size_t)sr * C::REC_STAGE;
        const float *rp = reinterpret_cast<const float *>(rec_stage + JP * 32 * (SPLIT ? 2 : 1));
        const float4 xs = *reinterpret_cast<const float4 *>(rp + h4 * 4);
        const float4 ys = *reinterpret_cast<const float4 *>(rp + 16 + h4 * 4);
        const float4 zs = *reinterpret_cast<const float4 *>(rp + 32 + h4 * 4);
        const float xa[4] = {xs.x, xs.y, xs.z, xs.w}, ya[4] = {ys.x, ys.y, ys.z, ys.w},
                    za[4] = {zs.x, zs.y, zs.z, zs.w};
        // Padded i (beyond N) carry T' = 0 and finite positions, so they add nothing.
        // r^2 in the exact FP32 order of the definition: the cutoff and the near/far
        // split are decided on the same value the reference computes.
        float r2v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) r2v[q] = pair_r2(xo, yo, zo, xa[q], ya[q], za[q]);
        const uint32_t a_stage = sA_u32 + (uint32_t)(sa * C::A_STAGE);
        if (C::TABLE) {
          int row[4];
          float tq[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float r2 = r2v[q];
            const float x = sqrt_approx(r2 * inv_dr2);   // r / dr
            const int m = __float2int_rd(x);
            tq[q] = x - __int2float_rn(m);
            row[q] = (r2 >= rlo2 && r2 <= r2max) ? m : n_r;   // far pairs of this pass; the rest read the zero row
          }
          if (!SPLIT) {
            // unit cb4 of a table row: {v_4cb4..+1, v_+2..+3, s_4cb4..+1, s_+2..+3} (bf16 pairs)
            uint32_t t2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) t2[q] = pack_bf16x2(tq[q], tq[q]);
            const uint4 *tab4 = reinterpret_cast<const uint4 *>(sTab);
#pragma unroll
            for (int cb4 = 0; cb4 < CB / 4; ++cb4) {
              uint4 w[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) w[q] = tab4[tab_unit<C::U>(row[q], cb4)];
              uint32_t F01[4], F23[4];   // {F_k, F_k+1} of pair q
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                F01[q] = bf16x2_fma(t2[q], w[q].z, w[q].x);
                F23[q] = bf16x2_fma(t2[q], w[q].w, w[q].y);
              }
              if (C::ATMEM) {
                // columns 2 h4, 2 h4 + 1 of base (4 cb4 + b)'s 8-column A tile in slot sa
                const uint32_t ta = a_tmem_row + (uint32_t)(sa * C::A_COLS + cb4 * 32);
                tmem_st2(ta, __byte_perm(F01[0], F01[1], 0x5410), __byte_perm(F01[2], F01[3], 0x5410));
                tmem_st2(ta + 8, __byte_perm(F01[0], F01[1], 0x7632), __byte_perm(F01[2], F01[3], 0x7632));
                tmem_st2(ta + 16, __byte_perm(F23[0], F23[1], 0x5410), __byte_perm(F23[2], F23[3], 0x5410));
                tmem_st2(ta + 24, __byte_perm(F23[0], F23[1], 0x7632), __byte_perm(F23[2], F23[3], 0x7632));
              } else {
                const uint32_t base = a_stage + (uint32_t)(cb4 * 4 * C::A_TILE) + a_row_off;
                st_shared_v2(base, __byte_perm(F01[0], F01[1], 0x5410), __byte_perm(F01[2], F01[3], 0x5410));
                st_shared_v2(base + C::A_TILE, __byte_perm(F01[0], F01[1], 0x7632), __byte_perm(F01[2], F01[3], 0x7632));
                st_shared_v2(base + 2 * C::A_TILE, __byte_perm(F23[0], F23[1], 0x5410), __byte_perm(F23[2], F23[3], 0x5410));
                st_shared_v2(base + 3 * C::A_TILE, __byte_perm(F23[0], F23[1], 0x7632), __byte_perm(F23[2], F23[3], 0x7632));
              }
            }
          } else {
            const float4 *tab4 = reinterpret_cast<const float4 *>(sTab);   // {v_k, s_k, v_k+1, s_k+1}
#pragma unroll
            for (int cb2 = 0; cb2 < CB / 2; ++cb2) {
              float F0[4], F1[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float4 w = tab4[tab_unit<C::U>(row[q], cb2)];
                F0[q] = fmaf(tq[q], w.y, w.x);
                F1[q] = fmaf(tq[q], w.w, w.z);
              }
              store_split4(a_stage + (uint32_t)((4 * cb2) * C::A_TILE) + a_row_off, C::A_TILE, F0[0], F0[1], F0[2], F0[3]);
              store_split4(a_stage + (uint32_t)((4 * cb2 + 2) * C::A_TILE) + a_row_off, C::A_TILE, F1[0], F1[1], F1[2],
                           F1[3]);
            }
          }
        }
        if (C::ATMEM) {
          tmem_st_wait();     // this thread's A columns are written ...
          tc_fence_before();  // ... and ordered before the barrier the MMA issuer waits on
        } else {
          fence_proxy_async_smem();
        }
        mbar_arrive(&bar_full[sa]);
        const int last_sa = sa;
        const uint32_t last_pa = pa;
        ++g;
        if (++sa == NS) {
          sa = 0;
          pa ^= 1u;
        }
        if (++sr == C::NR) {
          sr = 0;
          pr ^= 1u;
        }
        if (++seg_pos != seg_stages && sidx + 1 != se) continue;
        // End of an accumulation segment: TMEM -> registers -> destination.  The
        // tensor-core FP32 accumulator is flushed every seg_stages steps and summed
        // with round-to-nearest adds.
        const bool first_seg = seg_count == 0;
        seg_pos = 0;
        ++seg_count;
        const bool e_ok = wait_or_abort(&bar_mma[last_sa], last_pa, abort_flag);
        if (__any_sync(0xffffffffu, !e_ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int quarter = warp & 3, wq = warp >> 2;   // rows quarter*32 + lane; 4 warps share a quarter
        const int oe = t * 128 + quarter * 32 + lane;
        const bool oe_ok = oe < Nb;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        if (C::TABLE) {
          // The first segment of split 0 also replaces the self pair's BF16 product
          // (exact in FP32) by f_k(0) A_o T[j][o] in FP32.
          const float a_o = oe_ok ? args.area[un.voff + oe] : 0.f;
          for (int cb = wq; cb < CB; cb += C::NGEN / 128) {
            const int k = c0 + cb;
            const float f0 = (k < args.K) ? args.tab32[k].x : 0.f;   // f_k(0), FP32
            const float f0h = __bfloat162float(__float2bfloat16_rn(f0));
            const float f0l = __bfloat162float(__float2bfloat16_rn(f0 - f0h));
#pragma unroll
            for (int jc = 0; jc < JP; jc += 16) {
              uint32_t r[16];
              tmem_ld16(lane_base + (uint32_t)(cb * JP + jc), r);
              tmem_ld_wait();
              if (k < args.K && oe_ok) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                  const int j = jc + q;
                  if (j < args.J) {
                    float *dst = dbase + ((size_t)k * args.J + j) * dld + (oe - t * 128);
                    float v = __uint_as_float(r[q]);
                    if (first_seg && to_M && args.self_fix) {
                      const float tpv = a_o * args.T[(size_t)j * stride + un.voff + oe];
                      const float th = __bfloat162float(__float2bfloat16_rn(tpv));
                      float tc_self;
                      if (!SPLIT) {
                        tc_self = __bfloat162float(__ushort_as_bfloat16((unsigned short)(args.tab16[k] & 0xFFFFu))) * th;
                      } else {
                        const float tl = __bfloat162float(__float2bfloat16_rn(tpv - th));
                        tc_self = f0h * th + f0h * tl + f0l * th;
                      }
                      v += f0 * tpv - tc_self;
                    }
                    *dst = (first_seg && !dst_accumulates) ? v : *dst + v;
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

// Stream-K fix-up: block (g, p) leads when CTA p's stage range starts inside a tile and
// CTA p - 1's does not start inside the same tile; it adds the slots p, p+1, ... of that
// tile (in CTA order) to M for the bases of group g.
__global__ void streamk_fixup_kernel(float *__restrict__ M, const float *__restrict__ slots, int n_tiles, int SPT,
                                     int P, int CB, int K, int J, int N, long long stride) {
  const int g = blockIdx.x / P, p = blockIdx.x % P;
  const long long T_st = (long long)n_tiles * SPT;
  const long long s0 = T_st * p / P;
  if (s0 % SPT == 0) return;
  const long long t = s0 / SPT;
  if (p > 0 && T_st * (p - 1) / P > t * SPT) return;
  int p_end = p + 1;
  while (p_end < P && T_st * p_end / P < (t + 1) * SPT) ++p_end;
  const int k0 = g * CB, k1 = min(K, k0 + CB);
  const long long left = (long long)N - t * 128;
  const int rows = left < 128 ? (int)left : 128;
  const int n_el = (k1 - k0) * J * 128;
  constexpr int U = 4;   // elements per thread in flight
  for (int e0 = threadIdx.x; e0 < n_el; e0 += U * blockDim.x) {
    float acc[U];
    float *dst[U];
    size_t soff[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      const int row = e % 128, kj = e / 128;
      const bool ok = e < n_el && row < rows;
      const int k = k0 + kj / J, j = kj % J;
      dst[u] = ok ? M + ((size_t)k * J + j) * stride + t * 128 + row : nullptr;
      soff[u] = ((size_t)k * J + j) * 128 + row;
      acc[u] = ok ? *dst[u] : 0.f;
    }
    for (int q = p; q < p_end; ++q) {
      const float *sl = slots + (size_t)(g * P + q) * K * J * 128;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (dst[u]) acc[u] += sl[soff[u]];
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (dst[u]) *dst[u] = acc[u];
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

static tsr_status make_record_map(CUtensorMap *tmap, const uint8_t *rec, int n_steps, int REC) {
  auto encode = get_encode();
  if (!encode) {
    set_error("transfer_tc: cuTensorMapEncodeTiled unavailable");
    return TSR_ERR_CUDA;
  }
  const cuuint64_t gdim[2] = {32, (cuuint64_t)n_steps * REC / 128};
  const cuuint64_t gstride[1] = {128};
  const cuuint32_t box[2] = {32, (cuuint32_t)(REC / 128)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult cr = encode(tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint8_t *>(rec), gdim, gstride, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    set_error("transfer_tc: cuTensorMapEncodeTiled failed (%d)", (int)cr);
    return TSR_ERR_CUDA;
  }
  return TSR_OK;
}

// Launch one pass.  n_cols: bases (table modes) or Chebyshev terms (MODE_CHEB) in total.
template <int MODE, int CB, int JP, bool SPLIT, int NS>
static tsr_status launch_tc(const TcArgs &a0, int n_cols, const CUtensorMap &tmap, bool allow_split, cudaStream_t s) {
  using C = TcCfg<MODE, CB, JP, SPLIT, NS>;
  TcArgs a = a0;
  // The tensor-core FP32 accumulation does not round to nearest, so long sums are cut
  // into segments that the epilogue adds with round-to-nearest FP32 adds.
  a.seg_stages = (is_series(MODE) ? 16384 : 4096) / 16;
  a.n_groups = (n_cols + CB - 1) / CB;
  const size_t smem = C::smem_bytes(a.n_r, a.K);
  if (smem > 232448) {
    set_error("transfer_tc: shared memory %zu bytes exceeds the per-block limit (n_r too large)", smem);
    return TSR_ERR_UNSUPPORTED;
  }
  auto kern = transfer_tc_kernel<MODE, CB, JP, SPLIT, NS>;
  TSR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // Every CTA keeps one group: the grid is a multiple of the group count.
  const int G = a.n_groups;
  const int sms = num_sms();
  a.n_split = 1;
  const long units = (a.units ? (long)a.n_units_total : (long)a.n_otiles) * G;
  int grid = (int)std::min<long>(units, sms);
  grid = std::max(G, grid / G * G);
  // Stream-K for one mesh over all its records: equal stage ranges per CTA.
  const bool streamk = allow_split && !a.units;
  Scratch slots;
  if (streamk) {
    const long long T_st = (long long)a.n_otiles * a.n_steps;
    int P = std::max(1, sms / G);
    P = (int)std::min<long long>(P, std::max<long long>(1, T_st / 64));   // at least 64 stages per CTA
    a.streamk_P = P;
    grid = G * P;
    tsr_status st = slots.alloc(sizeof(float) * (size_t)G * P * a.K * a.J * 128, s);
    if (st != TSR_OK) return st;
    a.slots = static_cast<float *>(slots.p);
  }
  a.P = nullptr;
  KernelTimer timer(s);
  kern<<<grid, C::NTHREADS, smem, s>>>(tmap, a); ::tsr::count_launch();
  timer.stop();
  TSR_CUDA(cudaGetLastError());
  if (streamk) {
    streamk_fixup_kernel<<<G * a.streamk_P, 1024, 0, s>>>(a.M, a.slots, a.n_otiles, a.n_steps, a.streamk_P,
                                                          is_series(MODE) ? a.K : CB, a.K, a.J, a.N, a.stride);
    ::tsr::count_launch();
    TSR_CUDA(cudaGetLastError());
  }
  return TSR_OK;
}

// The table generator.  kb: bases per CTA group (4, 8, 12 or 16; 0 = the smallest
// group holding all K).
static bool atmem_enabled() {
  const char *e = std::getenv("TSR_TRANSFER_ATMEM");   // "0": A operand staged in shared memory
  return !(e && e[0] == '0');
}

static tsr_status dispatch_table(const TcArgs &a, int JP, bool split, const CUtensorMap &tmap, bool allow_split,
                                 cudaStream_t s, int kb = 0, int atmem = -1) {
  const int K = a.K;
  if (atmem < 0) atmem = atmem_enabled() ? 1 : 0;
  // A in tensor memory when the bases of a group and 2..4 A stages fit in 512 columns
  // next to the accumulators without splitting K further than the default grouping
  // (with J_pad = 32 only K <= 8 does; more groups would recompute every r).
  if (!split && atmem && (JP == 16 || (kb ? kb : K) <= 8)) {
    const int g = kb ? kb : (K <= 4 ? 4 : K <= 8 ? 8 : K <= 12 ? 12 : 16);
    if (JP == 16) {
      if (g == 4) return launch_tc<MODE_NEAR_TMEM, 4, 16, false, 4>(a, K, tmap, allow_split, s);
      if (g == 8) return launch_tc<MODE_NEAR_TMEM, 8, 16, false, 4>(a, K, tmap, allow_split, s);
      if (g == 12) return launch_tc<MODE_NEAR_TMEM, 12, 16, false, 3>(a, K, tmap, allow_split, s);
      return launch_tc<MODE_NEAR_TMEM, 16, 16, false, 2>(a, K, tmap, allow_split, s);
    }
    if (g == 4) return launch_tc<MODE_NEAR_TMEM, 4, 32, false, 4>(a, K, tmap, allow_split, s);
    return launch_tc<MODE_NEAR_TMEM, 8, 32, false, 3>(a, K, tmap, allow_split, s);
  }
  if (!split) {
    const int g = kb ? kb : (K <= 4 ? 4 : K <= 8 ? 8 : K <= 12 ? 12 : 16);
    if (JP == 16) {
      if (g == 4) return launch_tc<MODE_NEAR, 4, 16, false, 4>(a, K, tmap, allow_split, s);
      if (g == 8) return launch_tc<MODE_NEAR, 8, 16, false, 4>(a, K, tmap, allow_split, s);
      if (g == 12) return launch_tc<MODE_NEAR, 12, 16, false, 3>(a, K, tmap, allow_split, s);
      return launch_tc<MODE_NEAR, 16, 16, false, 2>(a, K, tmap, allow_split, s);
    }
    if (g == 4) return launch_tc<MODE_NEAR, 4, 32, false, 4>(a, K, tmap, allow_split, s);
    if (g == 8) return launch_tc<MODE_NEAR, 8, 32, false, 4>(a, K, tmap, allow_split, s);
    if (g == 12) return launch_tc<MODE_NEAR, 12, 32, false, 3>(a, K, tmap, allow_split, s);
    return launch_tc<MODE_NEAR, 16, 32, false, 2>(a, K, tmap, allow_split, s);
  }
  if (JP == 16) {
    if (K <= 4) return launch_tc<MODE_NEAR, 4, 16, true, 4>(a, K, tmap, allow_split, s);
    return launch_tc<MODE_NEAR, 8, 16, true, 2>(a, K, tmap, allow_split, s);
  }
  if (K <= 4) return launch_tc<MODE_NEAR, 4, 32, true, 4>(a, K, tmap, allow_split, s);
  return launch_tc<MODE_NEAR, 8, 32, true, 2>(a, K, tmap, allow_split, s);
}

// The far-field series generator (TSR_CHEB_BF16 terms).  conc: generator groups (steps
// written concurrently; three groups of 8 warps by default, 24 generator warps at 72
// registers).  With J_pad = 32 the accumulators take 384 of the 512 TMEM columns, which
// leaves room for one whole A slot in TMEM only: there each group's slot holds its first
// terms in the 128 free TMEM columns (5 of 12 with three slots) and the rest in shared
// memory (TSR_CHEB_HYB=0: every term in shared memory; TSR_CHEB_SMEM=0: the single TMEM
// slot).  With J_pad = 16 the A slots sit in TMEM beside the accumulators
// (TSR_CHEB_SMEM=1: in shared memory).
static tsr_status dispatch_cheb(const TcArgs &a, int JP, const CUtensorMap &tmap, bool allow_split, cudaStream_t s,
                                int conc = 0) {
  if (conc == 0) {
    const char *e = std::getenv("TSR_CHEB_CONC");   // diagnostic: "1", "2" or "3" steps in flight
    conc = (e && e[0] >= '1' && e[0] <= '3') ? e[0] - '0' : 3;
  }
  const char *e = std::getenv("TSR_CHEB_SMEM");   // diagnostic: "0" A in TMEM, "1" A in shared memory
  const int smem_a = (e && (e[0] == '0' || e[0] == '1')) ? e[0] - '0' : -1;
  if (JP == 16) {
    if (conc == 1) return launch_tc<MODE_CHEB, TSR_CHEB_BF16, 16, false, 1>(a, TSR_CHEB_BF16, tmap, allow_split, s);
    if (smem_a == 1) {
      if (conc == 3) return launch_tc<MODE_CHEB_S, TSR_CHEB_BF16, 16, false, 3>(a, TSR_CHEB_BF16, tmap, allow_split, s);
      return launch_tc<MODE_CHEB_S, TSR_CHEB_BF16, 16, false, 2>(a, TSR_CHEB_BF16, tmap, allow_split, s);
    }
    if (conc == 3) return launch_tc<MODE_CHEB, TSR_CHEB_BF16, 16, false, 3>(a, TSR_CHEB_BF16, tmap, allow_split, s);
    return launch_tc<MODE_CHEB, TSR_CHEB_BF16, 16, false, 2>(a, TSR_CHEB_BF16, tmap, allow_split, s);
  }
  if (smem_a == 0 || conc == 1)
    return launch_tc<MODE_CHEB, TSR_CHEB_BF16, 32, false, 1>(a, TSR_CHEB_BF16, tmap, allow_split, s);
  const char *h = std::getenv("TSR_CHEB_HYB");   // diagnostic: "0" every A term in shared memory
  if (!(h && h[0] == '0')) {
    if (conc == 3) return launch_tc<MODE_CHEB_H, TSR_CHEB_BF16, 32, false, 3>(a, TSR_CHEB_BF16, tmap, allow_split, s);
    return launch_tc<MODE_CHEB_H, TSR_CHEB_BF16, 32, false, 2>(a, TSR_CHEB_BF16, tmap, allow_split, s);
  }
  if (conc == 3) return launch_tc<MODE_CHEB_S, TSR_CHEB_BF16, 32, false, 3>(a, TSR_CHEB_BF16, tmap, allow_split, s);
  return launch_tc<MODE_CHEB_S, TSR_CHEB_BF16, 32, false, 2>(a, TSR_CHEB_BF16, tmap, allow_split, s);
}

// "table": the BF16 transfer uses the table generator even where the series is accurate
// (a diagnostic switch for comparing the two generators on the same inputs).
static bool bf16_table_forced() {
  const char *e = std::getenv("TSR_BF16_GENERATOR");
  return e && std::string(e) == "table";
}

static void fill_common_args(TcArgs &a, const tsr_basis *b, int J) {
  a.n_r = b->n_r;
  a.inv_dr = static_cast<float>((b->n_r - 1) / b->r_max);
  a.r2max = static_cast<float>(b->r_max * b->r_max);
  a.K = b->K;
  a.J = J;
  a.KP = b->KP;
  a.tab16 = b->tab16;
  a.tab32 = b->tab32;
  a.cheb = b->cheb;
  a.PCH = TSR_CHEB_P;
  a.x_alpha = b->x_alpha;
  a.x_beta = b->x_beta;
  a.status = device_status_ptr();
}

tsr_status transfer_tc(const tsr_basis *b, int N, const float *pos, const float *area, const float *T, int J,
                       bool split, float *M, cudaStream_t s) {
  const int JP = J <= 16 ? 16 : 32;
  const int n_steps = (N + 15) / 16;
  const int REC = rec_bytes(JP, split);
  Scratch rs;
  tsr_status st = rs.alloc((size_t)n_steps * REC, s);
  if (st != TSR_OK) return st;
  uint8_t *rec = static_cast<uint8_t *>(rs.p);
  TSR_CUDA(cudaMemsetAsync(rec, 0, (size_t)n_steps * REC, s));
  pretile_tc_kernel<<<(n_steps * 16 + 255) / 256, 256, 0, s>>>(pos, area, T, N, J, JP, split ? 1 : 0, REC, n_steps,
                                                                rec); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  CUtensorMap tmap;
  st = make_record_map(&tmap, rec, n_steps, REC);
  if (st != TSR_OK) return st;
  TcArgs a{};
  fill_common_args(a, b, J);
  a.N = N;
  a.n_steps = n_steps;
  a.n_otiles = (N + 127) / 128;
  a.pos = pos;
  a.area = area;
  a.T = T;
  a.M = M;
  a.stride = N;
  if (split) {
    // split BF16: every pair through the table, the self pair replaced in FP32
    a.rn2 = nullptr;
    a.self_fix = 1;
    return dispatch_table(a, JP, true, tmap, true, s);
  }
  // BF16: the far field on the tensor cores, the near field r < r_e exactly in FP32
  NearField nf;
  st = near_setup(nf, b, 1, nullptr, N, pos, N, area, T, J, s);
  if (st != TSR_OK) return st;
  a.rn2 = nf.rn2;
  a.self_fix = 0;
  st = (b->cheb_ok && !bf16_table_forced()) ? dispatch_cheb(a, JP, tmap, true, s) : dispatch_table(a, JP, false, tmap, true, s);
  if (st != TSR_OK) return st;
  return near_apply(nf, b, M, N, s);
}

// Batched transfer over independent meshes of uneven size: one persistent launch
// whose units are the (mesh, 128-row tile) pairs in longest-first order, each CTA
// taking every grid-th unit (so every CTA gets a similar mix of long and short
// units).  The plan holds the unit and mesh tables on the device; running it only
// enqueues kernels and stream-ordered scratch, so it can be captured in a CUDA graph.
tsr_status batch_plan_create(const tsr_basis *b, int n_mesh, const int64_t *offsets, int J, int prec,
                             tsr_batch_plan **out) {
  int device = -1;
  TSR_CUDA(cudaGetDevice(&device));
  tsr_batch_plan *p = new tsr_batch_plan();
  p->device = device;
  p->basis = b;
  p->n_mesh = n_mesh;
  p->J = J;
  p->prec = prec;
  p->gen = b->cheb_ok ? 0 : 1;
  p->offsets.assign(offsets, offsets + n_mesh + 1);
  p->total = offsets[n_mesh];
  std::vector<int> Nm(n_mesh), soff(n_mesh + 1, 0);
  std::vector<long long> voff(n_mesh + 1);
  for (int m = 0; m < n_mesh; ++m) {
    Nm[m] = (int)(offsets[m + 1] - offsets[m]);
    voff[m] = offsets[m];
    soff[m + 1] = soff[m] + (Nm[m] + 15) / 16;
  }
  voff[n_mesh] = offsets[n_mesh];
  p->total_steps = soff[n_mesh];
  std::vector<int4> units;
  for (int m = 0; m < n_mesh; ++m)
    for (int t = 0; t < (Nm[m] + 127) / 128; ++t) units.push_back(make_int4(m, t, 0, 1));
  std::stable_sort(units.begin(), units.end(), [&](const int4 &x, const int4 &y) { return Nm[x.x] > Nm[y.x]; });
  p->n_units = (int)units.size();
  const size_t b_units = sizeof(int4) * units.size(), b_voff = sizeof(long long) * (n_mesh + 1),
               b_N = sizeof(int) * n_mesh, b_soff = sizeof(int) * (n_mesh + 1);
  cudaError_t e = cudaMalloc(&p->tables, b_units + b_voff + b_N + b_soff + 64);
  if (e == cudaSuccess) {
    uint8_t *t = static_cast<uint8_t *>(p->tables);
    p->d_units = reinterpret_cast<int4 *>(t);
    p->d_voff = reinterpret_cast<long long *>(t + b_units);
    p->d_N = reinterpret_cast<int *>(t + b_units + b_voff);
    p->d_soff = p->d_N + n_mesh;
    e = cudaMemcpy(p->d_units, units.data(), b_units, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_voff, voff.data(), b_voff, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_N, Nm.data(), b_N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_soff, soff.data(), b_soff, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    set_error("tsr_batch_plan_create: %s", cudaGetErrorString(e));
    cudaFree(p->tables);
    delete p;
    return e == cudaErrorMemoryAllocation ? TSR_ERR_OOM : TSR_ERR_CUDA;
  }
  *out = p;
  return TSR_OK;
}

tsr_status batch_plan_run(const tsr_batch_plan *p, const float *pos, const float *area, const float *T, float *M,
                          cudaStream_t s) {
  const tsr_basis *b = p->basis;
  if (p->prec == TSR_FP32) return transfer_fp32_batched(b, p->n_mesh, p->offsets.data(), pos, area, T, p->J, M, s);
  const int J = p->J;
  const int JP = J <= 16 ? 16 : 32;
  const int REC = rec_bytes(JP, false);
  Scratch rs;
  tsr_status st = rs.alloc((size_t)p->total_steps * REC, s);
  if (st != TSR_OK) return st;
  uint8_t *rec = static_cast<uint8_t *>(rs.p);
  TSR_CUDA(cudaMemsetAsync(rec, 0, (size_t)p->total_steps * REC, s));
  pretile_tc_batched_kernel<<<(p->total_steps * 16 + 255) / 256, 256, 0, s>>>(
      pos, area, T, p->total, J, JP, 0, REC, p->total_steps, p->d_soff, p->n_mesh, p->d_N, p->d_voff, rec);
  ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  CUtensorMap tmap;
  st = make_record_map(&tmap, rec, p->total_steps, REC);
  if (st != TSR_OK) return st;
  // the near field of every mesh (its own r_e), exactly in FP32, after the far field
  NearField nf;
  st = near_setup(nf, b, p->n_mesh, p->d_voff, p->total, pos, p->total, area, T, J, s);
  if (st != TSR_OK) return st;
  TcArgs a{};
  fill_common_args(a, b, J);
  a.N = 0;
  a.n_steps = 1;
  a.n_otiles = 0;
  a.pos = pos;
  a.area = area;
  a.T = T;
  a.M = M;
  a.rn2 = nf.rn2;
  a.self_fix = 0;
  a.units = p->d_units;
  a.n_units_total = p->n_units;
  a.mesh_N = p->d_N;
  a.mesh_voff = p->d_voff;
  a.mesh_soff = p->d_soff;
  a.stride = p->total;
  st = (p->gen == 0 && b->cheb_ok) ? dispatch_cheb(a, JP, tmap, false, s, p->conc)
                                   : dispatch_table(a, JP, false, tmap, false, s, p->kb);
  if (st != TSR_OK) return st;
  return near_apply(nf, b, M, p->total, s);
}

// Times every generator configuration once on the caller's data and keeps the fastest
// in the plan: the far-field series with three or two steps in flight (and one at J_pad = 16), and the
// table with 4, 8, 12 or 16 bases per CTA group.  Synchronises the stream; not for use
// inside a capture.
tsr_status batch_plan_autotune(tsr_batch_plan *p, const float *pos, const float *area, const float *T, float *M,
                               cudaStream_t s, float *best_ms) {
  if (p->prec == TSR_FP32) {
    if (best_ms) *best_ms = 0.f;
    return TSR_OK;
  }
  struct Cand { int gen, conc, kb; };
  std::vector<Cand> cands;
  if (p->basis->cheb_ok) {
    cands.push_back({0, 3, 0});
    cands.push_back({0, 2, 0});
    if (p->J <= 16) cands.push_back({0, 1, 0});
  }
  for (int kb : {4, 8, 12, 16}) cands.push_back({1, 0, kb});
  cudaEvent_t e0, e1;
  TSR_CUDA(cudaEventCreate(&e0));
  TSR_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  Cand best_c = cands[0];
  for (const Cand &c : cands) {
    p->gen = c.gen;
    p->conc = c.conc;
    p->kb = c.kb;
    tsr_status st = batch_plan_run(p, pos, area, T, M, s);   // warm
    if (st == TSR_OK) {
      TSR_CUDA(cudaEventRecord(e0, s));
      st = batch_plan_run(p, pos, area, T, M, s);
      TSR_CUDA(cudaEventRecord(e1, s));
    }
    if (st != TSR_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return st;
    }
    TSR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    TSR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->gen = best_c.gen;
  p->conc = best_c.conc;
  p->kb = best_c.kb;
  if (best_ms) *best_ms = best;
  return TSR_OK;
}

tsr_status transfer_tc_batched(const tsr_basis *b, int n_mesh, const int64_t *offsets, const float *pos,
                               const float *area, const float *T, int J, float *M, cudaStream_t s) {
  tsr_batch_plan *p = nullptr;
  tsr_status st = batch_plan_create(b, n_mesh, offsets, J, TSR_BF16, &p);
  if (st != TSR_OK) return st;
  st = batch_plan_run(p, pos, area, T, M, s);
  const cudaError_t e = cudaStreamSynchronize(s);   // the plan's tables are freed below
  cudaFree(p->tables);
  delete p;
  if (st == TSR_OK && e != cudaSuccess) {
    set_error("transfer_tc_batched: %s", cudaGetErrorString(e));
    st = TSR_ERR_CUDA;
  }
  return st;
}

// FP32 batched: one launch per mesh on the strided concatenated arrays.
tsr_status transfer_fp32_batched(const tsr_basis *b, int n_mesh, const int64_t *offsets, const float *pos,
                                 const float *area, const float *T, int J, float *M, cudaStream_t s) {
  const long long total = offsets[n_mesh];
  for (int m = 0; m < n_mesh; ++m) {
    const long long v = offsets[m];
    const tsr_status st = transfer_fp32(b, (int)(offsets[m + 1] - v), pos + v, area + v, T + v, J, M + v, s, total);
    if (st != TSR_OK) return st;
  }
  return TSR_OK;
}

}  // namespace tsr
