// Exact FP32 near field of the BF16 transfer (Section 3, Eq. 6-7).
//
// The BF16 tensor-core transfer rounds every kernel value F_k[o,i] to 8 bits of
// mantissa.  Where a few close pairs carry much of M[k][.][o] (coarse meshes, or a
// basis whose near and far parts cancel), those roundings do not average out.  So
// the pairs with r_oi^2 < r_e^2 are taken out of the BF16 contraction and summed
// here in FP32, with the FP32 table of f_k and T'[j][i] = A_i T[j][i] in FP32:
//     M[k][j][o] += sum_{i : r_oi^2 < r_e^2, r_oi^2 <= r_max^2} A_i f_k(r_oi) T[j][i],
// r_e = max(r_floor, 2 h), h^2 = (sum_i A_i) / N the mean cell area of the mesh
// (r_floor is the lower end of the far-field series, r_max / 16).  The split is
// decided on the FP32 squared distance of the definition (pair_r2), computed the
// same way on both sides, so every pair is counted exactly once.
//
// GB300 layout: vertices are Morton-sorted (mesh index above the 30 Morton bits for
// batched meshes), so NEAR_ROWS consecutive sorted vertices form a compact patch
// ("tile") and 16 form a compact "chunk".  One block per tile (NEAR_ROWS output rows x
// the basis pairs) scans the chunk boxes of its mesh range, keeps the chunks whose box
// is within r_e of the tile box, stages their positions and T' in shared memory
// and accumulates two bases x J products per thread; results are added to M at the
// rows' original indices.  Everything is deterministic (fixed orders, no atomics).
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "handles.cuh"

namespace tsr {

__device__ __forceinline__ float near_pair_r2(float xo, float yo, float zo, float xi, float yi, float zi) {
  const float dx = __fsub_rn(xo, xi), dy = __fsub_rn(yo, yi), dz = __fsub_rn(zo, zi);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ int mesh_of_vertex(long long v, int n_mesh, const long long *__restrict__ voff) {
  if (n_mesh <= 1) return 0;
  int lo = 0, hi = n_mesh;   // voff[lo] <= v < voff[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (voff[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// One block per mesh: r_e^2 = max(r_floor^2, 4 sum(A) / N) and the mesh's bounding box.
__global__ void __launch_bounds__(1024) near_mesh_stats_kernel(int n_mesh, const long long *__restrict__ voff,
                                                               long long total, const float *__restrict__ pos,
                                                               long long stride, const float *__restrict__ area,
                                                               float r_floor2, float *__restrict__ rn2,
                                                               float *__restrict__ mbox) {
  __shared__ double s_sum[32];
  __shared__ float s_box[32][6];
  const int m = blockIdx.x;
  const long long v0 = n_mesh > 1 ? voff[m] : 0, v1 = n_mesh > 1 ? voff[m + 1] : total;
  double a = 0.0;
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  // four vertices per thread and pass, so that several loads are in flight
  for (long long vb = v0 + threadIdx.x; vb < v1; vb += 4 * (long long)blockDim.x) {
    float av[4], xv[3][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long v = vb + (long long)e * blockDim.x;
      const bool ok = v < v1;
      av[e] = ok ? area[v] : 0.f;
#pragma unroll
      for (int q = 0; q < 3; ++q) xv[q][e] = ok ? pos[(size_t)q * stride + v] : NAN;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      a += (double)av[e];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        lo[q] = fminf(lo[q], xv[q][e]);   // fminf / fmaxf ignore the NaN of a missing vertex
        hi[q] = fmaxf(hi[q], xv[q][e]);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      lo[q] = fminf(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
      hi[q] = fmaxf(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
    }
  }
  if (lane == 0) {
    s_sum[warp] = a;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      s_box[warp][q] = lo[q];
      s_box[warp][3 + q] = hi[q];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    float b[6] = {3e38f, 3e38f, 3e38f, -3e38f, -3e38f, -3e38f};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += s_sum[w];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        b[q] = fminf(b[q], s_box[w][q]);
        b[3 + q] = fmaxf(b[3 + q], s_box[w][3 + q]);
      }
    }
    const long long n = v1 - v0;
    const double h2x4 = n > 0 ? 4.0 * t / (double)n : 0.0;
    rn2[m] = (float)fmax((double)r_floor2, h2x4);
#pragma unroll
    for (int q = 0; q < 6; ++q) mbox[m * 6 + q] = n > 0 ? b[q] : 0.f;
  }
}

// Morton quantisation of the union of the mesh boxes: gq = {lo x, lo y, lo z, 1023 / extent}.
__global__ void near_global_box_kernel(int n_mesh, const float *__restrict__ mbox, float *__restrict__ gq) {
  if (threadIdx.x != 0) return;
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  for (int m = 0; m < n_mesh; ++m)
    for (int q = 0; q < 3; ++q) {
      lo[q] = fminf(lo[q], mbox[m * 6 + q]);
      hi[q] = fmaxf(hi[q], mbox[m * 6 + 3 + q]);
    }
  const float ext = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), fmaxf(hi[2] - lo[2], 1e-20f));
  gq[0] = lo[0];
  gq[1] = lo[1];
  gq[2] = lo[2];
  gq[3] = 1023.0f / ext;
}

__device__ __forceinline__ unsigned spread_bits10(unsigned x) {   // 10 bits -> every third bit
  x &= 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__global__ void near_keys_kernel(long long total, const float *__restrict__ pos, long long stride, int n_mesh,
                                 const long long *__restrict__ voff, const float *__restrict__ gq,
                                 unsigned long long *__restrict__ keys, int *__restrict__ vals) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v >= total) return;
  unsigned q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float t = (pos[(size_t)a * stride + v] - gq[a]) * gq[3];
    q[a] = (unsigned)fminf(fmaxf(t, 0.f), 1023.f);
  }
  const unsigned code = (spread_bits10(q[0]) << 2) | (spread_bits10(q[1]) << 1) | spread_bits10(q[2]);
  keys[v] = ((unsigned long long)mesh_of_vertex(v, n_mesh, voff) << 30) | code;
  vals[v] = (int)v;
}

// Sorted copies: positions [3][np], T' = A T in FP32 as rows [np][JP], the mesh of each
// sorted vertex ([np], -1 for padding) and its original index.
__global__ void near_gather_kernel(long long total, long long np, const int *__restrict__ perm,
                                   const float *__restrict__ pos, long long stride, const float *__restrict__ area,
                                   const float *__restrict__ T, int J, int JP, int n_mesh,
                                   const long long *__restrict__ voff, float *__restrict__ pos_s,
                                   float *__restrict__ tq, int *__restrict__ mesh_s) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= np) return;
  if (s < total) {
    const int v = perm[s];
#pragma unroll
    for (int a = 0; a < 3; ++a) pos_s[(size_t)a * np + s] = pos[(size_t)a * stride + v];
    const float av = area[v];
    for (int j = 0; j < JP; ++j) tq[(size_t)s * JP + j] = j < J ? av * T[(size_t)j * stride + v] : 0.f;
    mesh_s[s] = mesh_of_vertex(v, n_mesh, voff);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) pos_s[(size_t)a * np + s] = 1e30f;
    for (int j = 0; j < JP; ++j) tq[(size_t)s * JP + j] = 0.f;
    mesh_s[s] = -1;
  }
}

// Boxes of consecutive runs of `run` sorted vertices (the first `total` are real).
__global__ void near_box_kernel(const float *__restrict__ pos_s, long long np, long long total, int run, int n_box,
                                float *__restrict__ box) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_box) return;
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  const long long v0 = (long long)b * run, v1 = min(total, v0 + run);
  for (long long v = v0; v < v1; ++v) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float x = pos_s[(size_t)a * np + v];
      lo[a] = fminf(lo[a], x);
      hi[a] = fmaxf(hi[a], x);
    }
  }
  if (v1 <= v0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = 1e30f;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    box[b * 6 + a] = lo[a];
    box[b * 6 + 3 + a] = hi[a];
  }
}

#ifndef TSR_NEAR_ROWS
#define TSR_NEAR_ROWS 32
#endif
constexpr int NEAR_ROWS = TSR_NEAR_ROWS;   // output rows per block (a divisor of 128)
constexpr int NEAR_SCAN = 256;    // chunk boxes tested per pass
#ifndef TSR_NEAR_BATCH
#define TSR_NEAR_BATCH 4
#endif
constexpr int NEAR_BATCH = TSR_NEAR_BATCH;   // listed chunks staged per barrier (16 candidates each)

// Asynchronous global -> shared copies (cp.async): the next candidate batch lands while the
// current one is tested and summed, without holding registers.
__device__ __forceinline__ void near_cp16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void near_cp4(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
// Two FP32 lanes per instruction (fma.rn.f32x2): each lane rounds exactly as fmaf, so the
// sums are bit-identical to the scalar form.
__device__ __forceinline__ uint64_t near_f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void near_f2_unpack(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t near_f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ void near_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void near_cp_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One block per NEAR_ROWS sorted output rows (two or more blocks per SM interleave their
// phases).  Per batch of up to 16 NEAR_BATCH staged candidates i:
//  phase A: the block tests every (row, i) pair once (a warp covers 32 consecutive i of
//           one row) and records the near pairs as bit masks plus x = r / dr;
//  phase B: thread (row, kg) owns bases 2 kg, 2 kg + 1 and walks its row's set bits in
//           increasing i, adding A_i f_k(r) T[j][i] for every j (deterministic order).
template <int JP>
__global__ void __launch_bounds__(512) near_field_kernel(
    const float *__restrict__ pos_s, const float *__restrict__ tq, const int *__restrict__ mesh_s,
    const int *__restrict__ perm, long long np, long long total, const float *__restrict__ tile_box,
    const float *__restrict__ chunk_box, int n_mesh, const long long *__restrict__ voff,
    const float *__restrict__ rn2, const float4 *__restrict__ tab, int KG, int n_r, float inv_dr, float r2max,
    int K, int J, float *__restrict__ M, long long stride) {
  constexpr int NC = NEAR_BATCH * 16;   // candidates per batch
  __shared__ __align__(16) float sTb[2][NC * JP];   // two batches: one staged while the other is summed
  __shared__ float sxb[2][NC], syb[2][NC], szb[2][NC];
  __shared__ int smb[2][NC];
  __shared__ float s_xv[NEAR_ROWS][NC + 1];       // r / dr of the near pairs (+1: no bank conflicts)
  __shared__ unsigned s_mask[NEAR_ROWS][NC / 32];
  __shared__ float s_row[NEAR_ROWS][4];           // x, y, z, r_e^2 of the block's rows
  __shared__ int s_rmesh[NEAR_ROWS];
  __shared__ int s_list[NEAR_SCAN];
  __shared__ int s_warp[NEAR_SCAN / 32];
  __shared__ float s_tb[6];
  __shared__ int s_range[2];
  __shared__ float s_rn2m;
  const int tile = blockIdx.x;   // the block's rows of the sorted order, with their box
  const int kg = threadIdx.x % KG;
  const int ol = threadIdx.x / KG;
  const long long os = (long long)blockIdx.x * NEAR_ROWS + ol;
  const bool o_ok = ol < NEAR_ROWS && os < total;
  for (int r = threadIdx.x; r < NEAR_ROWS; r += blockDim.x) {
    const long long q = (long long)blockIdx.x * NEAR_ROWS + r;
    const bool ok = q < total;
    const int m = ok ? mesh_s[q] : -2;
    s_row[r][0] = ok ? pos_s[q] : 0.f;
    s_row[r][1] = ok ? pos_s[np + q] : 0.f;
    s_row[r][2] = ok ? pos_s[2 * np + q] : 0.f;
    s_row[r][3] = ok ? rn2[m] : 0.f;
    s_rmesh[r] = m;
  }
  if (threadIdx.x == 0) {
    // meshes of the tile's first and last rows; the chunks of those meshes (sorted blocks)
    const long long t0 = (long long)tile * NEAR_ROWS, t1 = min(total, t0 + NEAR_ROWS) - 1;
    const int m0 = mesh_s[t0], m1 = mesh_s[t1];
    const long long c0 = (n_mesh > 1 ? voff[m0] : 0) / 16;
    const long long c1 = ((n_mesh > 1 ? voff[m1 + 1] : total) + 15) / 16;
    s_range[0] = (int)c0;
    s_range[1] = (int)c1;
    float r = 0.f;
    for (int m = m0; m <= m1; ++m) r = fmaxf(r, rn2[m]);
    s_rn2m = r * 1.001f + 1e-6f;
#pragma unroll
    for (int q = 0; q < 6; ++q) s_tb[q] = tile_box[tile * 6 + q];
  }
  __syncthreads();
  uint64_t acc0[JP / 2], acc1[JP / 2];   // sums for (j, j + 1), two lanes per fma.rn.f32x2
#pragma unroll
  for (int j2 = 0; j2 < JP / 2; ++j2) acc0[j2] = acc1[j2] = 0ull;   // +0.0f in both lanes
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = (int)(blockDim.x >> 5);
  const int scan = min(NEAR_SCAN, (int)blockDim.x);   // chunk boxes tested per pass (a multiple of 32)
  for (int base = s_range[0]; base < s_range[1]; base += scan) {
    // compact the chunks of this pass whose box is within r_e of the tile box
    bool keep = false;
    const int c = base + (int)threadIdx.x;
    if ((int)threadIdx.x < scan && c < s_range[1]) {
      float d2 = 0.f;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float gap = fmaxf(0.f, fmaxf(s_tb[q] - chunk_box[(size_t)c * 6 + 3 + q], chunk_box[(size_t)c * 6 + q] - s_tb[3 + q]));
        d2 = fmaf(gap, gap, d2);
      }
      keep = d2 < s_rn2m;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if ((int)threadIdx.x < scan && lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, n_list = 0;
    for (int w = 0; w < scan / 32; ++w) {
      before += w < warp ? s_warp[w] : 0;
      n_list += s_warp[w];
    }
    if (keep) s_list[before + __popc(bal & ((1u << lane) - 1u))] = c;
    __syncthreads();
    // stage up to NEAR_BATCH listed chunks (16 i each) into buffer bs; the rest of the batch is empty
    auto stage = [&](int lb, int bs) {
      const int nb = min(NEAR_BATCH, n_list - lb);
      for (int q = threadIdx.x; q < nb * 16 * JP / 4; q += blockDim.x) {
        const int cc = q / (16 * JP / 4), w = q % (16 * JP / 4);
        near_cp16(reinterpret_cast<float4 *>(sTb[bs]) + q,
                  reinterpret_cast<const float4 *>(tq + (size_t)s_list[lb + cc] * 16 * JP) + w);
      }
      for (int q = threadIdx.x; q < NC; q += blockDim.x) {
        if (q < nb * 16) {
          const long long i = (long long)s_list[lb + q / 16] * 16 + (q % 16);
          near_cp4(&sxb[bs][q], pos_s + i);
          near_cp4(&syb[bs][q], pos_s + np + i);
          near_cp4(&szb[bs][q], pos_s + 2 * np + i);
          near_cp4(&smb[bs][q], mesh_s + i);
        } else {
          smb[bs][q] = -1;   // no candidate
        }
      }
      near_cp_commit();
    };
    if (n_list > 0) stage(0, 0);
    for (int lb = 0, bs = 0; lb < n_list; lb += NEAR_BATCH, bs ^= 1) {
      near_cp_wait();
      __syncthreads();   // batch lb is in buffer bs; the other buffer's last batch has been summed
      if (lb + NEAR_BATCH < n_list) stage(lb + NEAR_BATCH, bs ^ 1);
      const float *sT = sTb[bs], *sx = sxb[bs], *sy = syb[bs], *sz = szb[bs];
      const int *sm = smb[bs];
      // phase A: warp w takes 32 consecutive candidates of one row per turn
      for (int item = warp; item < NEAR_ROWS * (NC / 32); item += n_warps) {
        const int r = item / (NC / 32), wd = item % (NC / 32), ii = wd * 32 + lane;
        const float r2 = near_pair_r2(s_row[r][0], s_row[r][1], s_row[r][2], sx[ii], sy[ii], sz[ii]);
        const bool nr = sm[ii] == s_rmesh[r] && r2 < s_row[r][3] && r2 <= r2max;
        if (nr) s_xv[r][ii] = __fsqrt_rn(r2) * inv_dr;
        const unsigned bits = __ballot_sync(0xffffffffu, nr);
        if (lane == 0) s_mask[r][wd] = bits;
      }
      __syncthreads();
      // phase B
      if (o_ok) {
#pragma unroll
        for (int wd = 0; wd < NC / 32; ++wd) {
          unsigned bits = s_mask[ol][wd];
          while (bits) {
            const int ii = wd * 32 + __ffs(bits) - 1;
            bits &= bits - 1u;
            const float x = s_xv[ol][ii];
            const int m = min(static_cast<int>(x), n_r - 2);
            const float t = x - static_cast<float>(m);
            const float4 tb = __ldg(tab + (size_t)m * KG + kg);
            const float F0 = fmaf(t, tb.y, tb.x), F1 = fmaf(t, tb.w, tb.z);
            const uint64_t F0p = near_f2_pack(F0, F0), F1p = near_f2_pack(F1, F1);
            const float4 *tv = reinterpret_cast<const float4 *>(sT + ii * JP);
#pragma unroll
            for (int j4 = 0; j4 < JP / 4; ++j4) {
              const float4 v = tv[j4];
              const uint64_t va = near_f2_pack(v.x, v.y), vb = near_f2_pack(v.z, v.w);
              acc0[2 * j4] = near_f2_fma(F0p, va, acc0[2 * j4]);
              acc0[2 * j4 + 1] = near_f2_fma(F0p, vb, acc0[2 * j4 + 1]);
              acc1[2 * j4] = near_f2_fma(F1p, va, acc1[2 * j4]);
              acc1[2 * j4 + 1] = near_f2_fma(F1p, vb, acc1[2 * j4 + 1]);
            }
          }
        }
      }
      // (the next batch's barrier, after its copies landed, orders this phase B before its phase A)
    }
    __syncthreads();   // s_warp and s_list are rewritten by the next pass
  }
  if (o_ok) {
    const long long o = perm[os];
    const int k0 = 2 * kg, k1 = 2 * kg + 1;
#pragma unroll
    for (int j2 = 0; j2 < JP / 2; ++j2) {
      float a0[2], a1[2];
      near_f2_unpack(acc0[j2], a0[0], a0[1]);
      near_f2_unpack(acc1[j2], a1[0], a1[1]);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int j = 2 * j2 + e;
        if (j < J) {
          if (k0 < K) M[((size_t)k0 * J + j) * stride + o] += a0[e];
          if (k1 < K) M[((size_t)k1 * J + j) * stride + o] += a1[e];
        }
      }
    }
  }
}

tsr_status near_setup(NearField &nf, const tsr_basis *b, int n_mesh, const long long *d_voff, long long total,
                      const float *pos, long long stride, const float *area, const float *T, int J, cudaStream_t s) {
  nf.n_mesh = n_mesh;
  nf.total = total;
  nf.voff = d_voff;
  nf.J = J;
  nf.JP = (J + 3) & ~3;
  nf.np = (total + 127) / 128 * 128;
  nf.n_tiles = (int)(nf.np / NEAR_ROWS);   // row blocks of the near-field kernel
  nf.n_chunks = (int)(nf.np / 16);
  size_t sort_bytes = 0;
  TSR_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (unsigned long long *)nullptr,
                                           (unsigned long long *)nullptr, (int *)nullptr, (int *)nullptr,
                                           (int)total, 0, 64, s));
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t b_rn2 = al(sizeof(float) * n_mesh), b_mbox = al(sizeof(float) * 6 * n_mesh), b_gq = al(16),
               b_keys = al(sizeof(unsigned long long) * total), b_vals = al(sizeof(int) * total),
               b_pos = al(sizeof(float) * 3 * nf.np), b_tq = al(sizeof(float) * nf.np * nf.JP),
               b_mesh = al(sizeof(int) * nf.np), b_tbox = al(sizeof(float) * 6 * nf.n_tiles),
               b_cbox = al(sizeof(float) * 6 * nf.n_chunks), b_sort = al(sort_bytes);
  tsr_status st = nf.buf.alloc(b_rn2 + b_mbox + b_gq + 2 * b_keys + 2 * b_vals + b_pos + b_tq + b_mesh + b_tbox +
                                   b_cbox + b_sort, s);
  if (st != TSR_OK) return st;
  uint8_t *p = static_cast<uint8_t *>(nf.buf.p);
  auto take = [&](size_t bytes) {
    uint8_t *q = p;
    p += bytes;
    return q;
  };
  nf.rn2 = reinterpret_cast<float *>(take(b_rn2));
  float *mbox = reinterpret_cast<float *>(take(b_mbox));
  float *gq = reinterpret_cast<float *>(take(b_gq));
  auto *keys_in = reinterpret_cast<unsigned long long *>(take(b_keys));
  auto *keys = reinterpret_cast<unsigned long long *>(take(b_keys));
  int *vals_in = reinterpret_cast<int *>(take(b_vals));
  nf.perm = reinterpret_cast<int *>(take(b_vals));
  nf.pos_s = reinterpret_cast<float *>(take(b_pos));
  nf.tq = reinterpret_cast<float *>(take(b_tq));
  nf.mesh_s = reinterpret_cast<int *>(take(b_mesh));
  nf.tile_box = reinterpret_cast<float *>(take(b_tbox));
  nf.chunk_box = reinterpret_cast<float *>(take(b_cbox));
  void *sort_tmp = take(b_sort);
  const float r_floor = (float)b->r_near;
  near_mesh_stats_kernel<<<n_mesh, 1024, 0, s>>>(n_mesh, d_voff, total, pos, stride, area, r_floor * r_floor,
                                               nf.rn2, mbox);
  ::tsr::count_launch();
  near_global_box_kernel<<<1, 32, 0, s>>>(n_mesh, mbox, gq); ::tsr::count_launch();
  near_keys_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, pos, stride, n_mesh, d_voff, gq, keys_in,
                                                                    vals_in);
  ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  int end_bit = 30;
  while ((1ll << (end_bit - 30)) < n_mesh) ++end_bit;
  TSR_CUDA(cub::DeviceRadixSort::SortPairs(sort_tmp, sort_bytes, keys_in, keys, vals_in, nf.perm, (int)total, 0,
                                           end_bit, s));
  ::tsr::count_launch();
  near_gather_kernel<<<(unsigned)((nf.np + 255) / 256), 256, 0, s>>>(total, nf.np, nf.perm, pos, stride, area, T, J,
                                                                      nf.JP, n_mesh, d_voff, nf.pos_s, nf.tq,
                                                                      nf.mesh_s);
  ::tsr::count_launch();
  near_box_kernel<<<(nf.n_tiles + 127) / 128, 128, 0, s>>>(nf.pos_s, nf.np, total, NEAR_ROWS, nf.n_tiles,
                                                          nf.tile_box);
  ::tsr::count_launch();
  near_box_kernel<<<(nf.n_chunks + 127) / 128, 128, 0, s>>>(nf.pos_s, nf.np, total, 16, nf.n_chunks, nf.chunk_box);
  ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

template <int JP>
static void launch_near(const NearField &nf, const tsr_basis *b, float *M, long long stride, cudaStream_t s) {
  const int KG = b->KP / 2;
  const int threads = NEAR_ROWS * KG;
  const float inv_dr = static_cast<float>((b->n_r - 1) / b->r_max);
  const float r2max = static_cast<float>(b->r_max * b->r_max);
  near_field_kernel<JP><<<nf.n_tiles, threads, 0, s>>>(
      nf.pos_s, nf.tq, nf.mesh_s, nf.perm, nf.np, nf.total, nf.tile_box, nf.chunk_box, nf.n_mesh, nf.voff, nf.rn2,
      reinterpret_cast<const float4 *>(b->tab32), KG, b->n_r, inv_dr, r2max, b->K, nf.J, M, stride);
  ::tsr::count_launch();
}

tsr_status near_apply(const NearField &nf, const tsr_basis *b, float *M, long long stride, cudaStream_t s) {
  switch (nf.JP) {
#define NEAR_CASE(JPV) \
  case JPV: launch_near<JPV>(nf, b, M, stride, s); break;
    NEAR_CASE(4) NEAR_CASE(8) NEAR_CASE(12) NEAR_CASE(16) NEAR_CASE(20) NEAR_CASE(24) NEAR_CASE(28) NEAR_CASE(32)
#undef NEAR_CASE
    default:
      set_error("near field: J=%d unsupported", nf.J);
      return TSR_ERR_UNSUPPORTED;
  }
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

}  // namespace tsr
