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
// The rows of a run lie in a few contiguous spans of the CSR arrays (one per level
// of the run, one per path row, the poles), so the block reads its entries as one
// flat, coalesced stream whatever the row lengths, and cuts it into rows with a
// bitmap of row starts.
//
// Fixed-order arithmetic (results do not depend on scheduling): a row's sum is
// formed by lanes adding their consecutive entries in order, a segmented scan over
// the warp, the warp's steps in order and its ranges chained in order; each
// synthesis step is (a + d) / sqrt2 or (a - d) / sqrt2, as in the level-by-level
// inverse.
//
// With g = identity the same kernel yields the light-contracted basis images
// Z[k] = w_1^{-1} (S (e_k x l)) (K "vectors"); the relight of many edits on many
// copies is then those images plus relight_combine_many_kernel, B = sum_k g_k Z[k].
#include <algorithm>
#include <atomic>

#include "handles.cuh"

namespace tsr {

constexpr int RF_THREADS = 256;
constexpr int RF_LGSEG = 10;
constexpr int RF_SEG = 1 << RF_LGSEG;                      // Morton positions per run
constexpr int RF_MAX_LGN = 14 - RF_LGSEG;                  // log2 of the runs of a 128^2 chart (the library's nu <= 128)
constexpr int RF_MAX_TOP = 1 + RF_MAX_LGN;                 // path rows
constexpr int RF_MAX_ROWS = RF_MAX_TOP + RF_SEG - 1 + 2;   // + run details + the two poles
constexpr int RF_BW = (RF_MAX_ROWS + 3) & ~3;              // b^w row stride in shared memory
constexpr int RF_MAXC = 32;                                // copies per launch (kernel parameter space)
constexpr int RF_WARPS = RF_THREADS / 32;
__host__ __device__ constexpr int rf_units(int) { return 8; }   // groups of 4 entries per lane unit

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

// The lanes of one warp step: 32 consecutive lane units from unit u0 (below ur1) over
// the non-empty rows from rank rb on.  rows[r] = {first entry, entries, first unit, q}.
struct RfStep {
  unsigned H;     // lanes where a row starts
  int rel;        // the lane's row, from rb
  int lh;         // the lane where the lane's row starts in the step (-1: before it)
  int pa, n;      // the lane's row: first entry and entries
  int k;          // the lane's unit within its row
  int g0, ng, Lr; // the row's first aligned group, groups and units
  int rel31;      // lane 31's row, from rb
  int uend;       // end of the step's units
  bool act;       // the lane holds a unit
  bool ends;      // lane 31's row ends with the step
};

template <int U>
__device__ __forceinline__ RfStep rf_assign(const int4 *rows, int n_ne, int u0, int ur1, int rb, int lane) {
  RfStep a;
  a.uend = min(u0 + 32, ur1);
  const int4 ri = rb + lane <= n_ne ? rows[rb + lane] : make_int4(0, 0, 0x7fffffff, 0);
  const bool hd = rb + lane < n_ne && ri.z >= u0 && ri.z < a.uend;
  a.H = __reduce_or_sync(0xffffffffu, hd ? 1u << (ri.z - u0) : 0u);
  const unsigned Hl = a.H & ((2u << lane) - 1u);
  a.rel = __popc(Hl & ~1u);
  a.lh = Hl ? 31 - __clz(Hl) : -1;
  a.pa = __shfl_sync(0xffffffffu, ri.x, a.rel);
  a.n = __shfl_sync(0xffffffffu, ri.y, a.rel);
  const int cs = __shfl_sync(0xffffffffu, ri.z, a.rel);
  a.act = u0 + lane < a.uend;
  a.g0 = a.pa >> 2;
  a.ng = ((a.pa + a.n + 3) >> 2) - a.g0;
  a.Lr = (a.ng + U - 1) / U;
  a.k = u0 + lane - cs;
  a.rel31 = __shfl_sync(0xffffffffu, a.rel, 31);
  a.ends = rows[min(rb + a.rel31 + 1, n_ne)].z == a.uend;
  return a;
}

// The lane's groups k, k + Lr, ..., k + (U - 1) Lr of its row (zeros beyond the row).
template <int U>
__device__ __forceinline__ void rf_load(const float4 *__restrict__ val4, const uint2 *__restrict__ col4, const RfStep &a,
                                        float4 (&av)[U], uint2 (&kv)[U]) {
#pragma unroll
  for (int m = 0; m < U; ++m) {
    const int gi = a.k + m * a.Lr;
    av[m] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    kv[m] = make_uint2(0u, 0u);
    if (a.act && gi < a.ng) {
      av[m] = __ldg(val4 + a.g0 + gi);
      kv[m] = __ldg(col4 + a.g0 + gi);
    }
  }
}

// val * c_v[kj] added to the VV sums, with c_v[kj] = g_v[k] l[j] (k = kj / J, j = kj - k J)
// read as two small tables: l[j] (J <= 32 floats, one bank each, so the lanes never
// conflict) and g_v[k] (K <= 16 rows of VQ float4; the lanes of a row ask for one or two
// neighbouring k at a time).  k = floor((2 kj + 1) / 2J), the multiply-high of 2 kj + 1 by
// m2J = ceil(2^32 / 2J): exact for kj < 2^16 and 1 <= J <= 32 (the product's excess stays
// below 2^-15, under the margin 1 / 2J that the odd numerator leaves).
template <int VV>
__device__ __forceinline__ void rf_fma(const float *lt, const float4 *gs4, unsigned m2J, int J, int kj, float a,
                                       float (&acc)[VV]) {
  constexpr int VQ = (VV + 3) / 4;
  const int k = (int)__umulhi(2u * (unsigned)kj + 1u, m2J);
  const float t = a * lt[kj - k * J];
#pragma unroll
  for (int h = 0; h < VQ; ++h) {
    const float4 c = gs4[k * VQ + h];
    const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (4 * h + e < VV) acc[4 * h + e] = fmaf(t, cv[e], acc[4 * h + e]);
  }
}

template <int VV>
__global__ void __launch_bounds__(RF_THREADS, VV <= 6 ? 3 : 2) relight_fused_kernel(const __grid_constant__ RelightBatch bt, int K,
                                                                  int J, unsigned m2J, const float *__restrict__ l) {
  constexpr int VQ = (VV + 3) / 4;   // float4s per c row
  constexpr bool XDYN = VV > 6;      // b^w in dynamic shared memory (above 24 KB)
  constexpr int SQ = (RF_MAX_ROWS + RF_THREADS - 1) / RF_THREADS;   // local rows per thread
  constexpr int NB = SQ * RF_WARPS;  // (pass, warp) pairs of the row pass, <= 64
  constexpr int RF_U = rf_units(VV); // groups of 4 entries per lane unit
  // b^w of the block's rows by local row q: 0 the chart's scaling coefficient, 1 .. T - 1
  // the path rows, T - 1 + n the run's detail at local position n (1 <= n < L), R and
  // R + 1 the poles.
  __shared__ __align__(16) float bws[XDYN ? 1 : VV][RF_BW];
  // The non-empty rows in local-row order (rank): {first entry, entries, first lane
  // unit, q}; entry n_ne is a sentinel holding the total units.
  __shared__ int4 rows[RF_MAX_ROWS + 1];
  __shared__ int cnt[NB];            // packed (non-empty rows << 20 | units) per (pass, warp)
  __shared__ int lrank[RF_WARPS];
  __shared__ float fpart[RF_WARPS][VV], lpart[RF_WARPS][VV];
  __shared__ float lt[32];                 // l[j]
  __shared__ float4 gs4[16 * VQ];          // g_v[k] at [k][v / 4] (identity in basis-image mode)
  extern __shared__ float4 dyn4[];         // b^w when XDYN
  float (*bw)[RF_BW] = XDYN ? reinterpret_cast<float (*)[RF_BW]>(dyn4) : bws;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int ci = 0;   // the block's copy: the last with item0 <= blockIdx.x
  for (int hi = bt.n - 1; ci < hi;) {
    const int mid = (ci + hi + 1) >> 1;
    if (bt.c[mid].item0 <= (int)blockIdx.x) ci = mid; else hi = mid - 1;
  }
  const RelightCopy &cp = bt.c[ci];
  const int nu = cp.nu, lgP = cp.lgP;
  const int lgP2 = 2 * lgP, P2 = 1 << lgP2;
  const int lgL = min(lgP2, RF_LGSEG), L = 1 << lgL;
  const int lgn = lgP2 - lgL;   // log2(runs per chart)
  const int local = (int)blockIdx.x - cp.item0;
  const int d = local >> lgn, s = local & ((1 << lgn) - 1);
  const int T = 1 + lgn;        // path rows
  const int R = T + L - 1;
  const bool poles = (d == 0 && s == 0);
  const int R_tot = R + (poles ? 2 : 0);
  const int64_t wbase = (int64_t)d * P2;
  const int64_t *__restrict__ row_ptr = cp.row_ptr;
  const float4 *__restrict__ val4 = reinterpret_cast<const float4 *>(cp.val);
  const uint2 *__restrict__ col4 = reinterpret_cast<const uint2 *>(cp.col);

  // Row pointers of the block's rows, all in flight while the tables are set up (their
  // low words: entries lie below 2^31, relight_fusable).
  const int *__restrict__ rp32 = reinterpret_cast<const int *>(row_ptr);
  int p0[SQ], p1[SQ];
#pragma unroll
  for (int i = 0; i < SQ; ++i) {
    const int q = RF_THREADS * i + tid;
    p0[i] = p1[i] = 0;
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
      p0[i] = __ldg(rp32 + 2 * w);
      p1[i] = __ldg(rp32 + 2 * w + 2);
    }
  }

  // Empty rows contribute zeros.
  for (int q = tid; q < VV * RF_BW / 4; q += RF_THREADS)
    reinterpret_cast<float4 *>(&bw[0][0])[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (tid < J) lt[tid] = l[tid];
  if (tid < K * VQ) {   // basis-image mode (no g): g_v[k] = 1 for v = k, else 0
    const int k = tid / VQ, h = tid - k * VQ;
    float gk[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int v = 4 * h + e;
      gk[e] = v < VV ? (cp.g ? cp.g[v * K + k] : (v == k ? 1.0f : 0.0f)) : 0.0f;
    }
    gs4[tid] = make_float4(gk[0], gk[1], gk[2], gk[3]);
  }

  // A non-empty row of ng aligned groups of 4 entries (the first and last possibly
  // shared with its neighbours) takes ceil(ng / RF_U) lane units.  Rank and first unit
  // of each row: a packed prefix count over the rows in local-row order.
  int incv[SQ], ownv[SQ];
#pragma unroll
  for (int i = 0; i < SQ; ++i) {
    const int pa = p0[i], n = p1[i] - p0[i];
    const int ng = n > 0 ? ((pa + n + 3) >> 2) - (pa >> 2) : 0;
    ownv[i] = n > 0 ? (1 << 20) | ((ng + RF_U - 1) / RF_U) : 0;
    int inc = ownv[i];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    incv[i] = inc;
    if (lane == 31) cnt[i * RF_WARPS + warp] = inc;
  }
  __syncthreads();
  int tot, base_lo, base_hi;   // every warp scans the NB counts (two per lane)
  {
    const int c0 = 2 * lane < NB ? cnt[2 * lane] : 0, c1 = 2 * lane + 1 < NB ? cnt[2 * lane + 1] : 0;
    int inc = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    base_lo = inc - c0 - c1;
    base_hi = inc - c1;
    tot = __shfl_sync(0xffffffffu, inc, 31);
  }
  const int n_ne = tot >> 20, U_tot = tot & 0xFFFFF;
#pragma unroll
  for (int i = 0; i < SQ; ++i) {
    const int idx = i * RF_WARPS + warp;
    const int lo = __shfl_sync(0xffffffffu, base_lo, idx >> 1), hi = __shfl_sync(0xffffffffu, base_hi, idx >> 1);
    const int before = ((idx & 1) ? hi : lo) + incv[i] - ownv[i];
    if (ownv[i]) rows[before >> 20] = make_int4(p0[i], p1[i] - p0[i], before & 0xFFFFF, RF_THREADS * i + tid);
  }
  if (tid == 0) rows[n_ne] = make_int4(0, 0, U_tot, 0);
  __syncthreads();

  // b^w of the non-empty rows.  The rows' lane units are cut into eight contiguous
  // ranges, one per warp; a warp step gives its 32 lanes 32 consecutive units.  The
  // unit k of a row with L units takes the row's groups k, k + L, ..., k + (RF_U - 1) L
  // (those below ng), so the lanes of a row read consecutive groups at each load and
  // neighbouring lanes read nearby columns of the c table.  A lane adds val * c[col] of
  // its entries in order; the lanes of a row meet in a segmented scan over the warp
  // (rows start at lane boundaries); a row crossing steps continues in a carry; and
  // the eight ranges are chained in order by one thread.  Every sum is formed in the
  // same order whatever the scheduling.
  auto emit = [&](int rank, const float (&val)[VV]) {
    if (rank < 0 || rank >= n_ne) return;   // unreachable: ranks of non-empty rows only
    const int q = rows[rank].w;
#pragma unroll
    for (int v = 0; v < VV; ++v) bw[v][q] = val[v];
  };
  {
    const int per = 32 * (((U_tot + 31) / 32 + RF_WARPS - 1) / RF_WARPS);   // whole steps per warp
    const int ur0 = warp * per, ur1 = min(ur0 + per, U_tot);
    float C[VV];   // the row open at the end of the previous step
#pragma unroll
    for (int v = 0; v < VV; ++v) C[v] = 0.0f;
    int lr = -2;   // the range's open row at its end (-2: the row open at its start)
    if (ur0 < ur1) {
      int rb = 0;   // the row holding unit ur0: the last rank with first unit <= ur0
      {
        int hi = n_ne - 1;
        while (rb < hi) {
          const int mid = (rb + hi + 1) >> 1;
          if (rows[mid].z <= ur0) rb = mid; else hi = mid - 1;
        }
      }
      const int r0 = rb;
      const bool open_before = rows[r0].z < ur0;
      if (lane == 0) {
#pragma unroll
        for (int v = 0; v < VV; ++v) fpart[warp][v] = 0.0f;
      }
      __syncwarp();
      bool ends = false;
      for (int u0 = ur0; u0 < ur1; u0 += 32) {
        const RfStep A = rf_assign<RF_U>(rows, n_ne, u0, ur1, rb, lane);
        float4 av[RF_U];
        uint2 kv[RF_U];
        rf_load<RF_U>(val4, col4, A, av, kv);
        {   // entries of the row only: its first group (unit 0) and its last group may
            // hold entries of the neighbouring rows, whose values are set to zero (the
            // columns of every entry, the padding's included, index the c table)
          const int lo = A.pa & 3, hi = ((A.pa + A.n - 1) & 3) + 1;
#pragma unroll
          for (int m = 0; m < RF_U; ++m) {
            unsigned keep = A.k + m * A.Lr == A.ng - 1 ? (1u << hi) - 1u : 0xFu;
            if (m == 0 && A.k == 0) keep &= 0xFu << lo;
            av[m].x = (keep & 1u) ? av[m].x : 0.0f;
            av[m].y = (keep & 2u) ? av[m].y : 0.0f;
            av[m].z = (keep & 4u) ? av[m].z : 0.0f;
            av[m].w = (keep & 8u) ? av[m].w : 0.0f;
          }
        }
        float run[VV];
#pragma unroll
        for (int v = 0; v < VV; ++v) run[v] = 0.0f;
#pragma unroll
        for (int m = 0; m < RF_U; ++m) {
          rf_fma<VV>(lt, gs4, m2J, J, (int)(kv[m].x & 0xFFFFu), av[m].x, run);
          rf_fma<VV>(lt, gs4, m2J, J, (int)(kv[m].x >> 16), av[m].y, run);
          rf_fma<VV>(lt, gs4, m2J, J, (int)(kv[m].y & 0xFFFFu), av[m].z, run);
          rf_fma<VV>(lt, gs4, m2J, J, (int)(kv[m].y >> 16), av[m].w, run);
        }
        // Segmented inclusive scan: at distance o a lane adds the partial sum o lanes
        // back when its row started at or before that lane.
        const int dist = lane - A.lh;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          float t[VV];
#pragma unroll
          for (int v = 0; v < VV; ++v) t[v] = __shfl_up_sync(0xffffffffu, run[v], o);
          if (lane >= o && dist >= o)
#pragma unroll
            for (int v = 0; v < VV; ++v) run[v] = t[v] + run[v];
        }
        if (A.lh < 0)
#pragma unroll
          for (int v = 0; v < VV; ++v) run[v] = C[v] + run[v];
        ends = A.ends;
        const bool last = lane < 31 ? ((A.H >> (lane + 1)) & 1u) != 0 : ends;
        if (last) {
          const int r = rb + A.rel;
          if (r == r0 && open_before) {
#pragma unroll
            for (int v = 0; v < VV; ++v) fpart[warp][v] = run[v];
          } else {
            emit(r, run);
          }
        }
#pragma unroll
        for (int v = 0; v < VV; ++v) C[v] = ends ? 0.0f : __shfl_sync(0xffffffffu, run[v], 31);
        rb += A.rel31 + (ends ? 1 : 0);
      }
      if (ends) {
        lr = -1;   // no row open at the range end
      } else if (rb == r0 && open_before) {
        lr = -2;   // one row across the whole range: its part is the range's first part
        if (lane == 0)
#pragma unroll
          for (int v = 0; v < VV; ++v) fpart[warp][v] = C[v];
      } else {
        lr = rb;
      }
    } else if (lane == 0) {
#pragma unroll
      for (int v = 0; v < VV; ++v) fpart[warp][v] = 0.0f;
    }
    if (lane == 0) {
      lrank[warp] = lr;
#pragma unroll
      for (int v = 0; v < VV; ++v) lpart[warp][v] = C[v];
    }
  }
  __syncthreads();
  if (tid == 0) {   // chain the ranges in order
    float P[VV];
#pragma unroll
    for (int v = 0; v < VV; ++v) P[v] = 0.0f;
    int prank = -1;
    for (int w2 = 0; w2 < RF_WARPS; ++w2) {
#pragma unroll
      for (int v = 0; v < VV; ++v) P[v] += fpart[w2][v];
      if (lrank[w2] != -2) {
        if (prank >= 0) emit(prank, P);
#pragma unroll
        for (int v = 0; v < VV; ++v) P[v] = lpart[w2][v];
        prank = lrank[w2];
      }
    }
    if (prank >= 0) emit(prank, P);
  }
  __syncthreads();

  // Synthesis.  A thread owns a subtree: the 2^D = min(16, L) consecutive Morton
  // positions below one approximation at level 2^ls (ls = log2 L - D) of the run.  It
  // forms that approximation by walking down from the chart's scaling coefficient
  // (the chart's path to the run, then the run's levels), expands the D levels below
  // it in registers, and scatters the 2^D values (a square of vertices) to B.  Each
  // value is formed exactly as in the level-by-level synthesis, (a + d) / sqrt2 or
  // (a - d) / sqrt2 from its parent and the parent's detail; details are only read.
  const float rs2 = 0.70710678118654752440f;
  const int D = min(lgL, 4), ls = lgL - D;
  const unsigned m0 = (unsigned)s << lgL;
  const int r0 = (int)rf_compact(m0 >> 1), c0 = (int)rf_compact(m0);
  const int N = 10 * nu * nu + 2;
  float *__restrict__ B = cp.B;
  const int nv = bt.nv;
  for (int it = tid; it < (nv << ls); it += RF_THREADS) {
    const int v = it >> ls, p = it & ((1 << ls) - 1);
    const float *xv = &bw[v][T - 1];   // the run's details by local position
    // a right child takes a - d: d with its sign bit flipped (a + (-d) is a - d exactly)
    float a = bw[v][0];
    for (int lv = 0; lv < lgn; ++lv) {
      const unsigned flip = (unsigned)((s >> (lgn - 1 - lv)) & 1) << 31;
      a = (a + __uint_as_float(__float_as_uint(bw[v][1 + lv]) ^ flip)) * rs2;
    }
    for (int ln = 0; ln < ls; ++ln) {   // approximation index p >> (ls - ln) at level 2^ln
      const unsigned flip = (unsigned)((p >> (ls - ln - 1)) & 1) << 31;
      a = (a + __uint_as_float(__float_as_uint(xv[(1 << ln) + (p >> (ls - ln))]) ^ flip)) * rs2;
    }
    float o[16];
    o[0] = a;
#pragma unroll
    for (int lv = 0; lv < 4; ++lv) {
      if (lv < D) {
#pragma unroll
        for (int i = (1 << lv) - 1; i >= 0; --i) {   // descending: o[i] is read before o[2i], o[2i + 1] are written
          const float dd = xv[(1 << (ls + lv)) + (p << lv) + i];
          const float x = o[i];
          o[2 * i] = (x + dd) * rs2;
          o[2 * i + 1] = (x - dd) * rs2;
        }
      }
    }
    const unsigned mb = (unsigned)p << D;   // first Morton position of the subtree in the run
    const int rb = r0 + (int)rf_compact(mb >> 1), cb = c0 + (int)rf_compact(mb);
    float *__restrict__ Bv = B + (size_t)v * N + (size_t)d * nu * nu;
    if (D == 4 && rb + 3 < nu && cb + 3 < nu) {   // the whole 4 x 4 square inside the chart
      float *__restrict__ Bs = Bv + rb * nu + cb;
#pragma unroll
      for (int i = 0; i < 16; ++i) Bs[(((i >> 1) & 1) | ((i >> 2) & 2)) * nu + ((i & 1) | ((i >> 1) & 2))] = o[i];
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (i < (1 << D)) {
          const int r = rb + (((i >> 1) & 1) | ((i >> 2) & 2)), c = cb + ((i & 1) | ((i >> 1) & 2));
          if (r < nu && c < nu) Bv[r * nu + c] = o[i];
        }
      }
    }
  }
  if (poles && tid < nv) {
    B[(size_t)tid * N + 10 * (size_t)nu * nu] = bw[tid][R];
    B[(size_t)tid * N + 10 * (size_t)nu * nu + 1] = bw[tid][R + 1];
  }
}

bool relight_fusable(const tsr_compressed *c, int n_edit) {
  return c->wavelet == 0 && n_edit >= 1 && n_edit <= 2 && relight_fusable_basis(c);
}

bool relight_fusable_basis(const tsr_compressed *c) {
  return c->wavelet == 0 && c->P <= (1 << ((RF_MAX_LGN + RF_LGSEG) / 2)) && c->nnz < (1ll << 31);
}

// Dynamic shared memory of relight_fused_kernel<VV>: b^w when VV > 6.
template <int VV>
static size_t fused_smem() {
  return VV > 6 ? sizeof(float) * VV * RF_BW : 0;
}

// Launches relight_fused_kernel<VV> over the copies, RF_MAXC per launch.  g: per-copy
// [nv][K] pointers, or all null for the basis images (nv = K rows: c_k[kj] = l[j] for
// the entries of basis k).
template <int VV>
static tsr_status launch_fused(int n, const tsr_compressed *const *c, int nv, const float *const *gi, const float *l,
                               float *const *Bi, cudaStream_t s) {
  const int K = c[0]->K, J = c[0]->J;
  const size_t smem = fused_smem<VV>();
  const unsigned m2J = (unsigned)(((1ull << 32) + 2u * (unsigned)J - 1) / (2u * (unsigned)J));   // kj / J, see rf_fma
  {   // dynamic shared memory up to the largest case (K = 16, J = 32), set once per device
    static std::atomic<bool> attr_set[64];   // the call is idempotent: threads racing here set the same value
    int dev = 0;
    TSR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
      TSR_CUDA(cudaFuncSetAttribute(relight_fused_kernel<VV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)fused_smem<VV>()));
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
    relight_fused_kernel<VV><<<items, RF_THREADS, smem, s>>>(bt, K, J, m2J, l);
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
