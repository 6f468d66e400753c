// Self-shadowed SH irradiance transfer (Section 3, E(x_i) of Eq. 6, with the
// visibility term of Section 4's irradiance, E = V L, E11-E14): on displaced meshes
// part of the hemisphere above x_i is hidden by the mesh itself.
//   T[j][i] = (pi / S) sum_s Y_j(w_s) V(x_i, w_s) [F_t(eta, mu_s)]
// with w_s the S cosine-weighted Hammersley directions (u1 = (s + 1/2)/S, u2 the
// bit-reversed s; r = sqrt u1, phi = 2 pi u2, mu = sqrt(1 - u1)) in the frame of the
// unit normal n_i built by the branchless construction of Duff et al. (2017), rays
// from x_i + eps n_i, and V = 0 when the ray hits any triangle (Moller-Trumbore in
// FP32 with a fixed operation order, no contraction: the same decision the
// reference takes).
//
// GB300 layout: a linear BVH built on the device (Karras 2012): 30-bit Morton keys of
// the triangle centroids, made unique by appending the triangle index, sorted by CUB;
// internal nodes by the longest-common-prefix split; boxes bottom-up (the second
// child to arrive at a node merges), expanded by a small margin so that the box test
// never rejects a ray the exact triangle test would accept.  Tracing: a thread per
// vertex, its S rays in turn (any-hit, stack traversal), the J sums in registers.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "handles.cuh"

namespace tsr {

constexpr double kPiV = 3.14159265358979323846;
constexpr int VIS_STACK = 64;

struct Aabb {
  float lo[3], hi[3];
};

// ---------------------------------------------------------------- BVH build
__device__ __forceinline__ unsigned spread3(unsigned v) {   // 10 bits -> every third bit
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__global__ void tri_box_kernel(int F, const float *__restrict__ pos, int N, const int *__restrict__ tris,
                               Aabb *__restrict__ box, float *__restrict__ cen) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  Aabb b;
  for (int a = 0; a < 3; ++a) {
    const float x0 = pos[(size_t)a * N + tris[3 * f]], x1 = pos[(size_t)a * N + tris[3 * f + 1]],
                x2 = pos[(size_t)a * N + tris[3 * f + 2]];
    b.lo[a] = fminf(x0, fminf(x1, x2));
    b.hi[a] = fmaxf(x0, fmaxf(x1, x2));
    cen[(size_t)a * F + f] = 0.5f * (b.lo[a] + b.hi[a]);
  }
  box[f] = b;
}

// scene bounds of the centroids (one block)
__global__ void __launch_bounds__(1024) centroid_bounds_kernel(int F, const float *__restrict__ cen,
                                                               float *__restrict__ bounds) {
  __shared__ float red[6][32];
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  for (int f = threadIdx.x; f < F; f += blockDim.x)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], cen[(size_t)a * F + f]);
      hi[a] = fmaxf(hi[a], cen[(size_t)a * F + f]);
    }
  for (int a = 0; a < 3; ++a)
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; ++a) {
      red[a][threadIdx.x >> 5] = lo[a];
      red[3 + a][threadIdx.x >> 5] = hi[a];
    }
  __syncthreads();
  if (threadIdx.x < 3) {
    float l = 3e38f, h = -3e38f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      l = fminf(l, red[threadIdx.x][w]);
      h = fmaxf(h, red[3 + threadIdx.x][w]);
    }
    bounds[threadIdx.x] = l;
    bounds[3 + threadIdx.x] = h;
  }
}

__global__ void morton_key_kernel(int F, const float *__restrict__ cen, const float *__restrict__ bounds,
                                  unsigned long long *__restrict__ keys) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  unsigned q[3];
  for (int a = 0; a < 3; ++a) {
    const float ext = fmaxf(bounds[3 + a] - bounds[a], 1e-30f);
    const float u = fminf(fmaxf((cen[(size_t)a * F + f] - bounds[a]) / ext, 0.0f), 1.0f);
    q[a] = min(1023u, (unsigned)(u * 1024.0f));
  }
  const unsigned code = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
  keys[f] = ((unsigned long long)code << 32) | (unsigned)f;   // unique: the index breaks ties
}

// longest common prefix of sorted keys i and j (-1 outside [0, n))
__device__ __forceinline__ int lcp(const unsigned long long *keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  return __clzll(keys[i] ^ keys[j]);
}

// Internal node i of n - 1 (Karras 2012): children encoded as >= 0 internal, < 0 leaf ~index.
__global__ void build_internal_kernel(int n, const unsigned long long *__restrict__ keys, int *__restrict__ left,
                                      int *__restrict__ right, int *__restrict__ parent) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int d = (lcp(keys, n, i, i + 1) - lcp(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = lcp(keys, n, i, i - d);
  int lmax = 2;
  while (lcp(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (lcp(keys, n, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = lcp(keys, n, i, j);
  int s = 0;
  for (int div = 2;; div <<= 1) {
    const int t = (l + div - 1) / div;
    if (lcp(keys, n, i, i + (s + t) * d) > dnode) s += t;
    if (t <= 1) break;
  }
  const int g = i + s * d + min(d, 0);
  const int lc = (min(i, j) == g) ? ~g : g;
  const int rc = (max(i, j) == g + 1) ? ~(g + 1) : g + 1;
  left[i] = lc;
  right[i] = rc;
  if (lc >= 0) parent[lc] = i; else parent[(n - 1) + ~lc] = i;
  if (rc >= 0) parent[rc] = i; else parent[(n - 1) + ~rc] = i;
}

// Boxes bottom-up: leaf boxes from the sorted triangles, then each internal node's box
// by the second of its children to arrive.  Leaf l's parent is parent[n - 1 + l].
__global__ void bottom_up_kernel(int n, const unsigned long long *__restrict__ keys, const Aabb *__restrict__ tri_box,
                                 const int *__restrict__ left, const int *__restrict__ right,
                                 const int *__restrict__ parent, float margin, Aabb *__restrict__ leaf_box,
                                 Aabb *__restrict__ node_box, int *__restrict__ arrived) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  Aabb b = tri_box[(unsigned)(keys[l] & 0xFFFFFFFFull)];
  for (int a = 0; a < 3; ++a) {
    b.lo[a] -= margin;
    b.hi[a] += margin;
  }
  leaf_box[l] = b;
  if (n == 1) return;
  int p = parent[n - 1 + l];
  while (p >= 0) {
    __threadfence();
    if (atomicAdd(&arrived[p], 1) == 0) return;   // the sibling is not done yet
    __threadfence();
    const int lc = left[p], rc = right[p];
    const Aabb A = lc >= 0 ? node_box[lc] : leaf_box[~lc];
    const Aabb B = rc >= 0 ? node_box[rc] : leaf_box[~rc];
    Aabb u;
    for (int a = 0; a < 3; ++a) {
      u.lo[a] = fminf(A.lo[a], B.lo[a]);
      u.hi[a] = fmaxf(A.hi[a], B.hi[a]);
    }
    node_box[p] = u;
    p = (p == 0) ? -1 : parent[p];
  }
}

// ---------------------------------------------------------------- tracing
// Moller-Trumbore in FP32, no contraction, the reference's operation order.
__device__ __forceinline__ float dot3(const float *a, const float *b) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a[0], b[0]), __fmul_rn(a[1], b[1])), __fmul_rn(a[2], b[2]));
}
__device__ __forceinline__ void cross3(const float *a, const float *b, float *c) {
  c[0] = __fsub_rn(__fmul_rn(a[1], b[2]), __fmul_rn(a[2], b[1]));
  c[1] = __fsub_rn(__fmul_rn(a[2], b[0]), __fmul_rn(a[0], b[2]));
  c[2] = __fsub_rn(__fmul_rn(a[0], b[1]), __fmul_rn(a[1], b[0]));
}

__device__ bool tri_hit(const float *o, const float *d, const float *v0, const float *v1, const float *v2) {
  float e1[3], e2[3], p[3], tv[3], q[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = __fsub_rn(v1[a], v0[a]);
    e2[a] = __fsub_rn(v2[a], v0[a]);
    tv[a] = __fsub_rn(o[a], v0[a]);
  }
  cross3(d, e2, p);
  const float det = dot3(e1, p);
  if (!(fabsf(det) >= 1e-12f)) return false;
  const float inv = __fdiv_rn(1.0f, det);
  const float u = __fmul_rn(dot3(tv, p), inv);
  if (!(u >= 0.0f)) return false;
  cross3(tv, e1, q);
  const float v = __fmul_rn(dot3(d, q), inv);
  if (!(v >= 0.0f) || !(__fadd_rn(u, v) <= 1.0f)) return false;
  const float t = __fmul_rn(dot3(e2, q), inv);
  return t > 1e-4f;
}

__device__ __forceinline__ bool box_hit(const Aabb &b, const float *o, const float *inv_d) {
  float t0 = 0.0f, t1 = 3e38f;
  for (int a = 0; a < 3; ++a) {
    float ta = (b.lo[a] - o[a]) * inv_d[a], tb = (b.hi[a] - o[a]) * inv_d[a];
    if (ta > tb) {
      const float x = ta;
      ta = tb;
      tb = x;
    }
    t0 = fmaxf(t0, ta);
    t1 = fminf(t1, tb);
  }
  return t0 <= t1;
}

// Local cosine-weighted directions of the Hammersley set (FP64, kept in FP32) and mu_s.
__global__ void hemisphere_kernel(int S, float *__restrict__ loc, double *__restrict__ mu) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double u1 = (s + 0.5) / S;
  const double u2 = (double)__brev((unsigned)s) * (1.0 / 4294967296.0);
  const double r = sqrt(u1);
  loc[3 * s] = (float)(r * cos(2.0 * kPiV * u2));
  loc[3 * s + 1] = (float)(r * sin(2.0 * kPiV * u2));
  loc[3 * s + 2] = (float)sqrt(1.0 - u1);
  mu[s] = sqrt(1.0 - u1);
}

// real orthonormal SH (no Condon-Shortley phase) of a unit direction, FP32, l < order <= 5
__device__ void sh_eval_f32(int order, const float *w, float *Y) {
  const float z = fminf(fmaxf(w[2], -1.0f), 1.0f);
  const float st = sqrtf(fmaxf(0.0f, 1.0f - z * z));
  const float phi = atan2f(w[1], w[0]);
  float P[5][5];
  P[0][0] = 1.0f;
  for (int m = 1; m < order; ++m) P[m][m] = P[m - 1][m - 1] * (2 * m - 1) * st;
  for (int m = 0; m < order; ++m) {
    if (m + 1 < order) P[m + 1][m] = z * (2 * m + 1) * P[m][m];
    for (int l = m + 2; l < order; ++l) P[l][m] = ((2 * l - 1) * z * P[l - 1][m] - (l + m - 1) * P[l - 2][m]) / (l - m);
  }
  for (int l = 0; l < order; ++l)
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      float ratio = 1.0f;
      for (int q = l - am + 1; q <= l + am; ++q) ratio /= q;
      const float K = sqrtf((2 * l + 1) / (4.0f * (float)kPiV) * ratio);
      float v;
      if (m == 0) v = K * P[l][0];
      else if (m > 0) v = 1.41421356f * K * cosf(m * phi) * P[l][am];
      else v = 1.41421356f * K * sinf(am * phi) * P[l][am];
      Y[l * l + l + m] = v;
    }
}

__global__ void __launch_bounds__(128) trace_kernel(int N, const float *__restrict__ pos,
                                                    const float *__restrict__ normals, int F,
                                                    const int *__restrict__ tris, int n_leaf,
                                                    const unsigned long long *__restrict__ keys,
                                                    const int *__restrict__ left, const int *__restrict__ right,
                                                    const Aabb *__restrict__ node_box,
                                                    const Aabb *__restrict__ leaf_box, int S,
                                                    const float *__restrict__ loc, const double *__restrict__ mu,
                                                    double eta, float eps, int order, float *__restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int J = order * order;
  const float n32[3] = {normals[i], normals[N + i], normals[2 * N + i]};
  // frame of the normal in FP64 (Duff et al.), kept in FP32
  const double nx = n32[0], ny = n32[1], nz = n32[2];
  const double sign = nz >= 0.0 ? 1.0 : -1.0;
  const double a = -1.0 / (sign + nz), b = nx * ny * a;
  const float t1[3] = {(float)(1.0 + sign * nx * nx * a), (float)(sign * b), (float)(-sign * nx)};
  const float t2[3] = {(float)b, (float)(sign + ny * ny * a), (float)(-ny)};
  float o[3];
  for (int c = 0; c < 3; ++c) o[c] = __fadd_rn(pos[(size_t)c * N + i], __fmul_rn(eps, n32[c]));
  float acc[25];
  for (int q = 0; q < J; ++q) acc[q] = 0.0f;
  const float w0 = (float)(kPiV / S);
  for (int s = 0; s < S; ++s) {
    const float l0 = loc[3 * s], l1 = loc[3 * s + 1], l2 = loc[3 * s + 2];
    float d[3], inv_d[3];
    for (int c = 0; c < 3; ++c) {
      d[c] = __fadd_rn(__fadd_rn(__fmul_rn(l0, t1[c]), __fmul_rn(l1, t2[c])), __fmul_rn(l2, n32[c]));
      inv_d[c] = 1.0f / d[c];
    }
    // any-hit traversal
    bool hit = false;
    if (n_leaf == 1) {
      const int f = (int)(keys[0] & 0xFFFFFFFFull);
      float v0[3], v1[3], v2[3];
      for (int c = 0; c < 3; ++c) {
        v0[c] = pos[(size_t)c * N + tris[3 * f]];
        v1[c] = pos[(size_t)c * N + tris[3 * f + 1]];
        v2[c] = pos[(size_t)c * N + tris[3 * f + 2]];
      }
      hit = tri_hit(o, d, v0, v1, v2);
    } else {
      int stack[VIS_STACK];
      int sp = 0;
      stack[sp++] = 0;
      while (sp > 0 && !hit) {
        const int node = stack[--sp];
        const int ch[2] = {left[node], right[node]};
        for (int k = 0; k < 2 && !hit; ++k) {
          const int c = ch[k];
          if (c < 0) {
            if (!box_hit(leaf_box[~c], o, inv_d)) continue;
            const int f = (int)(keys[~c] & 0xFFFFFFFFull);
            float v0[3], v1[3], v2[3];
            for (int e = 0; e < 3; ++e) {
              v0[e] = pos[(size_t)e * N + tris[3 * f]];
              v1[e] = pos[(size_t)e * N + tris[3 * f + 1]];
              v2[e] = pos[(size_t)e * N + tris[3 * f + 2]];
            }
            hit = tri_hit(o, d, v0, v1, v2);
          } else if (box_hit(node_box[c], o, inv_d)) {
            if (sp < VIS_STACK) stack[sp++] = c;
          }
        }
      }
    }
    if (hit) continue;
    float w = w0;
    if (eta > 0.0) {   // incident Fresnel factor at the sample's cosine
      const double m = mu[s];
      const double ct = sqrt(fmax(1.0 - (1.0 - m * m) / (eta * eta), 0.0));
      const double rs = (m - eta * ct) / (m + eta * ct), rp = (eta * m - ct) / (eta * m + ct);
      w = (float)(w0 * (1.0 - 0.5 * (rs * rs + rp * rp)));
    }
    float Y[25];
    sh_eval_f32(order, d, Y);
    for (int q = 0; q < J; ++q) acc[q] = fmaf(w, Y[q], acc[q]);
  }
  for (int q = 0; q < J; ++q) T[(size_t)q * N + i] = acc[q];
}

tsr_status visibility_transfer(int N, const float *pos, const float *normals, int F, const int *tris, int J, int S,
                               double eta, float eps, float *T, cudaStream_t s) {
  const int order = (int)lround(std::sqrt((double)J));
  const int n = F, n_int = std::max(F - 1, 1);
  Scratch sc;
  const size_t b_box = sizeof(Aabb) * (size_t)F, b_cen = sizeof(float) * 3 * (size_t)F,
               b_keys = sizeof(unsigned long long) * (size_t)F, b_int = sizeof(int) * (size_t)n_int,
               b_par = sizeof(int) * (size_t)(n_int + F), b_loc = sizeof(float) * 3 * (size_t)S,
               b_mu = sizeof(double) * (size_t)S;
  // sort scratch size
  size_t sort_bytes = 0;
  cub::DeviceRadixSort::SortKeys(nullptr, sort_bytes, (unsigned long long *)nullptr, (unsigned long long *)nullptr,
                                 F, 0, 64, s);
  const size_t total = 2 * b_box + b_cen + 2 * b_keys + 3 * b_int + b_par + sizeof(Aabb) * (size_t)n_int + b_loc +
                       b_mu + sort_bytes + 64 + 16 * 16;
  tsr_status st = sc.alloc(total, s);
  if (st != TSR_OK) return st;
  uint8_t *p = static_cast<uint8_t *>(sc.p);
  auto take = [&](size_t bytes) {
    uint8_t *q = p;
    p += (bytes + 15) / 16 * 16;
    return q;
  };
  Aabb *tri_box = reinterpret_cast<Aabb *>(take(b_box));
  Aabb *leaf_box = reinterpret_cast<Aabb *>(take(b_box));
  float *cen = reinterpret_cast<float *>(take(b_cen));
  unsigned long long *keys_in = reinterpret_cast<unsigned long long *>(take(b_keys));
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(take(b_keys));
  int *left = reinterpret_cast<int *>(take(b_int));
  int *right = reinterpret_cast<int *>(take(b_int));
  int *arrived = reinterpret_cast<int *>(take(b_int));
  int *parent = reinterpret_cast<int *>(take(b_par));
  Aabb *node_box = reinterpret_cast<Aabb *>(take(sizeof(Aabb) * (size_t)n_int));
  float *loc = reinterpret_cast<float *>(take(b_loc));
  double *mu = reinterpret_cast<double *>(take(b_mu));
  float *bounds = reinterpret_cast<float *>(take(64));
  void *sort_tmp = take(sort_bytes);

  tri_box_kernel<<<(F + 255) / 256, 256, 0, s>>>(F, pos, N, tris, tri_box, cen); ::tsr::count_launch();
  centroid_bounds_kernel<<<1, 1024, 0, s>>>(F, cen, bounds); ::tsr::count_launch();
  morton_key_kernel<<<(F + 255) / 256, 256, 0, s>>>(F, cen, bounds, keys_in); ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  TSR_CUDA(cub::DeviceRadixSort::SortKeys(sort_tmp, sort_bytes, keys_in, keys, F, 0, 64, s));
  ::tsr::count_launch();
  TSR_CUDA(cudaMemsetAsync(arrived, 0, b_int, s));
  if (n > 1) {
    build_internal_kernel<<<(n - 1 + 255) / 256, 256, 0, s>>>(n, keys, left, right, parent); ::tsr::count_launch();
  }
  // margin: a few FP32 ulps of the scene size, so that box tests are conservative
  const float margin = 1e-5f;
  bottom_up_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, keys, tri_box, left, right, parent, margin, leaf_box,
                                                   node_box, arrived);
  ::tsr::count_launch();
  hemisphere_kernel<<<(S + 255) / 256, 256, 0, s>>>(S, loc, mu); ::tsr::count_launch();
  trace_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, pos, normals, F, tris, n, keys, left, right, node_box, leaf_box,
                                               S, loc, mu, eta, eps, order, T);
  ::tsr::count_launch();
  TSR_CUDA(cudaGetLastError());
  return TSR_OK;
}

}  // namespace tsr
