// mrdem_build.cu -- construction of the surrogate trees on the GPU.
//
// The same trees as the host builder (mrdem_hierarchy.cpp) describes, after
// Sec. 4, Algorithm 7 and Appendix A of Noble & Weinzierl (arXiv 2105.12415),
// built for all particles at once:
//   * shape: a node holding more than leaf_max fine triangles is split into
//     k clusters of prescribed sizes (n / k, the first n mod k one larger;
//     k = fanout, fewer when the clusters would fall below leaf_min).  The
//     shape depends on the counts alone, so the host lays out every node and
//     its range of a triangle permutation before any geometry is read;
//   * clusters: the recursive median split of the balanced k-means seeding:
//     a node's range is bisected along the principal axis of its triangle
//     centroids so that the first part holds the sizes of the first half of
//     its clusters, and so on down to single clusters.  One block per range
//     (k_bisect) finds the principal axis (FP64 covariance, Jacobi
//     rotations) and the element of the required rank by a radix select over
//     (projection, triangle index) keys, then partitions the range stably;
//     ranges of one tree level and one bisection depth run in one launch.
//     The Lloyd refinement of the host builder's k-means is not run: the
//     seeding already gives compact clusters of the prescribed sizes, and
//     correctness does not depend on the clusters (each surrogate's slack is
//     exact);
//   * per node (k_fit, one block per node): the surrogate triangle, fitted
//     to the corners of the node's triangles to make the largest distance
//     small (Appendix A's first term): the principal plane's enclosing
//     triangle with edge normals 120 degrees apart, scaled about its centroid,
//     then a coordinate descent on its nine coordinates (float, on at most
//     1536 sampled corners); its slack delta, the largest FP64 distance from
//     any corner to the stored float triangle, rounded up (the conservative
//     environment of Sec. 4); and the oriented box of the corners
//     (principal axes in float, FP64 extents rounded up).
// The result is handed to the host hierarchy record and uploaded like a host
// build (mrdem_hier_upload derives node spheres, planes and slot records).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mrdem_device.cuh"

namespace mrdem {
namespace {

using D3 = V3<double>;

constexpr int kBisectThreads = 256;
constexpr int kFitThreads = 128;
constexpr int kSample = 1536;  // corners the surrogate fit optimises on

// Bisection of perm[begin, begin + count): the nl elements of smallest key
// first (keys: projection on the principal axis, then triangle index).
struct BisectTask {
  int64_t begin;
  int32_t count, nl;
};

struct FitArgs {
  const int32_t* perm;       // global triangle indices, node ranges contiguous
  const int64_t* node_begin; // [n_nodes] range of each node in perm
  const int32_t* node_count;
  const int32_t* node_particle;
  const float* verts;        // body-frame vertices (all particles)
  const int32_t* tris;       // local vertex indices
  const int64_t* vert_off;   // [n + 1]
  const int64_t* tri_off;    // [n + 1]
  float* node_tri;           // [n_nodes * 9] out
  float* node_delta;         // [n_nodes] out
  float* node_box;           // [n_nodes * 16] out
  int32_t* error;            // set to 1 when a fitted surrogate is degenerate
  int64_t n_nodes;
};

// Sums of a block (all threads call; `vals` of N doubles per thread; the
// results are returned on every thread).
template <int N, int THREADS>
__device__ void block_sum(double (&vals)[N], double* smem /* [32 * N] */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k)
    for (int o = 16; o > 0; o >>= 1) vals[k] += __shfl_xor_sync(0xffffffffu, vals[k], o);
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < N; ++k) smem[w * N + k] = vals[k];
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    double s = 0.0;
    for (int j = 0; j < THREADS / 32; ++j) s += smem[j * N + k];
    vals[k] = s;
  }
}
template <int THREADS>
__device__ double block_max(double v, double* smem) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) smem[w] = v;
  __syncthreads();
  double m = smem[0];
  for (int j = 1; j < THREADS / 32; ++j) m = fmax(m, smem[j]);
  return m;
}
template <int THREADS>
__device__ float block_max_f(float v, float* smem) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) smem[w] = v;
  __syncthreads();
  float m = smem[0];
  for (int j = 1; j < THREADS / 32; ++j) m = fmaxf(m, smem[j]);
  return m;
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
// (each rotation annihilates one off-diagonal entry); eigenvalues ascending
// in w, eigenvectors as the columns of V.
__device__ void jacobi3(double A[3][3], double w[3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-30 * diag || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  int idx[3] = {0, 1, 2};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2 - i; ++j)
      if (A[idx[j]][idx[j]] > A[idx[j + 1]][idx[j + 1]]) {
        const int t = idx[j];
        idx[j] = idx[j + 1];
        idx[j + 1] = t;
      }
  double Vs[3][3];
  for (int c = 0; c < 3; ++c) {
    w[c] = A[idx[c]][idx[c]];
    for (int r = 0; r < 3; ++r) Vs[r][c] = V[r][idx[c]];
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) V[r][c] = Vs[r][c];
}

// Total order of floats as unsigned integers.
__device__ __forceinline__ uint32_t ordered_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// k_bisect: one block per task.
__global__ void __launch_bounds__(kBisectThreads) k_bisect(const BisectTask* __restrict__ tasks,
                                                           int n_tasks, int32_t* perm,
                                                           int32_t* tmp,
                                                           const double* __restrict__ cen) {
  __shared__ double red[32 * 9];
  __shared__ double axis_s[3];
  __shared__ unsigned hist[256];
  __shared__ uint64_t prefix_s;
  __shared__ int rank_s;
  __shared__ int scan_s[kBisectThreads / 32];
  for (int t = blockIdx.x; t < n_tasks; t += gridDim.x) {
    const BisectTask task = tasks[t];
    const int64_t b = task.begin;
    const int n = task.count;
    // mean, then covariance of the centroids
    double m[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < n; i += kBisectThreads) {
      const double* c = cen + 3 * (int64_t)perm[b + i];
      m[0] += c[0]; m[1] += c[1]; m[2] += c[2];
    }
    block_sum<3, kBisectThreads>(m, red);
    for (int k = 0; k < 3; ++k) m[k] /= n;
    double C[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += kBisectThreads) {
      const double* c = cen + 3 * (int64_t)perm[b + i];
      const double d0 = c[0] - m[0], d1 = c[1] - m[1], d2 = c[2] - m[2];
      C[0] += d0 * d0; C[1] += d0 * d1; C[2] += d0 * d2;
      C[3] += d1 * d1; C[4] += d1 * d2; C[5] += d2 * d2;
    }
    block_sum<6, kBisectThreads>(C, red);
    if (threadIdx.x == 0) {
      double A[3][3] = {{C[0], C[1], C[2]}, {C[1], C[3], C[4]}, {C[2], C[4], C[5]}};
      double w[3], V[3][3];
      jacobi3(A, w, V);
      for (int k = 0; k < 3; ++k) axis_s[k] = V[k][2];  // the largest variance
      prefix_s = 0;
      rank_s = task.nl;
    }
    __syncthreads();
    const double ax[3] = {axis_s[0], axis_s[1], axis_s[2]};
    auto key_of = [&](int i) -> uint64_t {
      const int32_t g = perm[b + i];
      const double* c = cen + 3 * (int64_t)g;
      const float pr = (float)((c[0] - m[0]) * ax[0] + (c[1] - m[1]) * ax[1] + (c[2] - m[2]) * ax[2]);
      return ((uint64_t)ordered_bits(pr) << 32) | (uint32_t)g;
    };
    // radix select: the key of rank nl (keys are distinct)
    for (int shift = 56; shift >= 0; shift -= 8) {
      for (int k = threadIdx.x; k < 256; k += kBisectThreads) hist[k] = 0;
      __syncthreads();
      const uint64_t pre = prefix_s;
      const uint64_t hi_mask = shift == 56 ? 0ull : ~0ull << (shift + 8);
      for (int i = threadIdx.x; i < n; i += kBisectThreads) {
        const uint64_t k = key_of(i);
        if ((k & hi_mask) == pre) atomicAdd(&hist[(k >> shift) & 255u], 1u);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int r = rank_s, d = 0;
        while (d < 255 && r >= (int)hist[d]) r -= (int)hist[d++];
        rank_s = r;
        prefix_s = pre | ((uint64_t)d << shift);
      }
      __syncthreads();
    }
    const uint64_t pivot = prefix_s;
    // stable partition: keys below the pivot first, into tmp, then back
    int base_l = 0, base_r = task.nl;
    for (int c0 = 0; c0 < n; c0 += kBisectThreads) {
      const int i = c0 + threadIdx.x;
      const bool in = i < n;
      const int32_t g = in ? perm[b + i] : 0;
      const bool left = in && key_of(i) < pivot;
      const unsigned bl = __ballot_sync(0xffffffffu, left), br = __ballot_sync(0xffffffffu, in && !left);
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
      if (lane == 0) scan_s[w] = __popc(bl) | (__popc(br) << 16);
      __syncthreads();
      int ol = 0, orr = 0, tl = 0, tr = 0;
      for (int j = 0; j < kBisectThreads / 32; ++j) {
        const int v = scan_s[j];
        if (j < w) { ol += v & 0xffff; orr += v >> 16; }
        tl += v & 0xffff;
        tr += v >> 16;
      }
      const unsigned below = (1u << lane) - 1u;
      if (left) tmp[b + base_l + ol + __popc(bl & below)] = g;
      else if (in) tmp[b + base_r + orr + __popc(br & below)] = g;
      base_l += tl;
      base_r += tr;
      __syncthreads();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kBisectThreads) perm[b + i] = tmp[b + i];
    __syncthreads();
  }
}

// Centroid of every fine triangle (FP64, body frame) and the validity of the
// input: indices inside the particle's vertices, finite coordinates, no
// degenerate triangle.
__global__ void k_centroids(int n, const int64_t* __restrict__ vert_off,
                            const int64_t* __restrict__ tri_off, const float* __restrict__ verts,
                            const int32_t* __restrict__ tris, int64_t n_tri,
                            const int32_t* __restrict__ tri_particle, double* cen,
                            int32_t* error) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tri;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int p = tri_particle[t];
    const int64_t nv = vert_off[p + 1] - vert_off[p];
    const float* V = verts + 3 * vert_off[p];
    D3 x[3];
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
      const int32_t v = tris[3 * t + k];
      ok = ok && v >= 0 && v < nv;
      x[k] = ok ? D3{V[3 * v], V[3 * v + 1], V[3 * v + 2]} : D3{0, 0, 0};
      ok = ok && isfinite(x[k].x) && isfinite(x[k].y) && isfinite(x[k].z);
    }
    const D3 nr = cross(x[1] - x[0], x[2] - x[0]);
    ok = ok && dot(nr, nr) > 0.0;
    if (!ok) atomicExch(error, 1);
    const D3 c = (1.0 / 3.0) * (x[0] + x[1] + x[2]);
    cen[3 * t] = c.x;
    cen[3 * t + 1] = c.y;
    cen[3 * t + 2] = c.z;
  }
}

__device__ float round_up_f32(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, FLT_MAX);
  return f;
}

// Largest squared distance of the staged sample points to triangle T (float,
// coordinates relative to the node's mean); block-wide.
__device__ float sample_max_dist2(const float* sx, const float* sy, const float* sz, int ns,
                                  const F3 T[3], float* red) {
  float m = 0.f;
  for (int i = threadIdx.x; i < ns; i += kFitThreads) {
    float w[3];
    const F3 p = {sx[i], sy[i], sz[i]};
    const F3 q = closest_on_triangle(p, T[0], T[1], T[2], w);
    const F3 d = p - q;
    m = fmaxf(m, dot(d, d));
  }
  return block_max_f<kFitThreads>(m, red);
}

__device__ __forceinline__ float tri_area_f(const F3 T[3]) {
  const F3 n = cross(T[1] - T[0], T[2] - T[0]);
  return 0.5f * sqrtf(dot(n, n));
}

// k_fit: surrogate triangle, slack and oriented box of every node.
__global__ void __launch_bounds__(kFitThreads) k_fit(FitArgs A) {
  __shared__ float sx[kSample], sy[kSample], sz[kSample];
  __shared__ double dred[32 * 12];
  __shared__ float fred[32];
  __shared__ float hbest[72];
  __shared__ double basis_s[12];  // e1, e2, n, mean
  __shared__ double box_s[12];    // box axes (float-rounded) and centre
  __shared__ float cand_s[9 * 10];
  __shared__ int ctl_s[2];
  for (int64_t node = blockIdx.x; node < A.n_nodes; node += gridDim.x) {
    const int64_t b = A.node_begin[node];
    const int n = A.node_count[node];
    const int p = A.node_particle[node];
    const float* V = A.verts + 3 * A.vert_off[p];
    const int npts = 3 * n;
    auto corner = [&](int i) -> D3 {
      const int64_t t = A.perm[b + i / 3];
      const int32_t v = A.tris[3 * t + i % 3];
      return {V[3 * v], V[3 * v + 1], V[3 * v + 2]};
    };
    // mean, covariance and the sum of the triangles' normals (orientation)
    double s[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < npts; i += kFitThreads) {
      const D3 c = corner(i);
      s[0] += c.x; s[1] += c.y; s[2] += c.z;
    }
    block_sum<3, kFitThreads>(s, dred);
    const D3 mean = {s[0] / npts, s[1] / npts, s[2] / npts};
    double C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < npts; i += kFitThreads) {
      const D3 d = corner(i) - mean;
      C[0] += d.x * d.x; C[1] += d.x * d.y; C[2] += d.x * d.z;
      C[3] += d.y * d.y; C[4] += d.y * d.z; C[5] += d.z * d.z;
    }
    for (int j = threadIdx.x; j < n; j += kFitThreads) {
      const D3 a = corner(3 * j), bb = corner(3 * j + 1), c = corner(3 * j + 2);
      const D3 nr = cross(bb - a, c - a);
      C[6] += nr.x; C[7] += nr.y; C[8] += nr.z;
    }
    block_sum<9, kFitThreads>(C, dred);
    if (threadIdx.x == 0) {
      double M[3][3] = {{C[0], C[1], C[2]}, {C[1], C[3], C[4]}, {C[2], C[4], C[5]}};
      double w[3], E[3][3];
      jacobi3(M, w, E);
      D3 e1 = {E[0][2], E[1][2], E[2][2]}, e2 = {E[0][1], E[1][1], E[2][1]};
      D3 nn = {E[0][0], E[1][0], E[2][0]};
      if (dot(nn, D3{C[6], C[7], C[8]}) < 0) {  // keep (e1, e2, n) right-handed
        nn = -1.0 * nn;
        e2 = -1.0 * e2;
      }
      basis_s[0] = e1.x; basis_s[1] = e1.y; basis_s[2] = e1.z;
      basis_s[3] = e2.x; basis_s[4] = e2.y; basis_s[5] = e2.z;
      basis_s[6] = nn.x; basis_s[7] = nn.y; basis_s[8] = nn.z;
      // box axes: the principal axes, orthonormalised and rounded to float
      D3 u0 = {E[0][2], E[1][2], E[2][2]}, u1 = {E[0][1], E[1][1], E[2][1]};
      u0 = (1.0 / sqrt(dot(u0, u0))) * u0;
      u1 = u1 - dot(u1, u0) * u0;
      u1 = (1.0 / sqrt(dot(u1, u1))) * u1;
      const D3 u2 = cross(u0, u1);
      const D3 u[3] = {u0, u1, u2};
      for (int k = 0; k < 3; ++k) {
        box_s[3 * k] = (double)(float)u[k].x;
        box_s[3 * k + 1] = (double)(float)u[k].y;
        box_s[3 * k + 2] = (double)(float)u[k].z;
      }
    }
    __syncthreads();
    const D3 e1 = {basis_s[0], basis_s[1], basis_s[2]}, e2 = {basis_s[3], basis_s[4], basis_s[5]};
    const D3 nn = {basis_s[6], basis_s[7], basis_s[8]};
    // the sample (every corner, or a stride through them), relative to the
    // mean, in float
    const int ns = npts < kSample ? npts : kSample;
    const double step = (double)npts / ns;
    float zmin = FLT_MAX, zmax = -FLT_MAX;
    for (int i = threadIdx.x; i < ns; i += kFitThreads) {
      const D3 d = corner(ns == npts ? i : (int)(i * step)) - mean;
      sx[i] = (float)d.x;
      sy[i] = (float)d.y;
      sz[i] = (float)d.z;
      const float z = (float)dot(d, nn);
      zmin = fminf(zmin, z);
      zmax = fmaxf(zmax, z);
    }
    zmax = block_max_f<kFitThreads>(zmax, fred);
    zmin = -block_max_f<kFitThreads>(-zmin, fred);
    // the enclosing triangle with edge normals 120 degrees apart in the
    // principal plane: 24 orientations, the one of least perimeter
    const float kPi = 3.14159265358979f;
    const F3 fe1 = {(float)e1.x, (float)e1.y, (float)e1.z}, fe2 = {(float)e2.x, (float)e2.y, (float)e2.z};
    for (int o = threadIdx.x; o < 72; o += kFitThreads) {
      const float a = (2 * kPi / 3) * (o / 3) / 24.f + 2 * kPi * (o % 3) / 3;
      const float cx = cosf(a), cy = sinf(a);
      float m = -FLT_MAX;
      for (int i = 0; i < ns; ++i) {
        const F3 d = {sx[i], sy[i], sz[i]};
        m = fmaxf(m, cx * dot(d, fe1) + cy * dot(d, fe2));
      }
      hbest[o] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int best = 0;
      float bc = FLT_MAX;
      for (int s24 = 0; s24 < 24; ++s24) {
        const float c = hbest[3 * s24] + hbest[3 * s24 + 1] + hbest[3 * s24 + 2];
        if (c < bc) { bc = c; best = s24; }
      }
      const double th = (2 * 3.14159265358979323846 / 3) * best / 24.0;
      const double zmid = 0.5 * ((double)zmin + (double)zmax);
      D3 T0[3];
      for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3;
        const double a0 = th + 2 * 3.14159265358979323846 * k / 3;
        const double a1 = th + 2 * 3.14159265358979323846 * k1 / 3;
        const double ax = cos(a0), ay = sin(a0), bx = cos(a1), by = sin(a1);
        const double det = ax * by - ay * bx;
        const double h0 = hbest[3 * best + k], h1 = hbest[3 * best + k1];
        const double x = (h0 * by - ay * h1) / det, y = (ax * h1 - h0 * bx) / det;
        T0[k] = x * e1 + y * e2 + zmid * nn;
      }
      if (dot(cross(T0[1] - T0[0], T0[2] - T0[0]), nn) < 0) {
        const D3 t = T0[1];
        T0[1] = T0[2];
        T0[2] = t;
      }
      for (int k = 0; k < 3; ++k) {
        cand_s[3 * k] = (float)T0[k].x;
        cand_s[3 * k + 1] = (float)T0[k].y;
        cand_s[3 * k + 2] = (float)T0[k].z;
      }
    }
    __syncthreads();
    // scaled copies about the centroid: the best as the start
    F3 T[3] = {{cand_s[0], cand_s[1], cand_s[2]}, {cand_s[3], cand_s[4], cand_s[5]},
               {cand_s[6], cand_s[7], cand_s[8]}};
    const F3 cenT = (1.f / 3.f) * (T[0] + T[1] + T[2]);
    const float area0 = tri_area_f(T);
    const float scales[9] = {1.0f, 0.85f, 0.7f, 0.55f, 0.4f, 0.25f, 0.12f, 0.05f, 0.02f};
    float best = FLT_MAX;
    F3 B[3] = {T[0], T[1], T[2]};
    for (int si = 0; si < 9; ++si) {
      F3 Cc[3];
      for (int k = 0; k < 3; ++k) Cc[k] = cenT + scales[si] * (T[k] - cenT);
      const float m = sample_max_dist2(sx, sy, sz, ns, Cc, fred);
      if (m < best) {
        best = m;
        for (int k = 0; k < 3; ++k) B[k] = Cc[k];
      }
    }
    // coordinate descent on the nine coordinates (block-uniform control)
    float size = 0.f;
    for (int k = 0; k < 3; ++k) size = fmaxf(size, sqrtf(dot(B[k] - cenT, B[k] - cenT)));
    float stp = 0.1f * fmaxf(size, 1e-12f);
    const float min_area = 1e-4f * fmaxf(tri_area_f(B), 1e-6f * area0);
    int evals = 0;
    const int max_evals = ns > 512 ? 36 : 90;
    for (int round = 0; round < 6 && evals < max_evals; ++round) {
      bool improved = true;
      while (improved && evals < max_evals) {
        improved = false;
        for (int c = 0; c < 9 && evals < max_evals; ++c) {
          for (int sg = 0; sg < 2; ++sg) {
            F3 Cc[3] = {B[0], B[1], B[2]};
            float* coord = &Cc[c / 3].x + (c % 3);
            *coord += sg == 0 ? stp : -stp;
            if (tri_area_f(Cc) < min_area) continue;
            const float m = sample_max_dist2(sx, sy, sz, ns, Cc, fred);
            ++evals;
            if (m < best) {
              best = m;
              for (int k = 0; k < 3; ++k) B[k] = Cc[k];
              improved = true;
              break;
            }
          }
        }
      }
      stp *= 0.5f;
    }
    // the stored surrogate (float, body frame)
    F3 S[3];
    for (int k = 0; k < 3; ++k)
      S[k] = {(float)(mean.x + (double)B[k].x), (float)(mean.y + (double)B[k].y),
              (float)(mean.z + (double)B[k].z)};
    const D3 Sd[3] = {{S[0].x, S[0].y, S[0].z}, {S[1].x, S[1].y, S[1].z}, {S[2].x, S[2].y, S[2].z}};
    const D3 ns3 = cross(Sd[1] - Sd[0], Sd[2] - Sd[0]);
    if (threadIdx.x == 0 && !(dot(ns3, ns3) > 0.0)) atomicExch(A.error, 1);
    // slack: the largest FP64 distance of any corner to the stored triangle
    double dmax = 0.0;
    for (int i = threadIdx.x; i < npts; i += kFitThreads) {
      const D3 c = corner(i);
      double w[3];
      const D3 q = closest_on_triangle(c, Sd[0], Sd[1], Sd[2], w);
      const D3 d = c - q;
      dmax = fmax(dmax, dot(d, d));
    }
    dmax = block_max<kFitThreads>(dmax, dred);
    // box: extents along the float axes about the mean, then the half widths
    // about the float centre
    const D3 u[3] = {{box_s[0], box_s[1], box_s[2]}, {box_s[3], box_s[4], box_s[5]},
                     {box_s[6], box_s[7], box_s[8]}};
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int i = threadIdx.x; i < npts; i += kFitThreads) {
      const D3 d = corner(i) - mean;
      for (int k = 0; k < 3; ++k) {
        const double t = dot(u[k], d);
        lo[k] = fmin(lo[k], t);
        hi[k] = fmax(hi[k], t);
      }
    }
    for (int k = 0; k < 3; ++k) {
      hi[k] = block_max<kFitThreads>(hi[k], dred);
      lo[k] = -block_max<kFitThreads>(-lo[k], dred);
    }
    D3 cb = mean;
    for (int k = 0; k < 3; ++k) cb = cb + (0.5 * (lo[k] + hi[k])) * u[k];
    const D3 cf = {(double)(float)cb.x, (double)(float)cb.y, (double)(float)cb.z};
    double half[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < npts; i += kFitThreads) {
      const D3 d = corner(i) - cf;
      for (int k = 0; k < 3; ++k) half[k] = fmax(half[k], fabs(dot(u[k], d)));
    }
    for (int k = 0; k < 3; ++k) half[k] = block_max<kFitThreads>(half[k], dred);
    if (threadIdx.x == 0) {
      float* t = A.node_tri + 9 * node;
      for (int k = 0; k < 3; ++k) {
        t[3 * k] = S[k].x;
        t[3 * k + 1] = S[k].y;
        t[3 * k + 2] = S[k].z;
      }
      A.node_delta[node] = round_up_f32(sqrt(dmax) * (1.0 + 1e-12));
      float* bx = A.node_box + 16 * node;
      bx[0] = (float)cf.x; bx[1] = (float)cf.y; bx[2] = (float)cf.z;
      for (int k = 0; k < 3; ++k) {
        bx[3 + 3 * k] = (float)u[k].x;
        bx[4 + 3 * k] = (float)u[k].y;
        bx[5 + 3 * k] = (float)u[k].z;
        bx[12 + k] = round_up_f32(half[k] * (1.0 + 1e-12));
      }
      bx[15] = 0.f;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side: the trees' shape from the counts
struct HNode {
  int32_t particle, count, level;
  int64_t begin;
  int32_t first_child = -1, n_children = 0;
};

template <typename T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() { cudaFree(p); }
  bool alloc(size_t n) {
    return cudaMalloc(&p, sizeof(T) * (n ? n : 1)) == cudaSuccess;
  }
};

}  // namespace

int build_hierarchy_device(const mrdem_params& prm, int32_t n, const int64_t* vert_off,
                           const float* d_verts, const int64_t* tri_off, const int32_t* d_tris,
                           HierHost* out, double* ms) {
  if (n <= 0 || !vert_off || !d_verts || !tri_off || !d_tris || !out) return MRDEM_ERR_INVALID;
  if (prm.fanout < 2 || prm.fanout > 8 || prm.leaf_max < 1 || prm.leaf_max > 32 || prm.leaf_min < 1)
    return MRDEM_ERR_INVALID;
  if (vert_off[0] != 0 || tri_off[0] != 0) return MRDEM_ERR_INVALID;
  for (int i = 0; i < n; ++i)
    if (vert_off[i + 1] <= vert_off[i] || tri_off[i + 1] <= tri_off[i]) return MRDEM_ERR_INVALID;
  if (tri_off[n] >= (int64_t)1 << 31 || vert_off[n] >= (int64_t)1 << 31) return MRDEM_ERR_INVALID;
  const int64_t n_tri = tri_off[n], n_verts = vert_off[n];
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaEventRecord(ev0);
  try {
    // ---- shape: nodes level by level, children contiguous; the bisection
    // tasks of each (level, depth)
    std::vector<HNode> nodes;
    nodes.reserve((size_t)(n_tri / std::max(1, prm.leaf_max)) * 2 + n + 16);
    for (int i = 0; i < n; ++i) nodes.push_back({i, (int32_t)(tri_off[i + 1] - tri_off[i]), 1, tri_off[i]});
    std::vector<std::vector<std::vector<BisectTask>>> tasks;  // [level][depth]
    size_t lo = 0, hi = nodes.size();
    int max_depth = 1;
    while (lo < hi) {
      std::vector<std::vector<BisectTask>> lt;
      for (size_t q = lo; q < hi; ++q) {
        const int cnt = nodes[q].count;
        if (cnt <= prm.leaf_max) continue;
        int k = prm.fanout;
        if (cnt / prm.fanout < prm.leaf_min)
          k = std::min(prm.fanout, std::max(2, (cnt + prm.leaf_max - 1) / prm.leaf_max));
        k = std::min(k, cnt);
        std::vector<int> sizes(k);
        for (int j = 0; j < k; ++j) sizes[j] = cnt / k + (j < cnt % k ? 1 : 0);
        // the median-split recursion over cluster ranges [k0, k1)
        struct R { int64_t b; int k0, k1, depth; };
        std::vector<R> st = {{nodes[q].begin, 0, k, 0}};
        while (!st.empty()) {
          R r = st.back();
          st.pop_back();
          if (r.k1 - r.k0 < 2) continue;
          const int km = (r.k0 + r.k1) / 2;
          int nl = 0, nt = 0;
          for (int j = r.k0; j < r.k1; ++j) {
            nt += sizes[j];
            if (j < km) nl += sizes[j];
          }
          if ((int)lt.size() <= r.depth) lt.resize(r.depth + 1);
          lt[r.depth].push_back({r.b, nt, nl});
          st.push_back({r.b, r.k0, km, r.depth + 1});
          st.push_back({r.b + nl, km, r.k1, r.depth + 1});
        }
        nodes[q].first_child = (int32_t)nodes.size();
        nodes[q].n_children = k;
        int64_t b = nodes[q].begin;
        for (int j = 0; j < k; ++j) {
          nodes.push_back({nodes[q].particle, sizes[j], nodes[q].level + 1, b});
          b += sizes[j];
          max_depth = std::max(max_depth, nodes[q].level + 1);
        }
      }
      tasks.push_back(std::move(lt));
      lo = hi;
      hi = nodes.size();
    }
    const int64_t n_nodes = (int64_t)nodes.size();
    if (n_nodes >= (int64_t)1 << 31) return MRDEM_ERR_INVALID;
    // ---- device work arrays
    std::vector<int32_t> h_tp(n_tri), h_perm(n_tri);
    for (int i = 0; i < n; ++i)
      for (int64_t t = tri_off[i]; t < tri_off[i + 1]; ++t) {
        h_tp[t] = i;
        h_perm[t] = (int32_t)t;
      }
    DevBuf<int64_t> d_voff, d_toff, d_nbeg;
    DevBuf<int32_t> d_tp, d_perm, d_tmp, d_err, d_ncnt, d_npart;
    DevBuf<double> d_cen;
    DevBuf<BisectTask> d_tasks;
    DevBuf<float> d_ntri, d_ndelta, d_nbox;
    size_t max_tasks = 1;
    for (auto& lt : tasks)
      for (auto& v : lt) max_tasks = std::max(max_tasks, v.size());
    if (!d_voff.alloc(n + 1) || !d_toff.alloc(n + 1) || !d_tp.alloc(n_tri) || !d_perm.alloc(n_tri) ||
        !d_tmp.alloc(n_tri) || !d_err.alloc(1) || !d_cen.alloc(3 * n_tri) ||
        !d_tasks.alloc(max_tasks) || !d_nbeg.alloc(n_nodes) || !d_ncnt.alloc(n_nodes) ||
        !d_npart.alloc(n_nodes) || !d_ntri.alloc(9 * n_nodes) || !d_ndelta.alloc(n_nodes) ||
        !d_nbox.alloc(16 * n_nodes)) {
      cudaGetLastError();
      return MRDEM_ERR_OOM;
    }
    cudaMemcpy(d_voff.p, vert_off, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(d_toff.p, tri_off, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(d_tp.p, h_tp.data(), sizeof(int32_t) * n_tri, cudaMemcpyHostToDevice);
    cudaMemcpy(d_perm.p, h_perm.data(), sizeof(int32_t) * n_tri, cudaMemcpyHostToDevice);
    cudaMemset(d_err.p, 0, sizeof(int32_t));
    int n_sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    k_centroids<<<n_sms * 8, 256>>>(n, d_voff.p, d_toff.p, d_verts, d_tris, n_tri, d_tp.p, d_cen.p,
                                    d_err.p);
    int32_t h_err = 0;
    if (cudaMemcpy(&h_err, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return MRDEM_ERR_CUDA;
    }
    if (h_err) return MRDEM_ERR_INVALID;
    // ---- clusters: bisections, level by level, depth by depth
    for (auto& lt : tasks)
      for (auto& v : lt) {
        if (v.empty()) continue;
        cudaMemcpy(d_tasks.p, v.data(), sizeof(BisectTask) * v.size(), cudaMemcpyHostToDevice);
        const int grid = (int)std::min<size_t>(v.size(), (size_t)n_sms * 64);
        k_bisect<<<grid, kBisectThreads>>>(d_tasks.p, (int)v.size(), d_perm.p, d_tmp.p, d_cen.p);
      }
    // ---- per node: surrogate, slack, box
    {
      std::vector<int64_t> nb(n_nodes);
      std::vector<int32_t> nc(n_nodes), np(n_nodes);
      for (int64_t q = 0; q < n_nodes; ++q) {
        nb[q] = nodes[q].begin;
        nc[q] = nodes[q].count;
        np[q] = nodes[q].particle;
      }
      cudaMemcpy(d_nbeg.p, nb.data(), sizeof(int64_t) * n_nodes, cudaMemcpyHostToDevice);
      cudaMemcpy(d_ncnt.p, nc.data(), sizeof(int32_t) * n_nodes, cudaMemcpyHostToDevice);
      cudaMemcpy(d_npart.p, np.data(), sizeof(int32_t) * n_nodes, cudaMemcpyHostToDevice);
    }
    FitArgs fa;
    fa.perm = d_perm.p;
    fa.node_begin = d_nbeg.p;
    fa.node_count = d_ncnt.p;
    fa.node_particle = d_npart.p;
    fa.verts = d_verts;
    fa.tris = d_tris;
    fa.vert_off = d_voff.p;
    fa.tri_off = d_toff.p;
    fa.node_tri = d_ntri.p;
    fa.node_delta = d_ndelta.p;
    fa.node_box = d_nbox.p;
    fa.error = d_err.p;
    fa.n_nodes = n_nodes;
    k_fit<<<(int)std::min<int64_t>(n_nodes, (int64_t)n_sms * 32), kFitThreads>>>(fa);
    if (cudaGetLastError() != cudaSuccess) return MRDEM_ERR_CUDA;
    // ---- the host record (as the host builder writes it)
    HierHost& h = *out;
    h = HierHost();
    h.n_particles = n;
    h.n_tri = n_tri;
    h.n_verts = n_verts;
    h.max_depth = max_depth;
    h.tri_off.assign(tri_off, tri_off + n + 1);
    h.vert_off.assign(vert_off, vert_off + n + 1);
    h.n_nodes = n_nodes;
    h.node_tri.resize(9 * n_nodes);
    h.node_delta.resize(n_nodes);
    h.node_box.resize(16 * n_nodes);
    std::vector<int32_t> perm(n_tri);
    if (cudaMemcpy(h.node_tri.data(), d_ntri.p, sizeof(float) * 9 * n_nodes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(h.node_delta.data(), d_ndelta.p, sizeof(float) * n_nodes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(h.node_box.data(), d_nbox.p, sizeof(float) * 16 * n_nodes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(perm.data(), d_perm.p, sizeof(int32_t) * n_tri, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&h_err, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return MRDEM_ERR_CUDA;
    }
    if (h_err) return MRDEM_ERR_INVALID;  // a degenerate surrogate
    cudaEventRecord(ev1);
    cudaEventSynchronize(ev1);
    if (ms) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev0, ev1);
      *ms = t;
    }
    // nodes, leaves' slot runs (each padded to a multiple of 4 slots) and
    // the per-slot records
    h.node_child.resize(2 * n_nodes);
    h.node_level.resize(n_nodes);
    h.root.resize(n);
    for (int i = 0; i < n; ++i) h.root[i] = i;
    int64_t slots = 0;
    for (int64_t q = 0; q < n_nodes; ++q)
      if (nodes[q].first_child < 0) slots += (nodes[q].count + 3) / 4 * 4;
    h.n_tri_pad = slots;
    if (slots >= (int64_t)1 << 31) return MRDEM_ERR_INVALID;
    h.slot_xyz.assign(9 * slots, 0.f);
    h.slot_vid.assign(3 * slots, -1);
    h.slot_tri.assign(slots, -1);
    h.slot_particle.assign(slots, -1);
    h.tri_slot.assign(n_tri, -1);
    std::vector<float> hv(3 * n_verts);
    std::vector<int32_t> ht(3 * n_tri);
    if (cudaMemcpy(hv.data(), d_verts, sizeof(float) * 3 * n_verts, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ht.data(), d_tris, sizeof(int32_t) * 3 * n_tri, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return MRDEM_ERR_CUDA;
    }
    int64_t slot = 0;
    for (int64_t q = 0; q < n_nodes; ++q) {
      const HNode& nd = nodes[q];
      h.node_level[q] = nd.level;
      if (nd.first_child >= 0) {
        h.node_child[2 * q] = nd.first_child;
        h.node_child[2 * q + 1] = nd.n_children;
        continue;
      }
      const int p = nd.particle;
      h.node_child[2 * q] = (int32_t)slot;
      h.node_child[2 * q + 1] = -nd.count;
      // a leaf's triangles in increasing index order, as the host builder
      std::vector<int32_t> leaf(perm.begin() + nd.begin, perm.begin() + nd.begin + nd.count);
      std::sort(leaf.begin(), leaf.end());
      for (int32_t g : leaf) {
        const int32_t t = (int32_t)(g - tri_off[p]);
        for (int k = 0; k < 3; ++k) {
          const int32_t v = ht[3 * g + k];
          h.slot_vid[3 * slot + k] = (int32_t)(vert_off[p] + v);
          for (int c = 0; c < 3; ++c) h.slot_xyz[9 * slot + 3 * k + c] = hv[3 * (vert_off[p] + v) + c];
        }
        h.slot_tri[slot] = t;
        h.slot_particle[slot] = p;
        h.tri_slot[g] = (int32_t)slot;
        ++slot;
      }
      slot = (slot + 3) / 4 * 4;
    }
    h.bound_r.resize(n);
    for (int i = 0; i < n; ++i) {
      double br = 0;
      for (int64_t v = vert_off[i]; v < vert_off[i + 1]; ++v)
        br = std::max(br, std::sqrt((double)hv[3 * v] * hv[3 * v] + (double)hv[3 * v + 1] * hv[3 * v + 1] +
                                    (double)hv[3 * v + 2] * hv[3 * v + 2]));
      float f = (float)br;
      if ((double)f < br) f = std::nextafter(f, FLT_MAX);
      h.bound_r[i] = f;
    }
  } catch (const std::bad_alloc&) {
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return MRDEM_ERR_OOM;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return MRDEM_OK;
}

}  // namespace mrdem
