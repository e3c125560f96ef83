// mrdem_detect.cu -- multiresolution contact detection on the GPU.
//
// Algorithm 5 of Noble & Weinzierl (arXiv 2105.12415) for a batch of particle
// pairs, level-synchronous, as a fixed sequence of kernels (capturable in one
// CUDA graph, no host synchronisation):
//   k_setup  one thread per pair: B->A relative transform (FP64, and its
//            float copy), then the root surrogate pair test;
//   k_level  one warp per surviving node pair: tests all child pairs (<= 8x8)
//            of the pair with the float penalty sweep + certificate against
//            delta_a + delta_b + 2 eps (conservative surrogates, Definition
//            "conservative"); survivors are compacted by warp ballot into the
//            next level's list, or into the leaf-pair list once both sides are
//            leaves (a side that is already a leaf stays while the other
//            unfolds, Algorithm 5);
//   k_tile   one warp per leaf pair, fetched dynamically: both leaves' fine
//            triangles staged in shared memory (B transformed into A's frame),
//            the la x lb products spread over the lanes, one fine pair per
//            lane: the float sweep of Eq. 3/4 (fixed iteration count,
//            Algorithm 4 top) and the certificate at 2 eps; survivors are the
//            candidates;
//   k_exact  one thread per candidate: the comparison-based distance of Sec. 3
//            (Algorithm 4 bottom), FP64, or float with FP64 for the final
//            value; contacts (d <= 2 eps) appended to the caller's buffers.
// The pruning only discards pairs whose certified lower bound exceeds the
// threshold, so the contact set equals the brute-force one (Lemma 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mrdem_geometry.cuh"
#include "mrdem_internal.h"

namespace mrdem {

using F3 = V3<float>;
using D3 = V3<double>;

// ---------------------------------------------------------------------------
// helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void quat_matrix(double w, double x, double y, double z, double R[9]) {
  double n = w * w + x * x + y * y + z * z;
  double s = 2.0 / n;
  double xx = s * x * x, yy = s * y * y, zz = s * z * z;
  double xy = s * x * y, xz = s * x * z, yz = s * y * z;
  double wx = s * w * x, wy = s * w * y, wz = s * w * z;
  R[0] = 1.0 - (yy + zz); R[1] = xy - wz;         R[2] = xz + wy;
  R[3] = xy + wz;         R[4] = 1.0 - (xx + zz); R[5] = yz - wx;
  R[6] = xz - wy;         R[7] = yz + wx;         R[8] = 1.0 - (xx + yy);
}

// Append `item` for each lane with `pred` to `list` (capacity cap); one
// atomic per warp.  Must be called by all 32 lanes.  Overflowing entries are
// dropped and the needed size is latched in *req.
__device__ __forceinline__ void warp_append(bool pred, int3 item, int3* list,
                                            unsigned long long* counter, int64_t cap,
                                            unsigned long long* req) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  if (!m) return;
  int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if ((int)lane_id() == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) {
    unsigned long long idx = base + __popc(m & ((1u << lane_id()) - 1u));
    if ((int64_t)idx < cap) list[idx] = item;
    else atomicMax(req, idx + 1);
  }
}

__device__ __forceinline__ F3 xf_point(const PairXf& X, F3 v) {
  return {fmaf(X.R[0], v.x, fmaf(X.R[1], v.y, fmaf(X.R[2], v.z, X.t[0]))),
          fmaf(X.R[3], v.x, fmaf(X.R[4], v.y, fmaf(X.R[5], v.z, X.t[1]))),
          fmaf(X.R[6], v.x, fmaf(X.R[7], v.y, fmaf(X.R[8], v.z, X.t[2])))};
}
__device__ __forceinline__ D3 xf_point64(const double* R, const double* t, D3 v) {
  return {R[0] * v.x + R[1] * v.y + R[2] * v.z + t[0], R[3] * v.x + R[4] * v.y + R[5] * v.z + t[1],
          R[6] * v.x + R[7] * v.y + R[8] * v.z + t[2]};
}

__device__ __forceinline__ void load_pairxf(const PairXf* xf, int p, PairXf& X) {
  const float4* s = reinterpret_cast<const float4*>(xf + p);
  float4 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2), d = __ldg(s + 3);
  X.R[0] = a.x; X.R[1] = a.y; X.R[2] = a.z; X.R[3] = a.w;
  X.R[4] = b.x; X.R[5] = b.y; X.R[6] = b.z; X.R[7] = b.w;
  X.R[8] = c.x; X.t[0] = c.y; X.t[1] = c.z; X.t[2] = c.w;
  X.tau = d.x; X.margin = d.y;
  X.A = __float_as_int(d.z); X.B = __float_as_int(d.w);
}

// Warp-aggregated statistics: lane 0 keeps the warp's running totals.
struct WarpCount {
  unsigned long long v = 0;
  __device__ __forceinline__ void add(bool pred) {
    unsigned m = __ballot_sync(0xffffffffu, pred);
    v += __popc(m);
  }
  __device__ __forceinline__ void flush(unsigned long long* dst) {
    if (lane_id() == 0 && v) atomicAdd(dst, v);
  }
};

// ---------------------------------------------------------------------------
// k_setup: per pair transforms + root test
__global__ void k_setup(HierDev H, int n_pairs, const int32_t* __restrict__ ab,
                        const double* __restrict__ eps, const double* __restrict__ poses,
                        PairXf* xf, PairXf64* xf64, SweepConst sc, int root_test, int3* list0,
                        int3* tiles, unsigned long long* cnt, unsigned long long* status,
                        int64_t cap_level, int64_t cap_tiles) {
  WarpCount tests, surv;
  int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n_pairs; base += stride) {
    int p = base + threadIdx.x;
    bool in = p < n_pairs;
    bool ok = false, survive = false, both_leaf = false;
    int ra = 0, rb = 0;
    if (in) {
      int A = ab[2 * p], B = ab[2 * p + 1];
      double e = eps[p];
      ok = A >= 0 && B >= 0 && A < H.n_particles && B < H.n_particles && isfinite(e) && e > 0.0;
      const double* pa = poses + 7 * (int64_t)(ok ? A : 0);
      const double* pb = poses + 7 * (int64_t)(ok ? B : 0);
      for (int k = 0; k < 7 && ok; ++k) ok = isfinite(pa[k]) && isfinite(pb[k]);
      ok = ok && (pa[3] * pa[3] + pa[4] * pa[4] + pa[5] * pa[5] + pa[6] * pa[6]) > 0.0 &&
           (pb[3] * pb[3] + pb[4] * pb[4] + pb[5] * pb[5] + pb[6] * pb[6]) > 0.0;
      PairXf64 X64;
      PairXf X;
      if (ok) {
        double RA[9], RB[9];
        quat_matrix(pa[3], pa[4], pa[5], pa[6], RA);
        quat_matrix(pb[3], pb[4], pb[5], pb[6], RB);
        double dt[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        double tn = 0;
        for (int r = 0; r < 3; ++r) {
          for (int c = 0; c < 3; ++c)
            X64.R[3 * r + c] = RA[r] * RB[c] + RA[3 + r] * RB[3 + c] + RA[6 + r] * RB[6 + c];
          X64.t[r] = RA[r] * dt[0] + RA[3 + r] * dt[1] + RA[6 + r] * dt[2];
          tn += X64.t[r] * X64.t[r];
        }
        for (int k = 0; k < 9; ++k) { X64.RA[k] = RA[k]; X.R[k] = (float)X64.R[k]; }
        for (int k = 0; k < 3; ++k) { X64.tA[k] = pa[k]; X.t[k] = (float)X64.t[k]; }
        X64.eps = e;
        X64.A = A; X64.B = B; X64.valid = 1; X64.pad = 0;
        X.tau = (float)(2.0 * e);
        // bound of the float rounding in the transformed coordinates, the
        // support dot products and |u| != 1 (about 2^-20 relative each)
        X.margin = (float)(ldexp(1.0, -16) * (H.bound_r[A] + H.bound_r[B] + sqrt(tn) + 2.0 * e));
        X.A = A; X.B = B;
        ra = H.root[A];
        rb = H.root[B];
        if (root_test) {
          float4 a0 = H.node_geo[3 * ra], a1 = H.node_geo[3 * ra + 1], a2 = H.node_geo[3 * ra + 2];
          float4 b0 = H.node_geo[3 * rb], b1 = H.node_geo[3 * rb + 1], b2 = H.node_geo[3 * rb + 2];
          F3 q0 = xf_point(X, {b0.x, b0.y, b0.z}), q1 = xf_point(X, {b1.x, b1.y, b1.z});
          F3 q2 = xf_point(X, {b2.x, b2.y, b2.z});
          bool cv;
          float gap = sweep_certificate<false>({a0.x, a0.y, a0.z}, {a1.x, a1.y, a1.z},
                                               {a2.x, a2.y, a2.z}, q0, q1, q2, sc, 0.f, &cv, nullptr);
          float thr = a0.w + b0.w + X.tau + X.margin;
          survive = !(gap > thr);
          both_leaf = H.node_child[ra].y < 0 && H.node_child[rb].y < 0;
        }
      } else {
        X64.valid = 0;
        for (int k = 0; k < 9; ++k) X.R[k] = 0.f;
        X.t[0] = X.t[1] = X.t[2] = 0.f;
        X.tau = 0.f; X.margin = 0.f; X.A = X.B = 0;
        atomicExch(status + ST_NONFINITE, 1ull);
      }
      xf[p] = X;
      xf64[p] = X64;
    }
    if (root_test) {
      tests.add(in && ok);
      surv.add(survive);
      warp_append(survive && both_leaf, make_int3(p, ra, rb), tiles, cnt + CNT_TILES, cap_tiles,
                  status + ST_REQ_TILES);
      warp_append(survive && !both_leaf, make_int3(p, ra, rb), list0, cnt + CNT_LEVEL, cap_level,
                  status + ST_REQ_LEVEL);
    }
  }
  tests.flush(cnt + CNT_STATS + MRDEM_STAT_TESTS);
  surv.flush(cnt + CNT_STATS + MRDEM_STAT_SURVIVORS);
}

// ---------------------------------------------------------------------------
// k_level: one warp per node pair of list `level`; tests its child pairs.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_level(HierDev H, const PairXf* __restrict__ xf,
                                                      SweepConst sc, const int3* __restrict__ in,
                                                      int level, int3* out, int3* tiles,
                                                      unsigned long long* cnt,
                                                      unsigned long long* status,
                                                      int64_t cap_level, int64_t cap_tiles) {
  __shared__ float4 sgeo[WARPS][16][3];
  __shared__ int sleaf[WARPS][16];
  __shared__ int snode[WARPS][16];
  const int w = threadIdx.x >> 5, lane = lane_id();
  int64_t n_in = (int64_t)cnt[CNT_LEVEL + level];
  if (n_in > cap_level) n_in = cap_level;
  const int slot_tests = MRDEM_STAT_TESTS + (level + 1 < MRDEM_STAT_LEVELS ? level + 1 : MRDEM_STAT_LEVELS - 1);
  WarpCount tests, surv;
  for (int64_t item = (int64_t)blockIdx.x * WARPS + w; item < n_in; item += (int64_t)gridDim.x * WARPS) {
    int3 it = in[item];
    PairXf X;
    load_pairxf(xf, it.x, X);
    int2 ca = H.node_child[it.y], cb = H.node_child[it.z];
    int na = ca.y > 0 ? ca.y : 1, abeg = ca.y > 0 ? ca.x : it.y;
    int nb = cb.y > 0 ? cb.y : 1, bbeg = cb.y > 0 ? cb.x : it.z;
    if (lane < na) {
      int node = abeg + lane;
      sgeo[w][lane][0] = H.node_geo[3 * node];
      sgeo[w][lane][1] = H.node_geo[3 * node + 1];
      sgeo[w][lane][2] = H.node_geo[3 * node + 2];
      sleaf[w][lane] = H.node_child[node].y < 0;
      snode[w][lane] = node;
    } else if (lane >= 8 && lane < 8 + nb) {
      int node = bbeg + lane - 8;
      float4 g0 = H.node_geo[3 * node], g1 = H.node_geo[3 * node + 1], g2 = H.node_geo[3 * node + 2];
      F3 q0 = xf_point(X, {g0.x, g0.y, g0.z}), q1 = xf_point(X, {g1.x, g1.y, g1.z});
      F3 q2 = xf_point(X, {g2.x, g2.y, g2.z});
      sgeo[w][lane][0] = make_float4(q0.x, q0.y, q0.z, g0.w);
      sgeo[w][lane][1] = make_float4(q1.x, q1.y, q1.z, 0.f);
      sgeo[w][lane][2] = make_float4(q2.x, q2.y, q2.z, 0.f);
      sleaf[w][lane] = H.node_child[node].y < 0;
      snode[w][lane] = node;
    }
    __syncwarp();
    int total = na * nb;
    for (int f0 = 0; f0 < total; f0 += 32) {
      int f = f0 + lane;
      bool act = f < total;
      int i = act ? f / nb : 0, j = act ? f - (f / nb) * nb : 0;
      bool s = false;
      if (act) {
        float4 a0 = sgeo[w][i][0], a1 = sgeo[w][i][1], a2 = sgeo[w][i][2];
        float4 b0 = sgeo[w][8 + j][0], b1 = sgeo[w][8 + j][1], b2 = sgeo[w][8 + j][2];
        bool cv;
        float gap = sweep_certificate<false>({a0.x, a0.y, a0.z}, {a1.x, a1.y, a1.z}, {a2.x, a2.y, a2.z},
                                             {b0.x, b0.y, b0.z}, {b1.x, b1.y, b1.z}, {b2.x, b2.y, b2.z},
                                             sc, 0.f, &cv, nullptr);
        s = !(gap > a0.w + b0.w + X.tau + X.margin);
      }
      bool leaves = act && sleaf[w][i] && sleaf[w][8 + j];
      int3 child = make_int3(it.x, act ? snode[w][i] : 0, act ? snode[w][8 + j] : 0);
      tests.add(act);
      surv.add(s);
      warp_append(s && leaves, child, tiles, cnt + CNT_TILES, cap_tiles, status + ST_REQ_TILES);
      warp_append(s && !leaves, child, out, cnt + CNT_LEVEL + level + 1, cap_level,
                  status + ST_REQ_LEVEL);
    }
    __syncwarp();
  }
  tests.flush(cnt + CNT_STATS + slot_tests);
  surv.flush(cnt + CNT_STATS + slot_tests + MRDEM_STAT_SURVIVORS);
}

// ---------------------------------------------------------------------------
// k_tile: one warp per leaf pair (dynamic fetch).  Both leaves' fine
// triangles are staged in shared memory (B moved into A's frame) together
// with a bounding sphere each (centroid, largest vertex distance).  Pass 1
// spreads the la x lb products over the lanes and keeps the pairs whose
// spheres come within the threshold (|c_a - c_b| - r_a - r_b bounds the
// distance from below); the survivors are compacted into a per-warp queue
// (the buffered comparisons of Sec. 5.4).  Pass 2 runs the penalty sweep and
// certificate over the queue, one fine pair per lane.
constexpr int kTileQueue = 1024;  // 32 x 32 products
struct TileSmem {
  float4 a[3][32];  // A: v0, v1, v2 (xyz), w = centroid x / y / z
  float4 b[3][32];
  float ra[32], rb[32];
  unsigned short q[kTileQueue];
};

__device__ __forceinline__ void stage_triangle(F3 v0, F3 v1, F3 v2, float4 (*dst)[32], float* rad,
                                               int lane) {
  F3 c = (1.f / 3.f) * ((v0 + v1) + v2);
  F3 d0 = v0 - c, d1 = v1 - c, d2 = v2 - c;
  float r2 = fmaxf(dot(d0, d0), fmaxf(dot(d1, d1), dot(d2, d2)));
  dst[0][lane] = make_float4(v0.x, v0.y, v0.z, c.x);
  dst[1][lane] = make_float4(v1.x, v1.y, v1.z, c.y);
  dst[2][lane] = make_float4(v2.x, v2.y, v2.z, c.z);
  rad[lane] = sqrtf(r2) * (1.f + 1e-6f);
}

template <bool CONV>
__global__ void __launch_bounds__(256) k_tile(HierDev H, const PairXf* __restrict__ xf,
                                              SweepConst sc, float conv_c,
                                              const int3* __restrict__ tiles, int3* cands,
                                              unsigned long long* cnt, unsigned long long* status,
                                              int64_t cap_tiles, int64_t cap_cands,
                                              const double* __restrict__ eps_d) {
  extern __shared__ float4 smem4[];
  const int w = threadIdx.x >> 5, lane = lane_id();
  TileSmem& S = reinterpret_cast<TileSmem*>(smem4)[w];
  int64_t n_tiles = (int64_t)cnt[CNT_TILES];
  if (n_tiles > cap_tiles) n_tiles = cap_tiles;
  WarpCount tests, spheres, ncand, nodot;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(cnt + CNT_FETCH + kMaxLevels, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if ((int64_t)t >= n_tiles) break;
    int3 it = tiles[t];
    PairXf X;
    load_pairxf(xf, it.x, X);
    float ce = conv_c * (float)__ldg(eps_d + it.x);
    float conv_tol2 = ce * ce;
    int2 ca = H.node_child[it.y], cb = H.node_child[it.z];
    int na = -ca.y, nb = -cb.y;
    if (lane < na) {
      F3 v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[c].x = __ldg(H.tri + (3 * c + 0) * H.stride + ca.x + lane);
        v[c].y = __ldg(H.tri + (3 * c + 1) * H.stride + ca.x + lane);
        v[c].z = __ldg(H.tri + (3 * c + 2) * H.stride + ca.x + lane);
      }
      stage_triangle(v[0], v[1], v[2], S.a, S.ra, lane);
    }
    if (lane < nb) {
      F3 v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        F3 u;
        u.x = __ldg(H.tri + (3 * c + 0) * H.stride + cb.x + lane);
        u.y = __ldg(H.tri + (3 * c + 1) * H.stride + cb.x + lane);
        u.z = __ldg(H.tri + (3 * c + 2) * H.stride + cb.x + lane);
        v[c] = xf_point(X, u);
      }
      stage_triangle(v[0], v[1], v[2], S.b, S.rb, lane);
    }
    __syncwarp();
    const float thr = X.tau + X.margin;
    const int total = na * nb;
    const float inv_nb = 1.0f / (float)nb;
    // pass 1: bounding-sphere cull, survivors compacted into the queue
    int nq = 0;
    for (int f0 = 0; f0 < total; f0 += 32) {
      int f = f0 + lane;
      bool act = f < total;
      int i = (int)(((float)f + 0.5f) * inv_nb);
      int j = f - i * nb;
      if (!act) { i = 0; j = 0; }
      float dx = S.a[0][i].w - S.b[0][j].w, dy = S.a[1][i].w - S.b[1][j].w;
      float dz = S.a[2][i].w - S.b[2][j].w;
      float lim = S.ra[i] + S.rb[j] + thr;
      bool keep = act && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= lim * lim;
      unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) S.q[nq + __popc(m & ((1u << lane) - 1u))] = (unsigned short)((i << 5) | j);
      nq += __popc(m);
    }
    spheres.v += lane == 0 ? (unsigned long long)total : 0ull;
    __syncwarp();
    // pass 2: penalty sweep + certificate on the queued pairs
    for (int q0 = 0; q0 < nq; q0 += 32) {
      int k = q0 + lane;
      bool act = k < nq;
      int code = act ? S.q[k] : 0;
      int i = code >> 5, j = code & 31;
      float4 a0 = S.a[0][i], a1 = S.a[1][i], a2 = S.a[2][i];
      float4 b0 = S.b[0][j], b1 = S.b[1][j], b2 = S.b[2][j];
      bool cv = true;
      float gap;
      if (sc.n_iter == 4)
        gap = sweep_certificate<CONV, 4>({a0.x, a0.y, a0.z}, {a1.x, a1.y, a1.z}, {a2.x, a2.y, a2.z},
                                         {b0.x, b0.y, b0.z}, {b1.x, b1.y, b1.z}, {b2.x, b2.y, b2.z},
                                         sc, conv_tol2, &cv, nullptr);
      else
        gap = sweep_certificate<CONV, 0>({a0.x, a0.y, a0.z}, {a1.x, a1.y, a1.z}, {a2.x, a2.y, a2.z},
                                         {b0.x, b0.y, b0.z}, {b1.x, b1.y, b1.z}, {b2.x, b2.y, b2.z},
                                         sc, conv_tol2, &cv, nullptr);
      bool s = act && !(gap > thr);
      tests.add(act);
      ncand.add(s);
      if (CONV) nodot.add(s && !cv);
      warp_append(s, make_int3(it.x, ca.x + i, cb.x + j), cands, cnt + CNT_CANDS, cap_cands,
                  status + ST_REQ_CANDS);
    }
    __syncwarp();
  }
  tests.flush(cnt + CNT_STATS + MRDEM_STAT_FINE_TESTS);
  spheres.flush(cnt + CNT_STATS + MRDEM_STAT_SPHERE_TESTS);
  ncand.flush(cnt + CNT_STATS + MRDEM_STAT_CANDIDATES);
  if (CONV) nodot.flush(cnt + CNT_STATS + MRDEM_STAT_UNCONVERGED);
}

// ---------------------------------------------------------------------------
// Final distance of one candidate.  P, Q: FP64 coordinates relative to the
// origin o (A's frame).  FP64: comparison-based in double.  FP32: the same in
// float on the rounded local coordinates; the pair is decided in float when
// its distance is clear of 2 eps by more than the float error bound, and the
// winning feature's distance is then re-evaluated in double; pairs near the
// threshold, near ties between features and near-parallel edge minima go to
// the full double evaluation.
struct CandResult {
  double d;
  D3 pa, pb;
  int feature;
  bool fp64_full;
};

__device__ __forceinline__ void eval_feature64(const D3 P[3], const D3 Q[3], int f, CandResult& r,
                                               bool& ok) {
  double w[3];
  ok = true;
  if (f < 3) {
    D3 q = closest_on_triangle(P[f], Q[0], Q[1], Q[2], w);
    r.pa = P[f]; r.pb = q;
  } else if (f < 6) {
    D3 p = closest_on_triangle(Q[f - 3], P[0], P[1], P[2], w);
    r.pa = p; r.pb = Q[f - 3];
  } else if (f < 15) {
    int i = (f - 6) / 3, j = (f - 6) % 3;
    int i1 = i == 2 ? 0 : i + 1, j1 = j == 2 ? 0 : j + 1;
    double s, t;
    bool par;
    closest_segments(P[i], P[i1], Q[j], Q[j1], &s, &t, &par);
    r.pa = P[i] + s * (P[i1] - P[i]);
    r.pb = Q[j] + t * (Q[j1] - Q[j]);
  } else {
    ok = false;  // crossings are re-tested in full
    return;
  }
  D3 dv = r.pa - r.pb;
  r.d = sqrt(dot(dv, dv));
  r.feature = f;
}

template <int PREC>
__device__ __forceinline__ bool candidate_distance(const D3 P[3], const D3 Q[3], double tau,
                                                   CandResult& r) {
  r.fp64_full = false;
  if (PREC == MRDEM_PREC_FP32) {
    F3 Pf[3], Qf[3];
    float L = 0.f;
    for (int k = 0; k < 3; ++k) {
      Pf[k] = {(float)P[k].x, (float)P[k].y, (float)P[k].z};
      Qf[k] = {(float)Q[k].x, (float)Q[k].y, (float)Q[k].z};
      L = fmaxf(L, fmaxf(fmaxf(fabsf(Pf[k].x), fabsf(Pf[k].y)), fabsf(Pf[k].z)));
      L = fmaxf(L, fmaxf(fmaxf(fabsf(Qf[k].x), fabsf(Qf[k].y)), fabsf(Qf[k].z)));
    }
    float second2;
    TriTriResult<float> rf = tri_tri_distance_ranked(Pf, Qf, &second2);
    double err = ldexp((double)L, -15);
    double d32 = rf.d;
    if (d32 > tau + err) return false;  // certainly no contact
    bool full = rf.near_parallel || fabs(d32 - tau) <= err || rf.feature >= 100 ||
                (double)sqrtf(second2) - d32 <= 2.0 * err;
    if (!full) {
      bool ok;
      eval_feature64(P, Q, rf.feature, r, ok);
      if (ok) return r.d <= tau;
    }
    r.fp64_full = true;
  }
  TriTriResult<double> rd = tri_tri_distance(P, Q);
  r.d = rd.d;
  r.pa = rd.pa;
  r.pb = rd.pb;
  r.feature = rd.feature;
  return r.d <= tau;
}

__device__ __forceinline__ void load_tri64(const HierDev& H, int slot, D3 T[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T[c].x = (double)__ldg(H.tri + (3 * c + 0) * H.stride + slot);
    T[c].y = (double)__ldg(H.tri + (3 * c + 1) * H.stride + slot);
    T[c].z = (double)__ldg(H.tri + (3 * c + 2) * H.stride + slot);
  }
}

template <int PREC>
__global__ void __launch_bounds__(128) k_exact(HierDev H, const PairXf64* __restrict__ xf64,
                                               const int3* __restrict__ cands,
                                               unsigned long long* cnt, unsigned long long* status,
                                               int64_t cap_cands, mrdem_contacts out) {
  int64_t n = (int64_t)cnt[CNT_CANDS];
  if (n > cap_cands) n = cap_cands;
  WarpCount ncon, n64;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    bool is_contact = false, full = false;
    CandResult r;
    int3 c = make_int3(0, 0, 0);
    if (k < n) {
      c = cands[k];
      const PairXf64& X = xf64[c.x];
      D3 Pb[3], Qb[3], P[3], Q[3];
      load_tri64(H, c.y, Pb);
      load_tri64(H, c.z, Qb);
      D3 o = Pb[0];
      for (int v = 0; v < 3; ++v) {
        P[v] = Pb[v] - o;
        Q[v] = xf_point64(X.R, X.t, Qb[v]) - o;
      }
      is_contact = candidate_distance<PREC>(P, Q, 2.0 * X.eps, r);
      full = r.fp64_full;
      if (is_contact) {
        r.pa = xf_point64(X.RA, X.tA, r.pa + o);
        r.pb = xf_point64(X.RA, X.tA, r.pb + o);
      }
    }
    ncon.add(is_contact);
    if (PREC == MRDEM_PREC_FP32) n64.add(full);
    unsigned m = __ballot_sync(0xffffffffu, is_contact);
    if (m) {
      int leader = __ffs(m) - 1;
      unsigned long long b = 0;
      if ((int)lane_id() == leader) b = atomicAdd((unsigned long long*)out.count, (unsigned long long)__popc(m));
      b = __shfl_sync(0xffffffffu, b, leader);
      if (is_contact) {
        unsigned long long idx = b + __popc(m & ((1u << lane_id()) - 1u));
        if ((int64_t)idx < out.capacity) {
          out.pair[idx] = c.x;
          out.tri_a[idx] = H.slot_tri[c.y];
          out.tri_b[idx] = H.slot_tri[c.z];
          out.dist[idx] = r.d;
          out.point_a[3 * idx] = r.pa.x; out.point_a[3 * idx + 1] = r.pa.y; out.point_a[3 * idx + 2] = r.pa.z;
          out.point_b[3 * idx] = r.pb.x; out.point_b[3 * idx + 1] = r.pb.y; out.point_b[3 * idx + 2] = r.pb.z;
        } else {
          atomicMax(status + ST_REQ_CONTACTS, idx + 1);
        }
      }
    }
  }
  ncon.flush(cnt + CNT_STATS + MRDEM_STAT_CONTACTS);
  if (PREC == MRDEM_PREC_FP32) n64.flush(cnt + CNT_STATS + MRDEM_STAT_FP64);
}

// ---------------------------------------------------------------------------
// Plain form: every fine triangle pair of one particle pair, FP64.
__global__ void __launch_bounds__(256) k_plain(HierDev H, const PairXf64* __restrict__ xf64, int p,
                                               int64_t na, int64_t nb, unsigned long long* status,
                                               mrdem_contacts out) {
  const PairXf64 X = xf64[p];
  if (!X.valid) return;
  int64_t total = na * nb;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double tau = 2.0 * X.eps;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    int64_t k = base + threadIdx.x;
    bool hit = false;
    TriTriResult<double> r;
    int ta = 0, tb = 0;
    if (k < total) {
      ta = (int)(k / nb);
      tb = (int)(k - (int64_t)ta * nb);
      int sa = H.tri_slot[H.tri_off[X.A] + ta], sb = H.tri_slot[H.tri_off[X.B] + tb];
      D3 P[3], Q[3], Qb[3];
      load_tri64(H, sa, P);
      load_tri64(H, sb, Qb);
      for (int v = 0; v < 3; ++v) Q[v] = xf_point64(X.R, X.t, Qb[v]);
      r = tri_tri_distance(P, Q);
      hit = r.d <= tau;
      if (hit) {
        r.pa = xf_point64(X.RA, X.tA, r.pa);
        r.pb = xf_point64(X.RA, X.tA, r.pb);
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (m) {
      int leader = __ffs(m) - 1;
      unsigned long long b = 0;
      if ((int)lane_id() == leader) b = atomicAdd((unsigned long long*)out.count, (unsigned long long)__popc(m));
      b = __shfl_sync(0xffffffffu, b, leader);
      if (hit) {
        unsigned long long idx = b + __popc(m & ((1u << lane_id()) - 1u));
        if ((int64_t)idx < out.capacity) {
          out.pair[idx] = p;
          out.tri_a[idx] = ta;
          out.tri_b[idx] = tb;
          out.dist[idx] = r.d;
          out.point_a[3 * idx] = r.pa.x; out.point_a[3 * idx + 1] = r.pa.y; out.point_a[3 * idx + 2] = r.pa.z;
          out.point_b[3 * idx] = r.pb.x; out.point_b[3 * idx + 1] = r.pb.y; out.point_b[3 * idx + 2] = r.pb.z;
        } else {
          atomicMax(status + ST_REQ_CONTACTS, idx + 1);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Explicit triangle pairs (the triangle-pair kernels on their own).
template <int PREC>
__global__ void k_tridist(int64_t n, const double* __restrict__ Pin, const double* __restrict__ Qin,
                          const double* __restrict__ eps, SweepConst sc, float conv_c, double* dist,
                          double* pa, double* pb, int32_t* feature, float* sx, float* sgap,
                          int32_t* sconv) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    D3 P[3], Q[3];
    for (int v = 0; v < 3; ++v) {
      P[v] = {Pin[9 * k + 3 * v], Pin[9 * k + 3 * v + 1], Pin[9 * k + 3 * v + 2]};
      Q[v] = {Qin[9 * k + 3 * v], Qin[9 * k + 3 * v + 1], Qin[9 * k + 3 * v + 2]};
    }
    D3 o = P[0];
    for (int v = 0; v < 3; ++v) { P[v] = P[v] - o; Q[v] = Q[v] - o; }
    double e = eps[k];
    if (sx || sgap || sconv) {
      F3 Pf[3], Qf[3];
      for (int v = 0; v < 3; ++v) {
        Pf[v] = {(float)P[v].x, (float)P[v].y, (float)P[v].z};
        Qf[v] = {(float)Q[v].x, (float)Q[v].y, (float)Q[v].z};
      }
      float ce = conv_c * (float)e;
      bool cv;
      float x[4];
      float g = sweep_certificate<true>(Pf[0], Pf[1], Pf[2], Qf[0], Qf[1], Qf[2], sc, ce * ce, &cv, x);
      if (sx) for (int q = 0; q < 4; ++q) sx[4 * k + q] = x[q];
      if (sgap) sgap[k] = g;
      if (sconv) sconv[k] = cv;
    }
    if (dist || pa || pb || feature) {
      CandResult r;
      // decide with threshold 2 eps like the pipeline; when the float path
      // rejects a pair (clearly beyond 2 eps) report its full FP64 distance
      bool hit = candidate_distance<PREC>(P, Q, 2.0 * e, r);
      if (!hit && PREC == MRDEM_PREC_FP32 && !r.fp64_full) {
        TriTriResult<double> rd = tri_tri_distance(P, Q);
        r.d = rd.d; r.pa = rd.pa; r.pb = rd.pb; r.feature = rd.feature;
      }
      if (dist) dist[k] = r.d;
      D3 a = r.pa + o, b = r.pb + o;
      if (pa) { pa[3 * k] = a.x; pa[3 * k + 1] = a.y; pa[3 * k + 2] = a.z; }
      if (pb) { pb[3 * k] = b.x; pb[3 * k + 1] = b.y; pb[3 * k + 2] = b.z; }
      if (feature) feature[k] = r.feature;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
static int ensure_pairs(mrdem_ctx* c, int64_t n) {
  if (n <= c->cap_pairs) return MRDEM_OK;
  int64_t cap = c->cap_pairs ? c->cap_pairs : 1024;
  while (cap < n) cap *= 2;
  cudaFree(c->xf);
  cudaFree(c->xf64);
  c->xf = nullptr;
  c->xf64 = nullptr;
  c->cap_pairs = 0;
  if (cudaMalloc(&c->xf, sizeof(PairXf) * cap) != cudaSuccess ||
      cudaMalloc(&c->xf64, sizeof(PairXf64) * cap) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->xf);
    c->xf = nullptr;
    return MRDEM_ERR_OOM;
  }
  c->cap_pairs = cap;
  return MRDEM_OK;
}

static SweepConst sweep_const(const mrdem_params& p) {
  SweepConst sc;
  sc.rho_reg = p.rho_reg;
  sc.rho_iter = p.rho_iter;
  sc.n_iter = p.n_iter;
  return sc;
}

static int finish(cudaStream_t) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_detect(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                  const double* eps, const double* poses, int precision, const mrdem_contacts* out,
                  int64_t* stats, cudaStream_t s) {
  int st = ensure_pairs(c, n_pairs);
  if (st) return st;
  const HierDev& H = hier->dev;
  const mrdem_params& prm = c->params;
  SweepConst sc = sweep_const(prm);
  cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * CNT_TOTAL, s);
  cudaMemsetAsync(out->count, 0, sizeof(int64_t), s);
  if (n_pairs > 0) {
    int threads = 256;
    int blocks = (int)std::min<int64_t>((n_pairs + threads - 1) / threads, (int64_t)c->n_sms * 8);
    {
      ProfScope ps(c, K_SETUP, s);
      k_setup<<<blocks, threads, 0, s>>>(H, (int)n_pairs, ab, eps, poses, c->xf, c->xf64, sc, 1,
                                         c->level_list[0], c->tiles, c->counters, c->status,
                                         c->cap_level, c->cap_tiles);
    }
    int steps = std::min(hier->h.max_depth - 1, kMaxLevels - 1);
    for (int l = 0; l < steps; ++l) {
      constexpr int W = 8;
      ProfScope ps(c, K_LEVEL, s);
      k_level<W><<<c->n_sms * 8, W * 32, 0, s>>>(H, c->xf, sc, c->level_list[l & 1], l,
                                                  c->level_list[(l + 1) & 1], c->tiles,
                                                  c->counters, c->status, c->cap_level,
                                                  c->cap_tiles);
    }
    int tw = prm.tile_warps;
    size_t smem = (size_t)tw * sizeof(TileSmem);
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(k_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * (int)sizeof(TileSmem));
      attr_set = true;
    }
    {
    ProfScope ps(c, K_TILE, s);
    k_tile<true><<<c->n_sms * prm.tile_blocks_per_sm, tw * 32, smem, s>>>(
        H, c->xf, sc, prm.conv_c, c->tiles, c->cands, c->counters, c->status, c->cap_tiles,
        c->cap_cands, eps);
    }
    int et = prm.exact_threads;
    ProfScope ps(c, K_EXACT, s);
    if (precision == MRDEM_PREC_FP64)
      k_exact<MRDEM_PREC_FP64><<<c->n_sms * 8, et, 0, s>>>(H, c->xf64, c->cands, c->counters,
                                                             c->status, c->cap_cands, *out);
    else
      k_exact<MRDEM_PREC_FP32><<<c->n_sms * 8, et, 0, s>>>(H, c->xf64, c->cands, c->counters,
                                                             c->status, c->cap_cands, *out);
  }
  if (stats)
    cudaMemcpyAsync(stats, c->counters + CNT_STATS, sizeof(int64_t) * MRDEM_STAT_COUNT,
                    cudaMemcpyDeviceToDevice, s);
  return finish(s);
}

int launch_plain(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                 const double* eps, const double* poses, const mrdem_contacts* out,
                 cudaStream_t s) {
  int st = ensure_pairs(c, n_pairs);
  if (st) return st;
  const HierDev& H = hier->dev;
  SweepConst sc = sweep_const(c->params);
  cudaMemsetAsync(out->count, 0, sizeof(int64_t), s);
  if (n_pairs == 0) return finish(s);
  int threads = 256;
  int blocks = (int)((n_pairs + threads - 1) / threads);
  k_setup<<<blocks, threads, 0, s>>>(H, (int)n_pairs, ab, eps, poses, c->xf, c->xf64, sc, 0,
                                     nullptr, nullptr, c->counters, c->status, 0, 0);
  std::vector<int32_t> hab(2 * n_pairs);
  if (cudaMemcpyAsync(hab.data(), ab, sizeof(int32_t) * 2 * n_pairs, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  const auto& to = hier->h.tri_off;
  for (int64_t p = 0; p < n_pairs; ++p) {
    int A = hab[2 * p], B = hab[2 * p + 1];
    if (A < 0 || B < 0 || A >= hier->h.n_particles || B >= hier->h.n_particles) continue;
    int64_t na = to[A + 1] - to[A], nb = to[B + 1] - to[B];
    int64_t total = na * nb;
    int64_t blocks2 = std::min<int64_t>((total + threads - 1) / threads, (int64_t)c->n_sms * 64);
    ProfScope ps(c, K_PLAIN, s);
    k_plain<<<(int)blocks2, threads, 0, s>>>(H, c->xf64, (int)p, na, nb, c->status, *out);
  }
  return finish(s);
}

int launch_triangle_distance(mrdem_ctx* c, int64_t n, const double* P, const double* Q,
                             const double* eps, int precision, double* dist, double* pa,
                             double* pb, int32_t* feature, float* sx, float* sgap, int32_t* sconv,
                             cudaStream_t s) {
  if (n == 0) return MRDEM_OK;
  SweepConst sc = sweep_const(c->params);
  int threads = 128;
  int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)c->n_sms * 16);
  ProfScope ps(c, K_TRIDIST, s);
  if (precision == MRDEM_PREC_FP64)
    k_tridist<MRDEM_PREC_FP64><<<blocks, threads, 0, s>>>(n, P, Q, eps, sc, c->params.conv_c, dist,
                                                           pa, pb, feature, sx, sgap, sconv);
  else
    k_tridist<MRDEM_PREC_FP32><<<blocks, threads, 0, s>>>(n, P, Q, eps, sc, c->params.conv_c, dist,
                                                           pa, pb, feature, sx, sgap, sconv);
  return finish(s);
}

}  // namespace mrdem
