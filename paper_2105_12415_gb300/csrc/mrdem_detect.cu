// mrdem_detect.cu -- multiresolution contact detection on the GPU.
//
// Algorithm 5 of Noble & Weinzierl (arXiv 2105.12415) for a batch of particle
// pairs, level-synchronous, as a fixed sequence of kernels (capturable in one
// CUDA graph, no host synchronisation):
//   k_setup        one thread per pair: B->A relative transform (FP64, and its
//                  float copy), then the root surrogate pair test;
//   k_expand       per surrogate level: child pairs of the surviving node
//                  pairs, bounding-sphere cull, survivors to the sweep list;
//   k_sweep_nodes  per surrogate level: penalty sweep + certificate against
//                  delta_a + delta_b + 2 eps (conservative surrogates, Sec. 4);
//                  survivors become the next level's items, or leaf-pair
//                  tiles once both sides are leaves (a side that is already a
//                  leaf stays while the other unfolds, Algorithm 5);
//   k_tile         one warp per leaf pair: fine triangles against the other
//                  leaf's surrogate, then sphere products; survivors to the
//                  fine list;
//   k_sweep_fine   one thread per fine pair: separation along the face
//                  normals, then the float sweep of Eq. 3/4 (fixed iteration
//                  count, Algorithm 4) and the certificate at 2 eps; survivors
//                  are the candidates;
//   exact          the comparison-based distance of Sec. 3 (Algorithm 4's
//                  fallback) per candidate: FP64 (k_exact64), or float with
//                  FP64 work items for the final value (mrdem_closest.cu);
//                  contacts (d <= 2 eps) appended to the caller's buffers.
// The pruning only discards pairs whose certified lower bound exceeds the
// threshold, so the contact set equals the brute-force one (Lemma 1).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "mrdem_device.cuh"

namespace mrdem {

namespace cg = cooperative_groups;
using F3 = V3<float>;
using D3 = V3<double>;

// Level item for the children of the node pair (node_a with child info ia,
// node_b with ib); a leaf side is its own one-element set.
__device__ __forceinline__ int4 make_level(int pair, int node_a, int node_b, int2 ia, int2 ib) {
  int ab = ia.y > 0 ? ia.x : node_a, na = ia.y > 0 ? ia.y : 1;
  int bb = ib.y > 0 ? ib.x : node_b, nb = ib.y > 0 ? ib.y : 1;
  return make_int4(pair, ab, bb, na | (nb << 8));
}

// ---------------------------------------------------------------------------
// k_setup: per pair transforms + root test
__global__ void k_setup(HierDev H, int n_pairs, const int32_t* __restrict__ ab,
                        const double* __restrict__ eps, const double* __restrict__ poses,
                        PairXf* xf, PairXf64* xf64, PairXfDD* xfdd, SweepConst sc,
                        int root_test, int4* list0,
                        TileItem* tiles, unsigned long long* cnt, unsigned long long* status,
                        int64_t cap_level, int64_t cap_tiles) {
  wait_prior_grid();
  WarpCount tests, surv;
  int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n_pairs; base += stride) {
    int p = base + threadIdx.x;
    bool in = p < n_pairs;
    bool ok = false, survive = false, both_leaf = false;
    int ra = 0, rb = 0;
    int2 ia = make_int2(0, 1), ib = make_int2(0, 1);
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
          ia = H.node_child[ra];
          ib = H.node_child[rb];
          F3 q0 = xf_point(X, {b0.x, b0.y, b0.z}), q1 = xf_point(X, {b1.x, b1.y, b1.z});
          F3 q2 = xf_point(X, {b2.x, b2.y, b2.z});
          bool cv;
          float gap = sweep_certificate<false>({a0.x, a0.y, a0.z}, {a1.x, a1.y, a1.z},
                                               {a2.x, a2.y, a2.z}, q0, q1, q2, sc, 0.f, &cv, nullptr);
          float thr = a0.w + b0.w + X.tau + X.margin;
          survive = !(gap > thr);
          both_leaf = ia.y < 0 && ib.y < 0;
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
      if (xfdd) {
        PairXfDD D;
        for (int k = 0; k < 9; ++k) {
          D.R[k] = dd(ok ? X64.R[k] : 0.0);
          D.RA[k] = dd(ok ? X64.RA[k] : 0.0);
        }
        for (int k = 0; k < 3; ++k) {
          D.t[k] = dd(ok ? X64.t[k] : 0.0);
          D.tA[k] = dd(ok ? X64.tA[k] : 0.0);
        }
        xfdd[p] = D;
      }
    }
    if (root_test) {
      tests.add(in && ok);
      surv.add(survive);
      warp_append(survive && both_leaf, make_tile(p, ra, rb, ia, ib), tiles, cnt + CNT_TILES,
                  cap_tiles, status + ST_REQ_TILES);
      warp_append(survive && !both_leaf, make_level(p, ra, rb, ia, ib), list0, cnt + CNT_LEVEL,
                  cap_level, status + ST_REQ_LEVEL);
    }
  }
  tests.flush(cnt + CNT_STATS + MRDEM_STAT_TESTS);
  surv.flush(cnt + CNT_STATS + MRDEM_STAT_SURVIVORS);
}

// ---------------------------------------------------------------------------
// The surrogate and fine tests are split into cheap culling kernels that
// emit compact lists of surviving pairs (the buffered comparisons of
// Sec. 5.4) and thread-per-pair sweep kernels that process those lists with
// every lane busy:
//   k_expand       the child pairs of surviving node pairs get a bounding-
//                  sphere test (node spheres precomputed in the body frame,
//                  radius including delta), then a separating-axis test of
//                  oriented boxes around their fine vertices; a warp takes up to 32 level
//                  items (fewer when the level is small, so that every
//                  resident warp has work) and deals their child pairs out
//                  to its lanes (near the leaves an item often has only 2 or
//                  4); survivors go to the sweep list;
//   k_sweep_nodes  one thread per listed node pair: penalty sweep + certificate
//                  against delta_a + delta_b + 2 eps; survivors become the
//                  next level's items, or leaf-pair tiles when both are leaves;
//   k_tile         one warp per leaf pair: fine triangles staged in shared
//                  memory, each tested against the other leaf's surrogate
//                  (Algorithm 5's fine-against-surrogate comparison), then the
//                  kept products against each other's bounding spheres;
//                  survivors go to the fine list;
//   k_sweep_fine   one thread per listed fine pair: the penalty sweep of
//                  Eq. 3/4 and the certificate at 2 eps; survivors are the
//                  candidates of the exact distance.
// Lists are taken in a fixed interleaved order by grids of exactly one
// resident wave.

// k_expand --------------------------------------------------------------------
// Loads of a work list or counter.  COH: the list was written earlier in
// the same launch by other blocks (the cooperative form), so the load goes
// through L2 (ld.global.cg), never the non-coherent read-only path.
template <bool COH>
__device__ __forceinline__ int4 ld_item(const int4* __restrict__ p) {
  if (COH) return __ldcg(p);
  return *p;
}
template <bool COH>
__device__ __forceinline__ int64_t ld_count(const unsigned long long* p) {
  if (COH) return (int64_t)__ldcg(p);
  return (int64_t)*p;
}

template <int WARPS>
struct ExpandSmem {
  int off[WARPS][32];
  int4 it[WARPS][32];
  int4 q[WARPS][128];
  int4 bq[WARPS][64];  // sphere survivors waiting for the box test
};

// The expand phase of a surrogate level (k_expand, k_levels, k_level): the
// child pairs of the level items get the node-sphere test; the sphere
// survivors queue per warp for the oriented-box test, which runs on full
// warps; the box survivors go to `sink` (warp-collective push(keep, item)).
// A warp takes up to max_items level items per pass.
template <int WARPS, bool COH, typename Sink>
__device__ __forceinline__ void expand_level(const HierDev& H, const PairXf* __restrict__ xf,
                                             const int4* __restrict__ in, int level,
                                             unsigned long long* cnt, int64_t cap_level,
                                             int max_items, int* off, int4* its, int4* bq,
                                             Sink& sink) {
  const int w = threadIdx.x >> 5, lane = lane_id();
  int64_t n_in = ld_count<COH>(cnt + CNT_LEVEL + level);
  if (n_in > cap_level) n_in = cap_level;
  const int slot_tests = MRDEM_STAT_TESTS + (level + 1 < MRDEM_STAT_LEVELS ? level + 1 : MRDEM_STAT_LEVELS - 1);
  WarpCount tests, boxcut;
  int nbq = 0;  // box-queue fill level (warp-uniform)
  // the oriented boxes of the last `take` queued sphere survivors: the two
  // children's fine geometry 2 eps apart (plus the pair's rounding margin)
  // means no fine pair below them can be a contact
  auto box_stage = [&](int take) {
    const bool have = lane < take;
    const int4 e = have ? bq[nbq - take + lane] : make_int4(0, 0, 0, 0);
    __syncwarp();
    nbq -= take;
    bool boxed = false;
    if (have) {
      PairXf X;
      load_pairxf(xf, e.x, X);
      boxed = boxes_apart_w(load_box(H, e.y), __ldg(H.node_boxw + e.y),
                            move_box(X, load_box(H, e.z)), __ldg(H.node_boxw + e.z),
                            X.tau + X.margin);
    }
    boxcut.add(boxed);
    sink.push(have && !boxed, e);
  };
  // items per warp and pass: the smallest power of two that spreads the
  // level over every resident warp, max_items at most (a power of two <= 32)
  const int64_t warps = (int64_t)gridDim.x * WARPS;
  int C = max_items;
  while (C > 1 && (int64_t)(C >> 1) * warps >= n_in) C >>= 1;
  const int64_t step = warps * C;
  int64_t base = ((int64_t)blockIdx.x * WARPS + w) * C;
  int4 nxt = lane < C && base + lane < n_in ? ld_item<COH>(in + base + lane) : make_int4(0, 0, 0, 0);
  for (; base < n_in; base += step) {
    // this warp's C items: child-pair counts, their offsets (exclusive scan)
    const int4 it = nxt;
    const bool valid = lane < C && base + lane < n_in;
    if (lane < C && base + step + lane < n_in) nxt = ld_item<COH>(in + base + step + lane);
    const int c = valid ? (it.w & 0xff) * ((it.w >> 8) & 0xff) : 0;
    const int incl = warp_scan(c);
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    off[lane] = incl - c;
    its[lane] = it;
    __syncwarp();
    for (int f0 = 0; f0 < total; f0 += 32) {
      const int f = f0 + lane;
      const bool act = f < total;
      // owner: the last of the C items whose offset is <= f (items without
      // child pairs share the next item's offset and are never picked)
      int l = 0;
      for (int b = C >> 1; b > 0; b >>= 1)
        if (off[l + b] <= f) l += b;
      const int4 o = its[l];
      const int nb = (o.w >> 8) & 0xff;
      const int r = act ? f - off[l] : 0;
      const int i = (int)(((float)r + 0.5f) * (1.0f / (float)(nb > 0 ? nb : 1)));
      const int j = r - i * nb;
      bool keep = false;
      if (act) {
        PairXf X;
        load_pairxf(xf, o.x, X);
        float4 p = __ldg(H.node_sph + o.y + i), q = __ldg(H.node_sph + o.z + j);
        F3 cq = xf_point(X, {q.x, q.y, q.z});
        float dx = p.x - cq.x, dy = p.y - cq.y, dz = p.z - cq.z;
        float lim = p.w + q.w + X.tau + X.margin;
        keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= lim * lim;
      }
      tests.add(act);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) bq[nbq + __popc(m & ((1u << lane) - 1u))] = make_int4(o.x, o.y + i, o.z + j, 0);
      nbq += __popc(m);
      __syncwarp();
      if (nbq >= 32) box_stage(32);
    }
    __syncwarp();
  }
  if (nbq > 0) box_stage(nbq);
  sink.finish();
  tests.flush(cnt + CNT_STATS + slot_tests);
  boxcut.flush(cnt + CNT_STATS + MRDEM_STAT_BOX_PRUNED);
}

// Box survivors to the sweep list of the level (k_expand, k_levels).
struct SweepListSink {
  WarpQueue<int4, 128> q;
  int4* sweep;
  unsigned long long* counter;
  int64_t cap;
  unsigned long long* req;
  __device__ __forceinline__ void push(bool keep, int4 e) { q.push(keep, e, sweep, counter, cap, req); }
  __device__ __forceinline__ void finish() { q.flush(sweep, counter, cap, req); }
};

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_expand(HierDev H, const PairXf* __restrict__ xf,
                                                       const int4* __restrict__ in, int level,
                                                       int4* sweep, unsigned long long* cnt,
                                                       unsigned long long* status,
                                                       int64_t cap_level, int64_t cap_sweep,
                                                       int max_items) {
  wait_prior_grid();
  __shared__ ExpandSmem<WARPS> sm;
  const int w = threadIdx.x >> 5;
  SweepListSink sink = {{sm.q[w]}, sweep, cnt + CNT_SWEEP + level, cap_sweep, status + ST_REQ_SWEEP};
  expand_level<WARPS, false>(H, xf, in, level, cnt, cap_level, max_items, sm.off[w], sm.it[w],
                             sm.bq[w], sink);
}

// k_sweep_nodes ---------------------------------------------------------------
struct SweepNodesSmem {
  TileItem tq[8][64];
  int4 lq[8][64];
};

// The surrogate-level test of one node pair e (pair, node of A, node of B)
// that passed the culls: the float penalty sweep with its certificate
// against delta_a + delta_b + 2 eps, then the surrogates' face normals as
// further separating axes.  True when the pair may hold a contact; ia, ib
// get the two nodes' child records.
__device__ __forceinline__ bool node_pair_survives(const HierDev& H, const PairXf* __restrict__ xf,
                                                   const SweepConst& sc, int4 e, int2& ia,
                                                   int2& ib) {
  PairXf X;
  load_pairxf(xf, e.x, X);
  float4 a0 = __ldg(H.node_geo + 3 * e.y), a1 = __ldg(H.node_geo + 3 * e.y + 1);
  float4 a2 = __ldg(H.node_geo + 3 * e.y + 2);
  float4 b0 = __ldg(H.node_geo + 3 * e.z), b1 = __ldg(H.node_geo + 3 * e.z + 1);
  float4 b2 = __ldg(H.node_geo + 3 * e.z + 2);
  ia = __ldg(H.node_child + e.y);
  ib = __ldg(H.node_child + e.z);
  F3 q0 = xf_point(X, {b0.x, b0.y, b0.z}), q1 = xf_point(X, {b1.x, b1.y, b1.z});
  F3 q2 = xf_point(X, {b2.x, b2.y, b2.z});
  bool cv;
  float gap;
  F3 p0 = {a0.x, a0.y, a0.z}, p1 = {a1.x, a1.y, a1.z}, p2 = {a2.x, a2.y, a2.z};
  if (sc.n_iter == 4)
    gap = sweep_certificate<false, 4>(p0, p1, p2, q0, q1, q2, sc, 0.f, &cv, nullptr);
  else
    gap = sweep_certificate<false, 0>(p0, p1, p2, q0, q1, q2, sc, 0.f, &cv, nullptr);
  const float thr = a0.w + b0.w + X.tau + X.margin;
  if (!(gap > thr)) gap = fmaxf(axis_gap(cross(p1 - p0, p2 - p0), p0, p1, p2, q0, q1, q2),
                                axis_gap(cross(q1 - q0, q2 - q0), p0, p1, p2, q0, q1, q2));
  return !(gap > thr);
}

template <bool COH>
__device__ __forceinline__ void sweep_level(const HierDev& H, const PairXf* __restrict__ xf,
                                            const SweepConst& sc, const int4* __restrict__ sweep,
                                            int level,
                                            int4* out, TileItem* tiles, unsigned long long* cnt,
                                            unsigned long long* status, int64_t cap_sweep,
                                            int64_t cap_level, int64_t cap_tiles,
                                            SweepNodesSmem& sm) {
  int64_t n = ld_count<COH>(cnt + CNT_SWEEP + level);
  if (n > cap_sweep) n = cap_sweep;
  const int slot_surv = MRDEM_STAT_SURVIVORS + (level + 1 < MRDEM_STAT_LEVELS ? level + 1 : MRDEM_STAT_LEVELS - 1);
  WarpCount nsweep, surv;
  const int w = threadIdx.x >> 5;
  WarpQueue<TileItem, 64> tq;
  WarpQueue<int4, 64> lq;
  tq.buf = sm.tq[w];
  lq.buf = sm.lq[w];
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    bool act = k < n, s = false;
    int4 e = act ? ld_item<COH>(sweep + k) : make_int4(0, 0, 0, 0);
    int2 ia = make_int2(0, 1), ib = make_int2(0, 1);
    if (act) s = node_pair_survives(H, xf, sc, e, ia, ib);
    bool leaves = ia.y < 0 && ib.y < 0;
    nsweep.add(act);
    surv.add(s);
    tq.push(s && leaves, make_tile(e.x, e.y, e.z, ia, ib), tiles, cnt + CNT_TILES, cap_tiles,
            status + ST_REQ_TILES);
    lq.push(s && !leaves, make_level(e.x, e.y, e.z, ia, ib), out, cnt + CNT_LEVEL + level + 1,
            cap_level, status + ST_REQ_LEVEL);
  }
  tq.flush(tiles, cnt + CNT_TILES, cap_tiles, status + ST_REQ_TILES);
  lq.flush(out, cnt + CNT_LEVEL + level + 1, cap_level, status + ST_REQ_LEVEL);
  nsweep.flush(cnt + CNT_STATS + MRDEM_STAT_LEVEL_SWEEPS);
  surv.flush(cnt + CNT_STATS + slot_surv);
}

__global__ void __launch_bounds__(256, 4) k_sweep_nodes(HierDev H, const PairXf* __restrict__ xf,
                                                     SweepConst sc, const int4* __restrict__ sweep,
                                                     int level, int4* out, TileItem* tiles,
                                                     unsigned long long* cnt,
                                                     unsigned long long* status, int64_t cap_sweep,
                                                     int64_t cap_level, int64_t cap_tiles) {
  wait_prior_grid();
  __shared__ SweepNodesSmem sm;
  sweep_level<false>(H, xf, sc, sweep, level, out, tiles, cnt, status, cap_sweep, cap_level,
                     cap_tiles, sm);
}

// k_levels: every surrogate level in one cooperative launch (level_kernel 1):
// for each level the expand phase and the sweep phase of the two kernels
// above, separated by grid-wide barriers, over the same one-wave grid (so
// the level lists keep their interleaved assignment).  The lists the phases
// read were written in the same launch, hence the L2 loads.  It saves the
// launches and the per-launch ramps; each barrier waits for the level's
// slowest block, as the launch boundary did.  Three blocks per SM (80
// registers; the two phases alone would take 111 and allow two).
constexpr int kLevelWarps = 8;
union LevelSmem {
  ExpandSmem<kLevelWarps> e;
  SweepNodesSmem s;
};
__global__ void __launch_bounds__(kLevelWarps * 32, 3) k_levels(
    HierDev H, const PairXf* __restrict__ xf, SweepConst sc, int4* list0, int4* list1,
    int4* sweep, TileItem* tiles, unsigned long long* cnt, unsigned long long* status,
    int64_t cap_level, int64_t cap_sweep, int64_t cap_tiles, int steps, int max_items) {
  wait_prior_grid();
  __shared__ LevelSmem sm;
  cg::grid_group g = cg::this_grid();
  const int w = threadIdx.x >> 5;
  for (int l = 0; l < steps; ++l) {
    SweepListSink sink = {{sm.e.q[w]}, sweep, cnt + CNT_SWEEP + l, cap_sweep, status + ST_REQ_SWEEP};
    expand_level<kLevelWarps, true>(H, xf, (l & 1) ? list1 : list0, l, cnt, cap_level, max_items,
                                    sm.e.off[w], sm.e.it[w], sm.e.bq[w], sink);
    g.sync();
    sweep_level<true>(H, xf, sc, sweep, l, ((l + 1) & 1) ? list1 : list0, tiles, cnt, status,
                      cap_sweep, cap_level, cap_tiles, sm.s);
    if (l + 1 < steps) g.sync();
  }
}

// k_level: one surrogate level in one launch (level_kernel 2).  The expand
// phase's box survivors queue per warp in shared memory and are swept by
// the same warp 32 at a time (the sweep phase above), so no sweep list goes
// through memory and a level is one launch instead of two.
template <int WARPS>
struct LevelFusedSmem {
  int off[WARPS][32];
  int4 it[WARPS][32];
  int4 bq[WARPS][64];
  int4 sq[WARPS][64];
  int4 lq[WARPS][64];
  TileItem tq[WARPS][64];
};
struct SweepHereSink {
  const HierDev& H;
  const PairXf* xf;
  const SweepConst& sc;
  int4* sq;
  int ns;  // queue fill level (warp-uniform)
  WarpQueue<TileItem, 64> tq;
  WarpQueue<int4, 64> lq;
  int4* out;
  TileItem* tiles;
  unsigned long long* cnt;
  unsigned long long* status;
  int level;
  int64_t cap_level, cap_tiles;
  WarpCount nsweep, surv;
  // the sweep phase on the last `take` queued node pairs
  __device__ __forceinline__ void stage(int take) {
    const int lane = lane_id();
    const bool have = lane < take;
    const int4 e = have ? sq[ns - take + lane] : make_int4(0, 0, 0, 0);
    __syncwarp();
    ns -= take;
    int2 ia = make_int2(0, 1), ib = make_int2(0, 1);
    const bool s = have && node_pair_survives(H, xf, sc, e, ia, ib);
    const bool leaves = ia.y < 0 && ib.y < 0;
    nsweep.add(have);
    surv.add(s);
    tq.push(s && leaves, make_tile(e.x, e.y, e.z, ia, ib), tiles, cnt + CNT_TILES, cap_tiles,
            status + ST_REQ_TILES);
    lq.push(s && !leaves, make_level(e.x, e.y, e.z, ia, ib), out, cnt + CNT_LEVEL + level + 1,
            cap_level, status + ST_REQ_LEVEL);
  }
  __device__ __forceinline__ void push(bool keep, int4 e) {
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) sq[ns + __popc(m & ((1u << lane_id()) - 1u))] = e;
    ns += __popc(m);
    __syncwarp();
    if (ns >= 32) stage(32);
  }
  __device__ __forceinline__ void finish() {
    if (ns > 0) stage(ns);
    tq.flush(tiles, cnt + CNT_TILES, cap_tiles, status + ST_REQ_TILES);
    lq.flush(out, cnt + CNT_LEVEL + level + 1, cap_level, status + ST_REQ_LEVEL);
    const int slot_surv = MRDEM_STAT_SURVIVORS + (level + 1 < MRDEM_STAT_LEVELS ? level + 1 : MRDEM_STAT_LEVELS - 1);
    nsweep.flush(cnt + CNT_STATS + MRDEM_STAT_LEVEL_SWEEPS);
    surv.flush(cnt + CNT_STATS + slot_surv);
  }
};
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_level(HierDev H, const PairXf* __restrict__ xf,
                                                      SweepConst sc, const int4* __restrict__ in,
                                                      int level, int4* out, TileItem* tiles,
                                                      unsigned long long* cnt,
                                                      unsigned long long* status,
                                                      int64_t cap_level, int64_t cap_tiles,
                                                      int max_items) {
  wait_prior_grid();
  __shared__ LevelFusedSmem<WARPS> sm;
  const int w = threadIdx.x >> 5;
  SweepHereSink sink = {H, xf, sc, sm.sq[w], 0, {}, {}, out, tiles, cnt, status, level,
                        cap_level, cap_tiles, {}, {}};
  sink.tq.buf = sm.tq[w];
  sink.lq.buf = sm.lq[w];
  expand_level<WARPS, false>(H, xf, in, level, cnt, cap_level, max_items, sm.off[w], sm.it[w],
                             sm.bq[w], sink);
}

// k_tile ----------------------------------------------------------------------
struct TileSmem {
  float4 sa[32];  // bounding spheres: centroid xyz, radius
  float4 sb[32];
  unsigned char ka[32], kb[32];  // triangles kept by the fine-vs-surrogate test
};

// A leaf's surrogate as seen from the other particle (A's frame): the unit
// normal and offset of its plane and its node sphere (centre, largest vertex
// distance + delta).
struct SurrogateBound {
  F3 n;
  float off;
  float4 sph;
};
// Can a point of the sphere (c, r) come within delta + thr of the surrogate
// triangle?  Two necessary conditions, both branch-free: within
// delta + thr + r of its plane (the distance to a triangle is at least the
// distance to its plane), and within the node radius + thr + r of the node
// centre.  A NaN keeps the sphere.
__device__ __forceinline__ bool sphere_near_surrogate(float4 s, const SurrogateBound& b,
                                                      float delta, float thr) {
  float pd = fabsf(fmaf(b.n.x, s.x, fmaf(b.n.y, s.y, fmaf(b.n.z, s.z, -b.off))));
  float dx = s.x - b.sph.x, dy = s.y - b.sph.y, dz = s.z - b.sph.z;
  float lim = b.sph.w + thr + s.w;
  return !(pd > delta + thr + s.w) && !(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > lim * lim);
}

__device__ __forceinline__ TileItem load_tile(const TileItem* tiles, int64_t t) {
  const int4* p = reinterpret_cast<const int4*>(tiles + t);
  int4 a = __ldg(p), b = __ldg(p + 1);
  TileItem r;
  r.pair = a.x; r.node_a = a.y; r.node_b = a.z; r.slot_a = a.w;
  r.slot_b = b.x; r.counts = b.y; r.pad0 = r.pad1 = 0;
  return r;
}


template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 4) k_tile(HierDev H, const PairXf* __restrict__ xf,
                                                     const TileItem* __restrict__ tiles,
                                                     int4* fine, unsigned long long* cnt,
                                                     unsigned long long* status, int64_t cap_tiles,
                                                     int64_t cap_fine) {
  wait_prior_grid();
  __shared__ TileSmem smem[WARPS];
  __shared__ int4 sq[WARPS][128];
  const int w = threadIdx.x >> 5, lane = lane_id();
  TileSmem& S = smem[w];
  WarpQueue<int4, 128> q;
  q.buf = sq[w];
  int64_t n_tiles = (int64_t)cnt[CNT_TILES];
  if (n_tiles > cap_tiles) n_tiles = cap_tiles;
  WarpCount spheres;
  unsigned ntile = 0, nfvs = 0;
  const int64_t step = (int64_t)gridDim.x * WARPS;
  int64_t t = (int64_t)blockIdx.x * WARPS + w;
  TileItem nxt;
  if (t < n_tiles) nxt = load_tile(tiles, t);
  for (; t < n_tiles; t += step) {
    const TileItem it = nxt;
    if (t + step < n_tiles) nxt = load_tile(tiles, t + step);
    ++ntile;
    PairXf X;
    load_pairxf(xf, it.pair, X);
    int na = it.counts & 0xff, nb = (it.counts >> 8) & 0xff;
    const float thr = X.tau + X.margin;
    bool keep_a = false, keep_b = false;
    // the two leaves' surrogates as seen from the other side (A's frame)
    const float da = __ldg(&H.node_geo[3 * it.node_a].w), db = __ldg(&H.node_geo[3 * it.node_b].w);
    float4 nA = __ldg(H.node_nrm + it.node_a), nB = __ldg(H.node_nrm + it.node_b);
    float4 sphA = __ldg(H.node_sph + it.node_a), sphB = __ldg(H.node_sph + it.node_b);
    SurrogateBound bA = {{nA.x, nA.y, nA.z}, nA.w, sphA};
    SurrogateBound bB;
    {
      F3 c = xf_point(X, {sphB.x, sphB.y, sphB.z});
      bB.sph = make_float4(c.x, c.y, c.z, sphB.w);
      // rotate the normal; the offset moves by n'.t
      bB.n = {fmaf(X.R[0], nB.x, fmaf(X.R[1], nB.y, X.R[2] * nB.z)),
              fmaf(X.R[3], nB.x, fmaf(X.R[4], nB.y, X.R[5] * nB.z)),
              fmaf(X.R[6], nB.x, fmaf(X.R[7], nB.y, X.R[8] * nB.z))};
      bB.off = nB.w + fmaf(bB.n.x, X.t[0], fmaf(bB.n.y, X.t[1], bB.n.z * X.t[2]));
    }
    if (lane < na) {
      float4 sp = __ldg(H.tri_sph + it.slot_a + lane);
      S.sa[lane] = sp;
      keep_a = sphere_near_surrogate(sp, bB, db, thr);
    }
    if (lane < nb) {
      float4 sb = __ldg(H.tri_sph + it.slot_b + lane);
      F3 c = xf_point(X, {sb.x, sb.y, sb.z});
      float4 sp = make_float4(c.x, c.y, c.z, sb.w);
      S.sb[lane] = sp;
      keep_b = sphere_near_surrogate(sp, bA, da, thr);
    }
    unsigned ma = __ballot_sync(0xffffffffu, keep_a), mb = __ballot_sync(0xffffffffu, keep_b);
    if (keep_a) S.ka[__popc(ma & ((1u << lane) - 1u))] = (unsigned char)lane;
    if (keep_b) S.kb[__popc(mb & ((1u << lane) - 1u))] = (unsigned char)lane;
    const int ka = __popc(ma), kb = __popc(mb);
    nfvs += (unsigned)(na + nb);
    __syncwarp();
    const int total = ka * kb;
    const float inv_kb = 1.0f / (float)(kb > 0 ? kb : 1);
    for (int f0 = 0; f0 < total; f0 += 32) {
      int f = f0 + lane;
      bool act = f < total;
      int ii = (int)(((float)f + 0.5f) * inv_kb);
      int jj = f - ii * kb;
      if (!act) { ii = 0; jj = 0; }
      int i = S.ka[ii], j = S.kb[jj];
      float4 p = S.sa[i], r = S.sb[j];
      float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
      float lim = (p.w + r.w) + thr;
      bool keep = act && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= lim * lim;
      q.push(keep, make_int4(it.pair, it.slot_a + i, it.slot_b + j, 0), fine, cnt + CNT_FINE,
             cap_fine, status + ST_REQ_SWEEP);
    }
    spheres.v += lane == 0 ? (unsigned)total : 0u;
    __syncwarp();
  }
  q.flush(fine, cnt + CNT_FINE, cap_fine, status + ST_REQ_SWEEP);
  if (lane == 0) {
    if (ntile) atomicAdd(cnt + CNT_STATS + MRDEM_STAT_TILES, (unsigned long long)ntile);
    if (nfvs) atomicAdd(cnt + CNT_STATS + MRDEM_STAT_FINE_SURROGATE, (unsigned long long)nfvs);
  }
  spheres.flush(cnt + CNT_STATS + MRDEM_STAT_SPHERE_TESTS);
}

// k_sweep_fine ----------------------------------------------------------------
// Fine pairs awaiting the sweep, per warp: A's triangle and B's (in A's
// frame) as 18 floats, the pair entry and the thresholds.  At most 31 wait
// between rounds and a round adds at most 32.
struct FineQueue {
  float g[18][64];
  int4 e[64];
  float thr[64], ce2[64];
};

template <int WARPS, bool CONV>
__global__ void __launch_bounds__(WARPS * 32) k_sweep_fine(
    HierDev H, const PairXf* __restrict__ xf, SweepConst sc, float conv_c,
    const int4* __restrict__ fine, int3* cands, unsigned long long* cnt, unsigned long long* status,
    int64_t cap_fine, int64_t cap_cands, const double* __restrict__ eps_d) {
  wait_prior_grid();
  __shared__ FineQueue smem[WARPS];
  __shared__ int3 scq[WARPS][64];
  const int w = threadIdx.x >> 5, lane = lane_id();
  FineQueue& Q = smem[w];
  WarpQueue<int3, 64> cq;
  cq.buf = scq[w];
  int64_t n = (int64_t)cnt[CNT_FINE];
  if (n > cap_fine) n = cap_fine;
  WarpCount tests, nsweep, ncand, nodot;
  int qn = 0;  // warp-uniform queue fill
  // the sweep and its certificate for queue entry `slot` (-1: idle lane)
  auto sweep_slot = [&](int slot) {
    bool s = false, cv = true;
    if (slot >= 0) {
      F3 v[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) v[c] = {Q.g[3 * c][slot], Q.g[3 * c + 1][slot], Q.g[3 * c + 2][slot]};
      float gap;
      if (sc.n_iter == 4)
        gap = sweep_certificate<CONV, 4>(v[0], v[1], v[2], v[3], v[4], v[5], sc, Q.ce2[slot], &cv, nullptr);
      else
        gap = sweep_certificate<CONV, 0>(v[0], v[1], v[2], v[3], v[4], v[5], sc, Q.ce2[slot], &cv, nullptr);
      s = !(gap > Q.thr[slot]);
    }
    nsweep.add(slot >= 0);
    ncand.add(s);
    if (CONV) nodot.add(s && !cv);
    const int4 e = Q.e[slot >= 0 ? slot : 0];
    cq.push(s, make_int3(e.x, e.y, e.z), cands, cnt + CNT_CANDS, cap_cands, status + ST_REQ_CANDS);
  };
  const int64_t step = (int64_t)gridDim.x * WARPS * 32;
  int64_t base = ((int64_t)blockIdx.x * WARPS + w) * 32;
  // the next round's entry is loaded a round ahead, so that a round's
  // gathers (transform, triangles) start at once
  int4 nxt = base + lane < n ? fine[base + lane] : make_int4(0, 0, 0, 0);
  for (; base < n; base += step) {
    const int64_t k = base + lane;
    const bool act = k < n;
    bool need = false;
    const int4 e = nxt;
    if (k + step < n) nxt = fine[k + step];
    F3 p0, p1, p2, q0, q1, q2;
    float thr = 0.f, ce = 0.f;
    if (act) {
      PairXf X;
      load_pairxf(xf, e.x, X);
      ce = conv_c * (float)__ldg(eps_d + e.x);
      F3 a[3], b[3];
      load_tri(H, e.y, a);
      load_tri(H, e.z, b);
      p0 = a[0]; p1 = a[1]; p2 = a[2];
      q0 = xf_point(X, b[0]); q1 = xf_point(X, b[1]); q2 = xf_point(X, b[2]);
      thr = X.tau + X.margin;
      // the face normals first: they separate most pairs at a tenth of the
      // sweep's cost
      float gap = fmaxf(axis_gap(cross(p1 - p0, p2 - p0), p0, p1, p2, q0, q1, q2),
                        axis_gap(cross(q1 - q0, q2 - q0), p0, p1, p2, q0, q1, q2));
      need = !(gap > thr);
    }
    tests.add(act);
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (need) {
      const int slot = qn + __popc(m & ((1u << lane) - 1u));
      const F3 v[6] = {p0, p1, p2, q0, q1, q2};
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        Q.g[3 * c][slot] = v[c].x;
        Q.g[3 * c + 1][slot] = v[c].y;
        Q.g[3 * c + 2][slot] = v[c].z;
      }
      Q.e[slot] = e;
      Q.thr[slot] = thr;
      Q.ce2[slot] = ce * ce;
    }
    qn += __popc(m);
    __syncwarp();
    if (qn >= 32) {
      sweep_slot(qn - 32 + lane);
      qn -= 32;
      __syncwarp();
    }
  }
  if (qn > 0) sweep_slot(lane < qn ? lane : -1);
  cq.flush(cands, cnt + CNT_CANDS, cap_cands, status + ST_REQ_CANDS);
  tests.flush(cnt + CNT_STATS + MRDEM_STAT_FINE_TESTS);
  nsweep.flush(cnt + CNT_STATS + MRDEM_STAT_FINE_SWEEPS);
  ncand.flush(cnt + CNT_STATS + MRDEM_STAT_CANDIDATES);
  if (CONV) nodot.flush(cnt + CNT_STATS + MRDEM_STAT_UNCONVERGED);
}

// ---------------------------------------------------------------------------
// Final distance of the candidates.
//   FP64 form: the comparison-based distance in double for every candidate
//   (k_exact64).
//   FP32 form of mrdem_detect: the float stage and double-float work items of
//   mrdem_closest.cu.
//   FP32 form of the allocation-free entry point, whose fixed scratch has no
//   room for work-item lists: one kernel (k_exact32) with the same float
//   stage (error bound err = 2^-15 max|coordinate| on coordinates relative to
//   A's first vertex); every sub-test within 2 err of the float minimum is
//   re-evaluated in double in the same thread and the smallest value is the
//   distance (the true minimiser is always among them); crossing or nearly
//   touching pairs go to a fallback list that k_exact64 finishes.
// k_exact32, the one-kernel FP32 form.  The float stage runs on float
// coordinates (B moved by the float transform; its error is within the
// pair's margin), so pairs it rejects never touch double arithmetic; the
// others are finished in double from the double transform.
__global__ void __launch_bounds__(256) k_exact32(HierDev H, const PairXf* __restrict__ xf,
                                                 const PairXf64* __restrict__ xf64,
                                                 const int3* __restrict__ cands,
                                                 unsigned long long* cnt,
                                                 unsigned long long* status, int64_t cap_cands,
                                                 int3* fallback, int64_t cap_fallback,
                                                 mrdem_contacts out) {
  int64_t n = (int64_t)cnt[CNT_CANDS];
  if (n > cap_cands) n = cap_cands;
  WarpCount ncon;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    int res = 0;
    int3 c = make_int3(0, 0, 0);
    double d = 0;
    D3 pa = {0, 0, 0}, pb = {0, 0, 0};
    unsigned mask = 0;
    if (k < n) {
      c = cands[k];
      PairXf X;
      load_pairxf(xf, c.x, X);
      F3 a[3], b[3];
      load_tri(H, c.y, a);
      load_tri(H, c.z, b);
      F3 Pf[3] = {{0.f, 0.f, 0.f}, a[1] - a[0], a[2] - a[0]};
      F3 Qf[3] = {xf_point(X, b[0]) - a[0], xf_point(X, b[1]) - a[0], xf_point(X, b[2]) - a[0]};
      res = cand_float_stage(Pf, Qf, (double)X.tau, X.margin, &mask);
    }
    // finish the accepted pairs in double (only these lanes touch FP64)
    if (res == 1) {
      const PairXf64& X64 = xf64[c.x];
      CandGeom g;
      cand_geom(H, X64, c, g);
      d = cand_double_stage(g, mask, pa, pb, nullptr, nullptr);
      if (d <= g.tau) {
        pa = xf_point64(X64.RA, X64.tA, pa + g.o);
        pb = xf_point64(X64.RA, X64.tA, pb + g.o);
      } else {
        res = 0;
      }
    }
    ncon.add(res == 1);
    write_contact(H, out, status, res == 1, c.x, c.y, c.z, d, pa, pb);
    warp_append(res < 0, c, fallback, cnt + CNT_FALLBACK, cap_fallback, status + ST_REQ_CANDS);
  }
  ncon.flush(cnt + CNT_STATS + MRDEM_STAT_CONTACTS);
}

// Full FP64 comparison-based distance for every entry of a list (the FP64
// form's candidates, or the fallback list of the one-kernel FP32 form).
__global__ void __launch_bounds__(256) k_exact64(HierDev H, const PairXf64* __restrict__ xf64,
                                                 const int3* __restrict__ list,
                                                 unsigned long long* cnt, int count_slot,
                                                 int64_t cap, unsigned long long* status,
                                                 int stat_slot, mrdem_contacts out, int32_t* pair_cnt) {
  wait_prior_grid();
  int64_t n = (int64_t)cnt[count_slot];
  if (n > cap) n = cap;
  WarpCount ncon, nall;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    bool hit = false;
    int3 c = make_int3(0, 0, 0);
    double d = 0;
    D3 pa = {0, 0, 0}, pb = {0, 0, 0};
    if (k < n) {
      c = list[k];
      const PairXf64& X = xf64[c.x];
      CandGeom g;
      cand_geom(H, X, c, g);
      TriTriResult<double> r = tri_tri_distance(g.P, g.Q);
      hit = r.d <= g.tau;
      d = r.d;
      if (hit) {
        pa = xf_point64(X.RA, X.tA, r.pa + g.o);
        pb = xf_point64(X.RA, X.tA, r.pb + g.o);
      }
    }
    ncon.add(hit);
    nall.add(k < n);
    write_contact(H, out, status, hit, c.x, c.y, c.z, d, pa, pb, pair_cnt);
  }
  ncon.flush(cnt + CNT_STATS + MRDEM_STAT_CONTACTS);
  if (stat_slot >= 0) nall.flush(cnt + CNT_STATS + stat_slot);
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
    CandGeom g;
    for (int v = 0; v < 3; ++v) {
      g.P[v] = {Pin[9 * k + 3 * v], Pin[9 * k + 3 * v + 1], Pin[9 * k + 3 * v + 2]};
      g.Q[v] = {Qin[9 * k + 3 * v], Qin[9 * k + 3 * v + 1], Qin[9 * k + 3 * v + 2]};
    }
    g.o = g.P[0];
    for (int v = 2; v >= 0; --v) { g.P[v] = g.P[v] - g.o; g.Q[v] = g.Q[v] - g.o; }
    double e = eps[k];
    g.tau = 2.0 * e;
    if (sx || sgap || sconv) {
      F3 Pf[3], Qf[3];
      for (int v = 0; v < 3; ++v) {
        Pf[v] = {(float)g.P[v].x, (float)g.P[v].y, (float)g.P[v].z};
        Qf[v] = {(float)g.Q[v].x, (float)g.Q[v].y, (float)g.Q[v].z};
      }
      float ce = conv_c * (float)e;
      bool cv;
      float x[4];
      float gp = sweep_certificate<true>(Pf[0], Pf[1], Pf[2], Qf[0], Qf[1], Qf[2], sc, ce * ce, &cv, x);
      if (sx) for (int q = 0; q < 4; ++q) sx[4 * k + q] = x[q];
      if (sgap) sgap[k] = gp;
      if (sconv) sconv[k] = cv;
    }
    if (dist || pa || pb || feature) {
      double d = 0;
      D3 a = {0, 0, 0}, b = {0, 0, 0};
      int f = -1;
      int res = -1;
      if (PREC == MRDEM_PREC_FP32) {
        // the detection's FP32 form: float stage, then double-float finishing
        // of the sub-tests it keeps, or of the full test for a fallback pair
        F3 Pf[3], Qf[3];
        float L = 0.f;
        for (int v = 0; v < 3; ++v) {
          Pf[v] = {(float)g.P[v].x, (float)g.P[v].y, (float)g.P[v].z};
          Qf[v] = {(float)g.Q[v].x, (float)g.Q[v].y, (float)g.Q[v].z};
          L = fmaxf(L, fmaxf(fmaxf(fabsf(Pf[v].x), fabsf(Pf[v].y)),
                             fmaxf(fmaxf(fabsf(Pf[v].z), fabsf(Qf[v].x)), fmaxf(fabsf(Qf[v].y), fabsf(Qf[v].z)))));
        }
        unsigned mask = 0;
        res = cand_float_stage(Pf, Qf, g.tau, 0.f, &mask);
        if (res != 0) {
          const int ks = L > 0.f ? ilogbf(L) : 0;
          const float sc2 = ldexpf(1.f, -ks);
          V3<dd> P[3], Q[3];
          for (int v = 0; v < 3; ++v) {
            P[v] = scale_dd(to_dd(g.P[v]), sc2);
            Q[v] = scale_dd(to_dd(g.Q[v]), sc2);
          }
          V3<dd> pa2, pb2;
          dd best;
          if (res == 1) {
            best = dd(INFINITY);
            for (int q = 0; q < 15; ++q) {
              if (!((mask >> q) & 1u)) continue;
              V3<dd> x, y;
              dd wa[3], wb[3];
              dd v2 = eval_subtest(P, Q, q, &x, &y, wa, wb);
              if (v2 < best) { best = v2; pa2 = x; pb2 = y; f = q; }
            }
            d = ldexp(to_double(dd_sqrt(best)), ks);
            if (!(d <= g.tau)) res = 0;
          } else {
            TriTriResult<dd> r = tri_tri_distance(P, Q);
            d = ldexp(to_double(r.d), ks);
            pa2 = r.pa; pb2 = r.pb; f = r.feature;
            res = 1;
          }
          const float us = ldexpf(1.f, ks);
          a = to_double(scale_dd(pa2, us));
          b = to_double(scale_dd(pb2, us));
        }
      }
      if (res != 1) {
        // FP64 form, or a pair the FP32 form puts beyond 2 eps: report the
        // full double result (feature -2 marks the FP32 form's rejection)
        TriTriResult<double> r = tri_tri_distance(g.P, g.Q);
        d = r.d; a = r.pa; b = r.pb; f = res == 0 ? -2 : r.feature;
      }
      if (dist) dist[k] = d;
      a = a + g.o;
      b = b + g.o;
      if (pa) { pa[3 * k] = a.x; pa[3 * k + 1] = a.y; pa[3 * k + 2] = a.z; }
      if (pb) { pb[3 * k] = b.x; pb[3 * k + 1] = b.y; pb[3 * k + 2] = b.z; }
      if (feature) feature[k] = f;
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
int ensure_pairs(mrdem_ctx* c, int64_t n) {
  if (n <= c->cap_pairs) return MRDEM_OK;
  int64_t cap = c->cap_pairs ? c->cap_pairs : 1024;
  while (cap < n) cap *= 2;
  cudaFree(c->xf);
  cudaFree(c->xf64);
  cudaFree(c->xfdd);
  cudaFree(c->pair_cnt);
  c->xf = nullptr;
  c->xf64 = nullptr;
  c->xfdd = nullptr;
  c->pair_cnt = nullptr;
  c->cap_pairs = 0;
  if (cudaMalloc(&c->xf, sizeof(PairXf) * cap) != cudaSuccess ||
      cudaMalloc(&c->xf64, sizeof(PairXf64) * cap) != cudaSuccess ||
      cudaMalloc(&c->xfdd, sizeof(PairXfDD) * cap) != cudaSuccess ||
      cudaMalloc(&c->pair_cnt, sizeof(int32_t) * cap) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->xf);
    cudaFree(c->xf64);
    cudaFree(c->xfdd);
    c->xf = nullptr;
    c->xf64 = nullptr;
    c->xfdd = nullptr;
    return MRDEM_ERR_OOM;
  }
  c->cap_pairs = cap;
  return MRDEM_OK;
}

// Blocks for a persistent launch: exactly the blocks that fit on the GPU at
// once (SMs x resident blocks per SM), so that interleaved work assignment
// has no second wave.
template <typename K>
static int one_wave(mrdem_ctx* c, K kernel, int threads, size_t smem) {
  const void* k = reinterpret_cast<const void*>(kernel);
  for (int i = 0; i < c->n_occ; ++i)
    if (c->occ[i].kernel == k && c->occ[i].threads == threads && c->occ[i].smem == smem)
      return c->occ[i].blocks * c->n_sms;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess || b <= 0) {
    cudaGetLastError();
    b = 1;
  }
  if (c->n_occ < (int)(sizeof(c->occ) / sizeof(c->occ[0]))) c->occ[c->n_occ++] = {k, threads, smem, b};
  return b * c->n_sms;
}

// Launch shapes: the autotuned entry of the call's size class, else the
// context's parameters.
Shape shape_for(const mrdem_ctx* c, int64_t n_pairs) {
  if (c->force_shape) return *c->force_shape;
  const int k = size_class(n_pairs);
  if (c->tuned_ok[k]) return c->tuned[k];
  const mrdem_params& p = c->params;
  return {p.level_warps, p.expand_items, p.node_threads, p.tile_warps, p.sweep_warps,
          p.exact_threads, p.level_kernel};
}

// Launch helpers over the kernels' block shapes (one template instance per
// shape; `pdl` chains the launch to the previous kernel of the stream).
template <typename... Exp, typename... Act>
static void launch_pdl(bool pdl, void (*kernel)(Exp...), int grid, int block, cudaStream_t s,
                       Act&&... args) {
  if (pdl) launch_after(kernel, grid, block, 0, s, std::forward<Act>(args)...);
  else kernel<<<grid, block, 0, s>>>(std::forward<Act>(args)...);
}
template <int W>
static void expand_w(mrdem_ctx* c, bool pdl, cudaStream_t s, const HierDev& H, const PairXf* xf,
                     const int4* in, int level, int4* sweep, unsigned long long* cnt,
                     unsigned long long* status, int64_t cap_level, int64_t cap_sweep, int items) {
  launch_pdl(pdl, k_expand<W>, one_wave(c, k_expand<W>, W * 32, 0), W * 32, s, H, xf, in, level,
             sweep, cnt, status, cap_level, cap_sweep, items);
}
static void launch_expand(mrdem_ctx* c, const Shape& sh, bool pdl, cudaStream_t s, const HierDev& H,
                          const PairXf* xf, const int4* in, int level, int4* sweep,
                          unsigned long long* cnt, unsigned long long* status, int64_t cap_level,
                          int64_t cap_sweep) {
  if (sh.level_warps == 2) expand_w<2>(c, pdl, s, H, xf, in, level, sweep, cnt, status, cap_level, cap_sweep, sh.expand_items);
  else if (sh.level_warps == 4) expand_w<4>(c, pdl, s, H, xf, in, level, sweep, cnt, status, cap_level, cap_sweep, sh.expand_items);
  else expand_w<8>(c, pdl, s, H, xf, in, level, sweep, cnt, status, cap_level, cap_sweep, sh.expand_items);
}
template <int W>
static void tile_w(mrdem_ctx* c, bool pdl, cudaStream_t s, const HierDev& H, const PairXf* xf,
                   const TileItem* tiles, int4* fine, unsigned long long* cnt,
                   unsigned long long* status, int64_t cap_tiles, int64_t cap_fine) {
  launch_pdl(pdl, k_tile<W>, one_wave(c, k_tile<W>, W * 32, 0), W * 32, s, H, xf, tiles, fine, cnt,
             status, cap_tiles, cap_fine);
}
static void launch_tile(mrdem_ctx* c, const Shape& sh, bool pdl, cudaStream_t s, const HierDev& H,
                        const PairXf* xf, const TileItem* tiles, int4* fine,
                        unsigned long long* cnt, unsigned long long* status, int64_t cap_tiles,
                        int64_t cap_fine) {
  if (sh.tile_warps == 2) tile_w<2>(c, pdl, s, H, xf, tiles, fine, cnt, status, cap_tiles, cap_fine);
  else if (sh.tile_warps == 4) tile_w<4>(c, pdl, s, H, xf, tiles, fine, cnt, status, cap_tiles, cap_fine);
  else tile_w<8>(c, pdl, s, H, xf, tiles, fine, cnt, status, cap_tiles, cap_fine);
}
template <int W>
static void sweep_fine_w(mrdem_ctx* c, bool pdl, cudaStream_t s, const HierDev& H,
                         const PairXf* xf, SweepConst sc, float conv_c, const int4* fine,
                         int3* cands, unsigned long long* cnt, unsigned long long* status,
                         int64_t cap_fine, int64_t cap_cands, const double* eps) {
  launch_pdl(pdl, k_sweep_fine<W, true>, one_wave(c, k_sweep_fine<W, true>, W * 32, 0), W * 32, s,
             H, xf, sc, conv_c, fine, cands, cnt, status, cap_fine, cap_cands, eps);
}
static void launch_sweep_fine(mrdem_ctx* c, const Shape& sh, bool pdl, cudaStream_t s,
                              const HierDev& H, const PairXf* xf, SweepConst sc, float conv_c,
                              const int4* fine, int3* cands, unsigned long long* cnt,
                              unsigned long long* status, int64_t cap_fine, int64_t cap_cands,
                              const double* eps) {
  if (sh.sweep_warps == 2) sweep_fine_w<2>(c, pdl, s, H, xf, sc, conv_c, fine, cands, cnt, status, cap_fine, cap_cands, eps);
  else if (sh.sweep_warps == 8) sweep_fine_w<8>(c, pdl, s, H, xf, sc, conv_c, fine, cands, cnt, status, cap_fine, cap_cands, eps);
  else sweep_fine_w<4>(c, pdl, s, H, xf, sc, conv_c, fine, cands, cnt, status, cap_fine, cap_cands, eps);
}
static void launch_sweep_nodes(mrdem_ctx* c, const Shape& sh, bool pdl, cudaStream_t s,
                               const HierDev& H, const PairXf* xf, SweepConst sc, const int4* sweep,
                               int level, int4* out, TileItem* tiles, unsigned long long* cnt,
                               unsigned long long* status, int64_t cap_sweep, int64_t cap_level,
                               int64_t cap_tiles) {
  const int t = sh.node_threads;
  launch_pdl(pdl, k_sweep_nodes, one_wave(c, k_sweep_nodes, t, 0), t, s, H, xf, sc, sweep, level,
             out, tiles, cnt, status, cap_sweep, cap_level, cap_tiles);
}
template <int W>
static void level_w(mrdem_ctx* c, bool pdl, cudaStream_t s, const HierDev& H, const PairXf* xf,
                    SweepConst sc, const int4* in, int level, int4* out, TileItem* tiles,
                    unsigned long long* cnt, unsigned long long* status, int64_t cap_level,
                    int64_t cap_tiles, int items) {
  launch_pdl(pdl, k_level<W>, one_wave(c, k_level<W>, W * 32, 0), W * 32, s, H, xf, sc, in, level,
             out, tiles, cnt, status, cap_level, cap_tiles, items);
}
// One surrogate level in one launch (k_level, level_kernel 2), with the
// k_expand shape's warps per block and items per warp.
static void launch_level_fused(mrdem_ctx* c, const Shape& sh, bool pdl, cudaStream_t s,
                               const HierDev& H, const PairXf* xf, SweepConst sc, const int4* in,
                               int level, int4* out, TileItem* tiles, unsigned long long* cnt,
                               unsigned long long* status, int64_t cap_level, int64_t cap_tiles) {
  if (sh.level_warps == 2) level_w<2>(c, pdl, s, H, xf, sc, in, level, out, tiles, cnt, status, cap_level, cap_tiles, sh.expand_items);
  else if (sh.level_warps == 4) level_w<4>(c, pdl, s, H, xf, sc, in, level, out, tiles, cnt, status, cap_level, cap_tiles, sh.expand_items);
  else level_w<8>(c, pdl, s, H, xf, sc, in, level, out, tiles, cnt, status, cap_level, cap_tiles, sh.expand_items);
}
// All surrogate levels in one cooperative launch (k_levels) on a one-wave
// grid: every block is resident, as the grid-wide barriers require.
static int launch_levels_coop(mrdem_ctx* c, cudaStream_t s, const HierDev& H, SweepConst sc,
                              int steps, int max_items) {
  const int grid = one_wave(c, k_levels, kLevelWarps * 32, 0);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kLevelWarps * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_levels, H, (const PairXf*)c->xf, sc,
                                           c->level_list[0], c->level_list[1], c->sweep, c->tiles,
                                           c->counters, c->status, c->cap_level, c->cap_sweep,
                                           c->cap_tiles, steps, max_items);
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}
// k_exact64 grid: 8 blocks per SM at 128 threads, the same threads per SM
// otherwise.
static int exact_blocks(const mrdem_ctx* c, int threads, int per_sm_128) {
  return c->n_sms * per_sm_128 * 128 / threads;
}

SweepConst sweep_const(const mrdem_params& p) {
  SweepConst sc;
  sc.rho_reg = p.rho_reg;
  sc.rho_iter = p.rho_iter;
  sc.n_iter = p.n_iter;
  return sc;
}

// ---------------------------------------------------------------------------
// Contacts ordered by pair: detection writes its contacts to a scratch list
// in whatever order the warps finish, counting them per pair as it goes; a
// counting sort over the pair index (exclusive scan, scatter) then writes
// them to the caller's buffers
// grouped by pair, pairs in increasing order (within a pair the order is
// not fixed).  The per-pair sums of forces and the adjoint then meet one or
// two pairs per warp instead of several.
// Exclusive scan of the per-pair counts in place, one block.
__global__ void __launch_bounds__(1024) k_sort_scan(int32_t* pair_cnt, int64_t n_pairs) {
  wait_prior_grid();
  block_exclusive_scan(pair_cnt, n_pairs, nullptr);
}

__global__ void __launch_bounds__(256) k_sort_scatter(mrdem_contacts tmp, int32_t* pair_cnt,
                                                      mrdem_contacts out) {
  wait_prior_grid();
  int64_t n = *tmp.count;
  if (blockIdx.x == 0 && threadIdx.x == 0) *out.count = n;
  if (n > tmp.capacity) n = tmp.capacity;
  const int lane = lane_id();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t k = base + threadIdx.x;
    const bool in = k < n;
    const int p = in ? tmp.pair[k] : -1;
    // the lanes holding one pair (a warp's contacts mostly share one) take
    // their slots with one atomic
    const unsigned grp = __match_any_sync(0xffffffffu, p);
    const int leader = __ffs(grp) - 1;
    int j0 = 0;
    if (in && lane == leader) j0 = atomicAdd(pair_cnt + p, __popc(grp));
    j0 = __shfl_sync(0xffffffffu, j0, leader);
    const int64_t j = (int64_t)j0 + __popc(grp & ((1u << lane) - 1u));
    if (!in || j >= out.capacity) continue;
    out.pair[j] = p;
    out.tri_a[j] = tmp.tri_a[k];
    out.tri_b[j] = tmp.tri_b[k];
    out.dist[j] = tmp.dist[k];
    for (int q = 0; q < 3; ++q) {
      out.point_a[3 * j + q] = tmp.point_a[3 * k + q];
      out.point_b[3 * j + q] = tmp.point_b[3 * k + q];
    }
  }
}

// Scratch contact list with the caller's capacity.
int ensure_tmp(mrdem_ctx* c, int64_t cap, mrdem_contacts* tmp) {
  if (cap > c->cap_tmp || !c->tmp_count) {
    cudaFree(c->tmp_i);
    cudaFree(c->tmp_d);
    if (!c->tmp_count && cudaMalloc(&c->tmp_count, sizeof(int64_t)) != cudaSuccess) {
      cudaGetLastError();
      return MRDEM_ERR_OOM;
    }
    c->tmp_i = nullptr;
    c->tmp_d = nullptr;
    c->cap_tmp = 0;
    const int64_t n = cap > 0 ? cap : 1;
    if (cudaMalloc(&c->tmp_i, sizeof(int32_t) * 3 * n) != cudaSuccess ||
        cudaMalloc(&c->tmp_d, sizeof(double) * 7 * n) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(c->tmp_i);
      c->tmp_i = nullptr;
      return MRDEM_ERR_OOM;
    }
    c->cap_tmp = n;
  }
  tmp->capacity = cap;
  tmp->count = c->tmp_count;
  tmp->pair = c->tmp_i;
  tmp->tri_a = c->tmp_i + c->cap_tmp;
  tmp->tri_b = c->tmp_i + 2 * c->cap_tmp;
  tmp->dist = c->tmp_d;
  tmp->point_a = c->tmp_d + c->cap_tmp;
  tmp->point_b = c->tmp_d + 4 * c->cap_tmp;
  return MRDEM_OK;
}

static int finish(cudaStream_t) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

// The pairs' transforms alone (no root test): float, FP64 and double-float.
int launch_setup_transforms(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs,
                            const int32_t* ab, const double* eps, const double* poses,
                            cudaStream_t s) {
  if (n_pairs <= 0) return MRDEM_OK;
  const int threads = 32;
  const int blocks = (int)std::min<int64_t>((n_pairs + threads - 1) / threads, (int64_t)c->n_sms * 64);
  ProfScope ps(c, K_SETUP, s);
  k_setup<<<blocks, threads, 0, s>>>(hier->dev, (int)n_pairs, ab, eps, poses, c->xf, c->xf64,
                                     c->xfdd, sweep_const(c->params), 0, c->level_list[0],
                                     c->tiles, c->counters, c->status, c->cap_level, c->cap_tiles);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

// The finest-level stage and what follows it, on the leaf-pair tiles listed
// in c->tiles (counter CNT_TILES): fine-vs-surrogate and sphere culls, the
// fine sweeps, the exact distance into tmp, and the contacts grouped by pair
// into out (pair_cnt holds each pair's count).
int launch_fine_tail(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const double* eps,
                     int precision, const mrdem_contacts* tmp, const mrdem_contacts* out,
                     const Shape& sh, cudaStream_t s) {
  const HierDev& H = hier->dev;
  const mrdem_params& prm = c->params;
  SweepConst sc = sweep_const(prm);
  {
    ProfScope ps(c, K_TILE, s);
    launch_tile(c, sh, true, s, H, c->xf, c->tiles, c->sweep, c->counters, c->status,
                c->cap_tiles, c->cap_sweep);
  }
  {
    ProfScope ps(c, K_SWEEP_FINE, s);
    launch_sweep_fine(c, sh, true, s, H, c->xf, sc, prm.conv_c, c->sweep, c->cands, c->counters,
                      c->status, c->cap_sweep, c->cap_cands, eps);
  }
  const int et = sh.exact_threads;
  if (precision == MRDEM_PREC_FP64) {
    ProfScope ps(c, K_EXACT, s);
    launch_after(k_exact64, exact_blocks(c, et, 8), et, 0, s, H, c->xf64, c->cands, c->counters,
                 (int)CNT_CANDS, c->cap_cands, c->status, (int)MRDEM_STAT_FP64, *tmp,
                 c->pair_cnt);
  } else {
    int r = launch_exact_fp32(c, hier, tmp, et, s);
    if (r) return r;
  }
  // the contacts, grouped by pair, into the caller's buffers
  {
    ProfScope ps(c, K_SORT, s);
    const int sb = c->n_sms * 4;
    launch_after(k_sort_scan, 1, 1024, 0, s, c->pair_cnt, n_pairs);
    launch_after(k_sort_scatter, sb, 256, 0, s, *tmp, c->pair_cnt, *out);
  }
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_detect(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                  const double* eps, const double* poses, int precision, const mrdem_contacts* out,
                  int64_t* stats, cudaStream_t s) {
  int st = ensure_pairs(c, n_pairs);
  if (st) return st;
  mrdem_contacts tmp;
  st = ensure_tmp(c, out->capacity, &tmp);
  if (st) return st;
  const HierDev& H = hier->dev;
  const mrdem_params& prm = c->params;
  SweepConst sc = sweep_const(prm);
  cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * CNT_TOTAL, s);
  cudaMemsetAsync(out->count, 0, sizeof(int64_t), s);
  cudaMemsetAsync(tmp.count, 0, sizeof(int64_t), s);
  if (n_pairs > 0) cudaMemsetAsync(c->pair_cnt, 0, sizeof(int32_t) * n_pairs, s);
  if (n_pairs > 0) {
    // one warp per block: the FP64 setup work spreads over every SM
    int threads = 32;
    int blocks = (int)std::min<int64_t>((n_pairs + threads - 1) / threads, (int64_t)c->n_sms * 64);
    {
      ProfScope ps(c, K_SETUP, s);
      k_setup<<<blocks, threads, 0, s>>>(H, (int)n_pairs, ab, eps, poses, c->xf, c->xf64, c->xfdd,
                                         sc, 1,
                                         c->level_list[0], c->tiles, c->counters, c->status,
                                         c->cap_level, c->cap_tiles);
    }
    int steps = std::min(hier->h.max_depth - 1, kMaxLevels - 1);
    const Shape sh = shape_for(c, n_pairs);
    if (sh.level_kernel == 1 && steps > 0) {
      ProfScope ps(c, K_LEVEL, s);
      int r = launch_levels_coop(c, s, H, sc, steps, sh.expand_items);
      if (r) return r;
    }
    for (int l = 0; l < steps && sh.level_kernel != 1; ++l) {
      if (sh.level_kernel == 2) {
        ProfScope ps(c, K_LEVEL, s);
        launch_level_fused(c, sh, true, s, H, c->xf, sc, c->level_list[l & 1], l,
                           c->level_list[(l + 1) & 1], c->tiles, c->counters, c->status,
                           c->cap_level, c->cap_tiles);
        continue;
      }
      {
        ProfScope ps(c, K_LEVEL, s);
        launch_expand(c, sh, true, s, H, c->xf, c->level_list[l & 1], l, c->sweep, c->counters,
                      c->status, c->cap_level, c->cap_sweep);
      }
      ProfScope ps(c, K_SWEEP_NODES, s);
      launch_sweep_nodes(c, sh, true, s, H, c->xf, sc, c->sweep, l, c->level_list[(l + 1) & 1],
                         c->tiles, c->counters, c->status, c->cap_sweep, c->cap_level,
                         c->cap_tiles);
    }
    int r = launch_fine_tail(c, hier, n_pairs, eps, precision, &tmp, out, sh, s);
    if (r) return r;
  }
  if (stats)
    cudaMemcpyAsync(stats, c->counters + CNT_STATS, sizeof(int64_t) * MRDEM_STAT_COUNT,
                    cudaMemcpyDeviceToDevice, s);
  return finish(s);
}

// ---------------------------------------------------------------------------
// Autotuner: times the detection kernels under candidate launch shapes on the
// caller's workload and keeps the fastest shape of each kernel for the call's
// size class.  Nine shapes are run: every (k_expand warps, items per warp)
// combination once, and the other kernels' values spread over the nine so
// that each value is timed three or more times (the kernels run one after
// another on lists of the same content whatever the shapes, so each kernel's
// time depends on its own shape only).  Each shape runs reps + 1 times, the
// first untimed; kernels are timed by the context's event pairs.  The
// combined shape is then timed as a whole against the same shape with the
// levels in one cooperative launch and with one launch per level at each
// block size, and the fastest is kept.
int autotune(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
             const double* eps, const double* poses, int precision, const mrdem_contacts* out,
             int reps, int32_t* chosen, double* ms) {
  static const int LW[3] = {2, 4, 8}, EI[3] = {8, 16, 32}, NT[2] = {128, 256};
  static const int TW[3] = {2, 4, 8}, SW[3] = {2, 4, 8}, ET[3] = {64, 128, 256};
  if (cudaDeviceSynchronize() != cudaSuccess) return MRDEM_ERR_CUDA;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  const mrdem_params& p = c->params;
  const Shape base = {p.level_warps, p.expand_items, p.node_threads, p.tile_warps, p.sweep_warps,
                      p.exact_threads, p.level_kernel};
  double t_exp[3][3] = {}, t_nodes[2] = {}, t_tile[3] = {}, t_sweep[3] = {}, t_exact[3] = {};
  int n_exp[3][3] = {}, n_nodes[2] = {}, n_tile[3] = {}, n_sweep[3] = {}, n_exact[3] = {};
  const bool prof_was = c->prof;
  std::vector<ProfRec> saved;
  saved.swap(c->prof_recs);
  int st = MRDEM_OK;
  // one timed run of `reps` detections under shape sh: per-kernel sums
  auto run = [&](const Shape& sh, double* per_kernel, double* total) -> int {
    c->force_shape = &sh;
    int r = launch_detect(c, hier, n_pairs, ab, eps, poses, precision, out, nullptr, s);  // untimed
    cudaEvent_t a = nullptr, b = nullptr;
    if (r == MRDEM_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
      r = MRDEM_ERR_CUDA;
    c->prof = per_kernel != nullptr;
    if (r == MRDEM_OK) cudaEventRecord(a, s);
    for (int k = 0; k < reps && r == MRDEM_OK; ++k)
      r = launch_detect(c, hier, n_pairs, ab, eps, poses, precision, out, nullptr, s);
    if (r == MRDEM_OK) cudaEventRecord(b, s);
    c->prof = false;
    c->force_shape = nullptr;
    if (cudaStreamSynchronize(s) != cudaSuccess) r = MRDEM_ERR_CUDA;
    if (r == MRDEM_OK) {
      float t = 0.f;
      cudaEventElapsedTime(&t, a, b);
      *total = t / reps;
    }
    for (auto& rec : c->prof_recs) {
      float t = 0.f;
      if (r == MRDEM_OK && cudaEventElapsedTime(&t, rec.a, rec.b) == cudaSuccess && per_kernel)
        per_kernel[rec.kernel] += t / reps;
      c->ev_pool.push_back(rec.a);
      c->ev_pool.push_back(rec.b);
    }
    c->prof_recs.clear();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    // a list that overflowed makes the timings meaningless: report it (the
    // status stays latched for mrdem_check)
    unsigned long long h[ST_TOTAL] = {};
    if (r == MRDEM_OK &&
        cudaMemcpy(h, c->status, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) {
      for (int k = ST_REQ_LEVEL; k < ST_TOTAL; ++k)
        if (h[k]) r = MRDEM_ERR_CAPACITY;
      if (h[ST_NONFINITE]) r = MRDEM_ERR_NONFINITE;
    }
    if (cudaGetLastError() != cudaSuccess && r == MRDEM_OK) r = MRDEM_ERR_CUDA;
    return r;
  };
  for (int i = 0; i < 9 && st == MRDEM_OK; ++i) {
    const int e = i % 3, f = i / 3, g = (i + 1) % 3, q = (i + 2) % 3, x = (i + i / 3) % 3;
    const Shape sh = {LW[e], EI[f], NT[i % 2], TW[g], SW[q], ET[x], 0};
    double kt[K_COUNT] = {}, tot = 0.0;
    st = run(sh, kt, &tot);
    if (st != MRDEM_OK) break;
    t_exp[e][f] += kt[K_LEVEL];
    ++n_exp[e][f];
    t_nodes[i % 2] += kt[K_SWEEP_NODES];
    ++n_nodes[i % 2];
    t_tile[g] += kt[K_TILE];
    ++n_tile[g];
    t_sweep[q] += kt[K_SWEEP_FINE];
    ++n_sweep[q];
    t_exact[x] += kt[K_EXACT];
    ++n_exact[x];
  }
  Shape best = base;
  if (st == MRDEM_OK) {
    auto argmin = [](const double* t, const int* n, int m) {
      int k = 0;
      for (int j = 1; j < m; ++j)
        if (n[j] && (!n[k] || t[j] / n[j] < t[k] / n[k])) k = j;
      return k;
    };
    int be = 0, bf = 0;
    for (int e = 0; e < 3; ++e)
      for (int f = 0; f < 3; ++f)
        if (n_exp[e][f] && t_exp[e][f] / n_exp[e][f] < t_exp[be][bf] / n_exp[be][bf]) {
          be = e;
          bf = f;
        }
    best = {LW[be], EI[bf], NT[argmin(t_nodes, n_nodes, 2)], TW[argmin(t_tile, n_tile, 3)],
            SW[argmin(t_sweep, n_sweep, 3)], ET[argmin(t_exact, n_exact, 3)], 0};
    double t_base = 0.0, t_best = 0.0, t_coop = 0.0;
    st = run(base, nullptr, &t_base);
    if (st == MRDEM_OK) st = run(best, nullptr, &t_best);
    // the same shape with every surrogate level in one cooperative launch
    Shape coop = best;
    coop.level_kernel = 1;
    if (st == MRDEM_OK) st = run(coop, nullptr, &t_coop);
    if (st == MRDEM_OK && t_coop < t_best) {
      best = coop;
      t_best = t_coop;
    }
    // and with each level's two phases in one launch (k_level), whose
    // register use differs from k_expand's: each of its block sizes
    for (int e = 0; e < 3 && st == MRDEM_OK; ++e) {
      Shape fused = coop;
      fused.level_kernel = 2;
      fused.level_warps = LW[e];
      double t_fused = 0.0;
      st = run(fused, nullptr, &t_fused);
      if (st == MRDEM_OK && t_fused < t_best) {
        best = fused;
        t_best = t_fused;
      }
    }
    if (st == MRDEM_OK) {
      const int k = size_class(n_pairs);
      c->tuned[k] = best;
      c->tuned_ok[k] = true;
      if (ms) {
        ms[0] = t_base;
        ms[1] = t_best;
      }
      if (chosen) {
        chosen[0] = best.level_warps;
        chosen[1] = best.expand_items;
        chosen[2] = best.node_threads;
        chosen[3] = best.tile_warps;
        chosen[4] = best.sweep_warps;
        chosen[5] = best.exact_threads;
        chosen[6] = best.level_kernel;
      }
    }
  }
  c->prof = prof_was;
  c->prof_recs.swap(saved);
  cudaStreamDestroy(s);
  return st;
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
  int threads = 32;
  int blocks = (int)((n_pairs + threads - 1) / threads);
  k_setup<<<blocks, threads, 0, s>>>(H, (int)n_pairs, ab, eps, poses, c->xf, c->xf64, nullptr,
                                     sc, 0,
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
    const int pt = 256;
    int64_t blocks2 = std::min<int64_t>((total + pt - 1) / pt, (int64_t)c->n_sms * 64);
    ProfScope ps(c, K_PLAIN, s);
    k_plain<<<(int)blocks2, pt, 0, s>>>(H, c->xf64, (int)p, na, nb, c->status, *out);
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

// ---------------------------------------------------------------------------
// Detection without allocation.  All work lists of one call live in a fixed
// file-scope device array, so the call needs no device memory beyond its
// inputs and outputs.  Limits (each fixed list; the call reports an overflow
// in its statistics and the result is then incomplete):
namespace {
constexpr int64_t kNaPairs = 1024;       // particle pairs per call
constexpr int64_t kNaLevel = 1 << 16;    // node-pair items per level
constexpr int64_t kNaTiles = 1 << 16;    // leaf-pair tiles
constexpr int64_t kNaSweep = 1 << 17;    // pairs waiting for a sweep
constexpr int64_t kNaCands = 1 << 16;    // fine candidates
constexpr size_t na_align(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNaOffCnt = 0;
constexpr size_t kNaOffSt = na_align(kNaOffCnt + sizeof(unsigned long long) * mrdem::CNT_TOTAL);
constexpr size_t kNaOffXf = na_align(kNaOffSt + sizeof(unsigned long long) * mrdem::ST_TOTAL);
constexpr size_t kNaOffXf64 = na_align(kNaOffXf + sizeof(mrdem::PairXf) * kNaPairs);
constexpr size_t kNaOffL0 = na_align(kNaOffXf64 + sizeof(mrdem::PairXf64) * kNaPairs);
constexpr size_t kNaOffL1 = na_align(kNaOffL0 + sizeof(int4) * kNaLevel);
constexpr size_t kNaOffTiles = na_align(kNaOffL1 + sizeof(int4) * kNaLevel);
constexpr size_t kNaOffSweep = na_align(kNaOffTiles + sizeof(mrdem::TileItem) * kNaTiles);
constexpr size_t kNaOffCands = na_align(kNaOffSweep + sizeof(int4) * kNaSweep);
constexpr size_t kNaBytes = na_align(kNaOffCands + sizeof(int3) * kNaCands);  // about 7.2 MB
}  // namespace

// The scratch itself: every GPU that loads this library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

namespace mrdem {
namespace {

// Device address of the scratch array, looked up once per device (host code
// cannot use the symbol itself as a device pointer).
std::mutex g_na_mutex;
void* g_na_addr[256] = {nullptr};

int noalloc_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= 256) return MRDEM_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MRDEM_ERR_CUDA;
    }
    g_na_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_na_addr[device]);
  return MRDEM_OK;
}

// Copies the overflow and invalid-input flags of the call into its statistics.
__global__ void k_noalloc_status(const unsigned long long* status, int64_t* stats) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long req = 0;
    for (int k = ST_REQ_LEVEL; k <= ST_REQ_SWEEP; ++k) req = req > status[k] ? req : status[k];
    stats[MRDEM_STAT_NOALLOC_OVERFLOW] = (int64_t)req;
    stats[MRDEM_STAT_NOALLOC_INVALID] = (int64_t)status[ST_NONFINITE];
  }
}

}  // namespace
}  // namespace mrdem

extern "C" int mrdem_detect_noalloc(const mrdem_hier* hier, int64_t n_pairs,
                                    const int32_t* pair_ab, const double* pair_eps,
                                    const double* poses, int32_t precision,
                                    const mrdem_contacts* out, int64_t* stats,
                                    mrdem_stream stream) {
  using namespace mrdem;
  if (!hier || !hier->d_mem || !hier->ctx || !out || !out->count || !stats) return MRDEM_ERR_INVALID;
  if (n_pairs < 0 || n_pairs > kNaPairs) return MRDEM_ERR_INVALID;
  if (n_pairs > 0 && (!pair_ab || !pair_eps || !poses)) return MRDEM_ERR_INVALID;
  if (out->capacity < 0 ||
      (out->capacity > 0 && (!out->pair || !out->tri_a || !out->tri_b || !out->dist ||
                             !out->point_a || !out->point_b)))
    return MRDEM_ERR_INVALID;
  if (precision != MRDEM_PREC_FP32 && precision != MRDEM_PREC_FP64) return MRDEM_ERR_INVALID;
  mrdem_ctx* c = hier->ctx;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  int st = noalloc_scratch(c->device, &base);
  if (st != MRDEM_OK) {
    if (prev >= 0) cudaSetDevice(prev);
    return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + kNaOffCnt);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(base + kNaOffSt);
  PairXf* xf = reinterpret_cast<PairXf*>(base + kNaOffXf);
  PairXf64* xf64 = reinterpret_cast<PairXf64*>(base + kNaOffXf64);
  int4* lists[2] = {reinterpret_cast<int4*>(base + kNaOffL0), reinterpret_cast<int4*>(base + kNaOffL1)};
  TileItem* tiles = reinterpret_cast<TileItem*>(base + kNaOffTiles);
  int4* sweep = reinterpret_cast<int4*>(base + kNaOffSweep);
  int3* cands = reinterpret_cast<int3*>(base + kNaOffCands);
  const HierDev& H = hier->dev;
  const mrdem_params& prm = c->params;
  SweepConst sc = sweep_const(prm);
  // the array keeps the previous call's contents: clear what starts at zero
  cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * CNT_TOTAL, s);
  cudaMemsetAsync(status, 0, sizeof(unsigned long long) * ST_TOTAL, s);
  cudaMemsetAsync(out->count, 0, sizeof(int64_t), s);
  if (n_pairs > 0) {
    int threads = 32;
    int blocks = (int)std::min<int64_t>((n_pairs + threads - 1) / threads, (int64_t)c->n_sms * 64);
    k_setup<<<blocks, threads, 0, s>>>(H, (int)n_pairs, pair_ab, pair_eps, poses, xf, xf64, nullptr,
                                       sc, 1,
                                       lists[0], tiles, cnt, status, kNaLevel, kNaTiles);
    int steps = std::min(hier->h.max_depth - 1, kMaxLevels - 1);
    const Shape sh = shape_for(c, n_pairs);
    for (int l = 0; l < steps; ++l) {
      launch_expand(c, sh, false, s, H, xf, lists[l & 1], l, sweep, cnt, status, kNaLevel, kNaSweep);
      launch_sweep_nodes(c, sh, false, s, H, xf, sc, sweep, l, lists[(l + 1) & 1], tiles, cnt,
                         status, kNaSweep, kNaLevel, kNaTiles);
    }
    launch_tile(c, sh, false, s, H, xf, tiles, sweep, cnt, status, kNaTiles, kNaSweep);
    launch_sweep_fine(c, sh, false, s, H, xf, sc, prm.conv_c, sweep, cands, cnt, status, kNaSweep,
                      kNaCands, pair_eps);
    const int et = sh.exact_threads;
    if (precision == MRDEM_PREC_FP64) {
      k_exact64<<<exact_blocks(c, et, 8), et, 0, s>>>(H, xf64, cands, cnt, CNT_CANDS, kNaCands,
                                                       status, MRDEM_STAT_FP64, *out, nullptr);
    } else {
      // the first level list is free once the tiles are done: the fallback list
      k_exact32<<<exact_blocks(c, et, 8), et, 0, s>>>(H, xf, xf64, cands, cnt, status, kNaCands,
                                                       reinterpret_cast<int3*>(lists[0]), kNaLevel,
                                                       *out);
      k_exact64<<<exact_blocks(c, et, 4), et, 0, s>>>(H, xf64,
                                                       reinterpret_cast<const int3*>(lists[0]), cnt,
                                                       CNT_FALLBACK, kNaLevel, status,
                                                       MRDEM_STAT_FP64, *out, nullptr);
    }
  }
  cudaMemcpyAsync(stats, cnt + CNT_STATS, sizeof(int64_t) * MRDEM_STAT_COUNT,
                  cudaMemcpyDeviceToDevice, s);
  k_noalloc_status<<<1, 32, 0, s>>>(status, stats);
  cudaError_t e = cudaGetLastError();
  if (prev >= 0) cudaSetDevice(prev);
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}
