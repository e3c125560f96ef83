// mrdem_frontier.cu -- the active sets of the multiresolution implicit Euler
// step (Algorithm 6 of Noble & Weinzierl, arXiv 2105.12415) on the GPU.
//
// Per particle pair the active set is a cut through the product of the two
// surrogate trees: node pairs such that every pair of fine triangles lies
// below exactly one, kept across the Picard iterations in depth-first order
// of the product tree (a pair's children side by side, A's child index
// major; a leaf side stays while the other unfolds, as in Algorithm 5).  One
// call tests every item at the iteration's poses and writes the next sets:
//   k_setup      the pairs' transforms (mrdem_detect.cu);
//   k_as_test    per item, in stages joined by per-warp queues: the
//                certified tests of a surrogate level (node spheres,
//                oriented boxes, the float penalty sweep with its
//                certificate and the face normals) against
//                delta_a + delta_b + 2 eps.  Apart: bottom.  Otherwise a pair
//                of leaves goes to the tile list of the finest-level stage,
//                any other pair is widened (its output count is its number
//                of children) and, when the sweep converged within that
//                threshold, is a surrogate contact (the implicit guess);
//   k_as_narrow  one thread per item: the first child of a group (child
//                index 0 of its parent pair) checks that the group's last
//                child sits where a complete group ends and that every
//                member's status byte says bottom and not vetoed; then it
//                emits the parent and the others nothing (narrowing);
//   k_as_scan_*  the output offsets, in input order, so the next sets stay
//                in depth-first order (chunk sums, their scan, chunk rescans);
//   k_as_emit    one thread per item: its output items;
//   the finest-level stage of mrdem_detect on the tile list (fine culls,
//   fine sweeps, exact distance, contacts grouped by pair).
// The memory set U of the paper is kept as two flags per item: bit 1 on a
// pair made by narrowing, bit 0 on the children of a widened item that
// carried either bit; a group with a bit-0 member is never narrowed.
#include <cuda_runtime.h>

#include <algorithm>

#include "mrdem_device.cuh"

namespace mrdem {
namespace {

constexpr int kAsThreads = 256;
constexpr int32_t kVeto = 1, kNarrowed = 2;
enum : int8_t { AS_BOT = 0, AS_LEAF = 1, AS_WIDEN = 2, AS_PARENT = 3, AS_MERGED = 4 };
// Added by k_as_test to the outcome of an item that may not be narrowed (a
// vetoed item, or one that is not a valid node pair), so that k_as_narrow
// reads a group's eligibility from its status bytes alone.
constexpr int8_t AS_KEEP = 0x10;

using F3 = V3<float>;
using D3 = V3<double>;

// The child set of node v as one side of a pair: (first child, count), or
// v itself when v is a leaf.
__device__ __forceinline__ int2 side_of(const HierDev& H, int v) {
  const int2 c = __ldg(H.node_child + v);
  return c.y > 0 ? c : make_int2(v, 1);
}
// The pair whose unfolding listed (a, b): the side(s) on the deeper level
// came from their parents, a shallower side (a leaf) stayed.  False for a
// pair of roots.
__device__ __forceinline__ bool parent_pair(const HierDev& H, int a, int b, int& pa, int& pb) {
  const int2 ua = __ldg(H.node_up + a), ub = __ldg(H.node_up + b);
  const int k = max(ua.y, ub.y);
  pa = ua.y == k ? ua.x : a;
  pb = ub.y == k ? ub.x : b;
  return pa >= 0 && pb >= 0;
}
// Position of (a, b) among the children of (pa, pb), and their number.
__device__ __forceinline__ int child_index(const HierDev& H, int a, int b, int pa, int pb,
                                           int* size) {
  const int2 sa = side_of(H, pa), sb = side_of(H, pb);
  *size = sa.y * sb.y;
  return (a - sa.x) * sb.y + (b - sb.x);
}
__device__ __forceinline__ bool item_ok(const HierDev& H, int4 it, int64_t n_pairs) {
  return it.x >= 0 && it.x < n_pairs && it.y >= 0 && it.z >= 0 && it.y < H.n_nodes &&
         it.z < H.n_nodes;
}
__device__ __forceinline__ int64_t clamp_count(const mrdem_active_set& s) {
  const int64_t n = *s.count;
  return n < s.capacity ? n : s.capacity;
}

// Append a surrogate contact (warp-collective): pair, the two node indices,
// distance and world points.
__device__ __forceinline__ void write_surrogate(const mrdem_contacts& out,
                                                unsigned long long* status, bool hit, int pair,
                                                int a, int b, double d, D3 pa, D3 pb) {
  const unsigned m = __ballot_sync(0xffffffffu, hit);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if ((int)lane_id() == leader)
    base = atomicAdd((unsigned long long*)out.count, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (!hit) return;
  const unsigned long long idx = base + __popc(m & ((1u << lane_id()) - 1u));
  if ((int64_t)idx < out.capacity) {
    out.pair[idx] = pair;
    out.tri_a[idx] = a;
    out.tri_b[idx] = b;
    out.dist[idx] = d;
    out.point_a[3 * idx] = pa.x; out.point_a[3 * idx + 1] = pa.y; out.point_a[3 * idx + 2] = pa.z;
    out.point_b[3 * idx] = pb.x; out.point_b[3 * idx + 1] = pb.y; out.point_b[3 * idx + 2] = pb.z;
  } else {
    atomicMax(status + ST_REQ_CONTACTS, idx + 1);
  }
}

__global__ void __launch_bounds__(kAsThreads) k_as_init(HierDev H, int64_t n_pairs,
                                                        const int32_t* __restrict__ ab,
                                                        mrdem_active_set out) {
  int4* o = reinterpret_cast<int4*>(out.item);
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs; p += step) {
    const int A = ab[2 * p], B = ab[2 * p + 1];
    const bool ok = A >= 0 && B >= 0 && A < H.n_particles && B < H.n_particles;
    o[p] = make_int4((int)p, ok ? H.root[A] : -1, ok ? H.root[B] : -1, 0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *out.count = n_pairs;
}

template <int NIT>
__device__ __forceinline__ float node_sweep(F3 p0, F3 p1, F3 p2, F3 q0, F3 q1, F3 q2,
                                            const SweepConst& sc, float tol2, bool* cv,
                                            float* x) {
  return sweep_certificate<true, NIT>(p0, p1, p2, q0, q1, q2, sc, tol2, cv, x);
}

// k_as_test runs an item's tests in three stages joined by two per-warp
// queues of item indices in shared memory: the node spheres for every
// item; the oriented boxes for the sphere survivors, 32 at a time; the
// float sweep, its certificate, the face normals and the outcome for the box
// survivors, 32 at a time.  So the two costlier tests run on full warps
// instead of on the few lanes of a round whose items survived.
constexpr int kAsQueue = 64;
struct AsQueues {
  int64_t box[kAsQueue];
  int64_t sweep[kAsQueue];
};
struct AsTestArgs {
  HierDev H;
  const PairXf* xf;
  const PairXf64* xf64;
  SweepConst sc;
  float conv_c;
  const double* eps;
  const int4* items;
  int8_t* st;
  int32_t* em;
  TileItem* tiles;
  unsigned long long* cnt;
  unsigned long long* status;
  int64_t cap_tiles;
  mrdem_contacts sur;
};

__device__ __forceinline__ void as_bottom(const AsTestArgs& A, int64_t k, bool keep) {
  A.st[k] = (int8_t)(keep ? AS_BOT | AS_KEEP : AS_BOT);
  A.em[k] = 1;
}
// Queue the lanes with `pred` (warp-collective); n is warp-uniform.
__device__ __forceinline__ void as_push(int64_t* q, int& n, bool pred, int64_t k) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (pred) q[n + __popc(m & ((1u << lane_id()) - 1u))] = k;
  n += __popc(m);
  __syncwarp();
}

// The sweep stage on the last `take` entries of the sweep queue.
__device__ __forceinline__ void as_sweep_stage(const AsTestArgs& A, AsQueues& Q, int& nq,
                                               int take) {
  const int lane = lane_id();
  const bool have = lane < take;
  const int64_t k = have ? Q.sweep[nq - take + lane] : -1;
  __syncwarp();
  nq -= take;
  const HierDev& H = A.H;
  int s = AS_BOT, e = 1;
  int2 ia = make_int2(0, 1), ib = make_int2(0, 1);
  int4 it = make_int4(-1, -1, -1, 0);
  bool hit = false;
  double d = 0.0;
  D3 pw = {0, 0, 0}, qw = {0, 0, 0};
  if (have) {
    it = A.items[k];
    PairXf X;
    load_pairxf(A.xf, it.x, X);
    const int a = it.y, b = it.z;
    const float4 a0 = __ldg(H.node_geo + 3 * a), a1 = __ldg(H.node_geo + 3 * a + 1);
    const float4 a2 = __ldg(H.node_geo + 3 * a + 2);
    const float4 b0 = __ldg(H.node_geo + 3 * b), b1 = __ldg(H.node_geo + 3 * b + 1);
    const float4 b2 = __ldg(H.node_geo + 3 * b + 2);
    const F3 p0 = {a0.x, a0.y, a0.z}, p1 = {a1.x, a1.y, a1.z}, p2 = {a2.x, a2.y, a2.z};
    const F3 q0 = xf_point(X, {b0.x, b0.y, b0.z}), q1 = xf_point(X, {b1.x, b1.y, b1.z});
    const F3 q2 = xf_point(X, {b2.x, b2.y, b2.z});
    const float ce = A.conv_c * (float)__ldg(A.eps + it.x);
    bool cv = false;
    float x[4];
    float gap = A.sc.n_iter == 4 ? node_sweep<4>(p0, p1, p2, q0, q1, q2, A.sc, ce * ce, &cv, x)
                                 : node_sweep<0>(p0, p1, p2, q0, q1, q2, A.sc, ce * ce, &cv, x);
    const float thr = a0.w + b0.w + X.tau + X.margin;
    if (!(gap > thr))
      gap = fmaxf(axis_gap(cross(p1 - p0, p2 - p0), p0, p1, p2, q0, q1, q2),
                  axis_gap(cross(q1 - q0, q2 - q0), p0, p1, p2, q0, q1, q2));
    if (!(gap > thr)) {
      ia = __ldg(H.node_child + a);
      ib = __ldg(H.node_child + b);
      if (ia.y < 0 && ib.y < 0) {
        s = AS_LEAF;
      } else {
        s = AS_WIDEN;
        e = (ia.y > 0 ? ia.y : 1) * (ib.y > 0 ? ib.y : 1);
        // the iterate's points (A's frame): a surrogate contact when the
        // sweep converged within the surrogates' threshold
        const F3 pp = p0 + x[0] * (p1 - p0) + x[1] * (p2 - p0);
        const F3 qq = q0 + x[2] * (q1 - q0) + x[3] * (q2 - q0);
        const F3 r = pp - qq;
        if (cv && sqrtf(dot(r, r)) <= a0.w + b0.w + X.tau) {
          const PairXf64& X64 = A.xf64[it.x];
          pw = xf_point64(X64.RA, X64.tA, D3{(double)pp.x, (double)pp.y, (double)pp.z});
          qw = xf_point64(X64.RA, X64.tA, D3{(double)qq.x, (double)qq.y, (double)qq.z});
          const D3 w = pw - qw;
          d = sqrt(dot(w, w));
          hit = true;
        }
      }
    }
  }
  warp_append(s == AS_LEAF, make_tile(it.x, it.y, it.z, ia, ib), A.tiles, A.cnt + CNT_TILES,
              A.cap_tiles, A.status + ST_REQ_TILES);
  write_surrogate(A.sur, A.status, hit, it.x, it.y, it.z, d, pw, qw);
  if (have) {
    A.st[k] = (int8_t)(s == AS_BOT && (it.w & kVeto) ? AS_BOT | AS_KEEP : s);
    A.em[k] = e;
  }
}

// The box stage on the last `take` entries of the box queue; survivors go
// to the sweep queue, which is drained in full warps.
__device__ __forceinline__ void as_box_stage(const AsTestArgs& A, AsQueues& Q, int& nb, int& ns,
                                             int take) {
  const int lane = lane_id();
  const bool have = lane < take;
  const int64_t k = have ? Q.box[nb - take + lane] : -1;
  __syncwarp();
  nb -= take;
  bool keep = false;
  if (have) {
    const int4 it = A.items[k];
    PairXf X;
    load_pairxf(A.xf, it.x, X);
    const int a = it.y, b = it.z;
    keep = !boxes_apart_w(load_box(A.H, a), __ldg(A.H.node_boxw + a),
                          move_box(X, load_box(A.H, b)), __ldg(A.H.node_boxw + b),
                          X.tau + X.margin);
    if (!keep) as_bottom(A, k, it.w & kVeto);
  }
  as_push(Q.sweep, ns, keep, k);
  if (ns >= 32) as_sweep_stage(A, Q, ns, 32);
}

__global__ void __launch_bounds__(kAsThreads) k_as_test(const __grid_constant__ AsTestArgs A,
                                                        int64_t n_pairs, mrdem_active_set in) {
  wait_prior_grid();
  __shared__ AsQueues queues[kAsThreads / 32];
  AsQueues& Q = queues[threadIdx.x >> 5];
  const HierDev& H = A.H;
  const int64_t n = clamp_count(in);
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int nb = 0, ns = 0;  // queue fill levels (warp-uniform)
  // every lane of a warp runs the same rounds (the stages are warp-collective)
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += step) {
    const int64_t k = base + threadIdx.x;
    bool keep = false;
    if (k < n) {
      const int4 it = A.items[k];
      const bool ok = item_ok(H, it, n_pairs);
      if (ok) {
        PairXf X;
        load_pairxf(A.xf, it.x, X);
        const float4 sa = __ldg(H.node_sph + it.y), sb = __ldg(H.node_sph + it.z);
        const F3 cb = xf_point(X, {sb.x, sb.y, sb.z});
        const float dx = sa.x - cb.x, dy = sa.y - cb.y, dz = sa.z - cb.z;
        const float lim = sa.w + sb.w + X.tau + X.margin;
        keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= lim * lim;
      }
      if (!keep) as_bottom(A, k, !ok || (it.w & kVeto));
    }
    as_push(Q.box, nb, keep, k);
    if (nb >= 32) as_box_stage(A, Q, nb, ns, 32);
  }
  while (nb > 0) as_box_stage(A, Q, nb, ns, nb < 32 ? nb : 32);
  while (ns > 0) as_sweep_stage(A, Q, ns, ns < 32 ? ns : 32);
}

__global__ void __launch_bounds__(kAsThreads) k_as_narrow(HierDev H, int64_t n_pairs,
                                                          mrdem_active_set in, int8_t* st,
                                                          int32_t* em, int64_t* counts) {
  wait_prior_grid();
  const int64_t n = clamp_count(in);
  const int4* items = reinterpret_cast<const int4*>(in.item);
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  WarpCount narrowed;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += step) {
    const int64_t k = base + threadIdx.x;
    bool lead = false;
    // Only the group's first child (child index 0) decides.  The sets are in
    // depth-first order, so when the item size - 1 places further is the
    // same parent's last child, the items between are its other children
    // (each child's part of the cut is one item, the child itself): the
    // group is complete, and it is narrowed when every member is bottom and
    // may be narrowed (status byte AS_BOT exactly).  The leader alone reads
    // and writes its members' bytes.
    if (k < n && st[k] == AS_BOT) {
      const int4 it = items[k];
      int pa, pb, size;
      if (parent_pair(H, it.y, it.z, pa, pb) &&
          child_index(H, it.y, it.z, pa, pb, &size) == 0 && k + size <= n) {
        bool ok = true;
        if (size > 1) {
          const int4 o = items[k + size - 1];
          int qa, qb, sz;
          ok = o.x == it.x && item_ok(H, o, n_pairs) && parent_pair(H, o.y, o.z, qa, qb) &&
               qa == pa && qb == pb && child_index(H, o.y, o.z, pa, pb, &sz) == size - 1;
        }
        for (int j = 1; j < size && ok; ++j) ok = st[k + j] == AS_BOT;
        if (ok) {
          lead = true;
          for (int j = 1; j < size; ++j) {
            st[k + j] = AS_MERGED;
            em[k + j] = 0;
          }
          st[k] = AS_PARENT;
        }
      }
    }
    narrowed.add(lead);
  }
  narrowed.flush(reinterpret_cast<unsigned long long*>(counts + 1));
}

// Output offsets: an exclusive scan of the per-item output counts in place,
// in three passes over a one-wave grid (each block owns one contiguous
// chunk): chunk sums, one block scanning them (and writing the total), then
// each chunk rescanned tile by tile from its offset.  Offsets are stored as
// int32, clamped (an output that large overflows the capacity anyway).
constexpr int kScanMaxBlocks = 1024;
__device__ __forceinline__ void chunk_of(int64_t n, int64_t& b, int64_t& e) {
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  b = (int64_t)blockIdx.x * chunk;
  e = b + chunk < n ? b + chunk : n;
}
__global__ void __launch_bounds__(kAsThreads) k_as_scan_part(mrdem_active_set in,
                                                             const int32_t* __restrict__ em,
                                                             int64_t* bsum) {
  wait_prior_grid();
  __shared__ int64_t wsum[kAsThreads / 32];
  int64_t b, e;
  chunk_of(clamp_count(in), b, e);
  int64_t v = 0;
  const int64_t bt = blockDim.x;
  int64_t i = b + threadIdx.x;
  for (; i + 3 * bt < e; i += 4 * bt) v += (int64_t)em[i] + em[i + bt] + em[i + 2 * bt] + em[i + 3 * bt];
  for (; i < e; i += bt) v += em[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane_id() == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kAsThreads / 32; ++w) t += wsum[w];
    bsum[blockIdx.x] = t;
  }
}
__global__ void __launch_bounds__(kScanMaxBlocks) k_as_scan_top(int64_t* bsum, int nb,
                                                                int64_t* total) {
  wait_prior_grid();
  __shared__ int64_t part[kScanMaxBlocks];
  const int t = threadIdx.x;
  const int64_t v = t < nb ? bsum[t] : 0;
  part[t] = v;
  __syncthreads();
  for (int o = 1; o < kScanMaxBlocks; o <<= 1) {
    const int64_t x = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  if (t < nb) bsum[t] = part[t] - v;
  if (t == kScanMaxBlocks - 1) *total = part[t];
}
__global__ void __launch_bounds__(kAsThreads) k_as_scan_apply(mrdem_active_set in, int32_t* em,
                                                              const int64_t* __restrict__ bsum) {
  wait_prior_grid();
  __shared__ int wtot[kAsThreads / 32];
  int64_t b, e;
  chunk_of(clamp_count(in), b, e);
  int64_t carry = bsum[blockIdx.x];
  const int w = threadIdx.x >> 5;
  // four consecutive counts per thread and pass
  for (int64_t base = b; base < e; base += 4 * (int64_t)blockDim.x) {
    const int64_t i = base + 4 * (int64_t)threadIdx.x;
    int v[4], sum = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = i + u < e ? em[i + u] : 0;
      sum += v[u];
    }
    const int incl = warp_scan(sum);
    if (lane_id() == 31) wtot[w] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int k = 0; k < kAsThreads / 32; ++k) {
      before += k < w ? wtot[k] : 0;
      all += wtot[k];
    }
    int64_t o = carry + before + incl - sum;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (i + u < e) em[i + u] = (int32_t)(o < INT32_MAX ? o : INT32_MAX);
      o += v[u];
    }
    carry += all;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kAsThreads) k_as_emit(HierDev H, mrdem_active_set in,
                                                        const int8_t* __restrict__ st,
                                                        const int32_t* __restrict__ off,
                                                        mrdem_active_set out, int64_t* counts,
                                                        unsigned long long* status) {
  wait_prior_grid();
  const int64_t n = clamp_count(in);
  const int64_t total = *out.count;
  if (blockIdx.x == 0 && threadIdx.x == 0 && total > out.capacity)
    atomicMax(status + ST_REQ_ACTIVE, (unsigned long long)total);
  const int4* items = reinterpret_cast<const int4*>(in.item);
  int4* o4 = reinterpret_cast<int4*>(out.item);
  const int64_t cap = out.capacity;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  WarpCount widened;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += step) {
    const int64_t k = base + threadIdx.x;
    bool w = false;
    if (k < n) {
      const int64_t o = off[k], next = k + 1 < n ? (int64_t)off[k + 1] : total;
      const int s = st[k];
      const int4 it = items[k];
      if (s == AS_PARENT) {
        int pa, pb;
        parent_pair(H, it.y, it.z, pa, pb);
        if (o < cap) o4[o] = make_int4(it.x, pa, pb, kNarrowed);
      } else if (s == AS_WIDEN) {
        w = true;
        const int2 sa = side_of(H, it.y), sb = side_of(H, it.z);
        const int cf = (it.w & (kVeto | kNarrowed)) ? kVeto : 0;
        for (int64_t r = 0; r < next - o && o + r < cap; ++r)
          o4[o + r] = make_int4(it.x, sa.x + (int)(r / sb.y), sb.x + (int)(r % sb.y), cf);
      } else if (s != AS_MERGED) {
        if (o < cap) o4[o] = it;
      }
    }
    widened.add(w);
  }
  widened.flush(reinterpret_cast<unsigned long long*>(counts));
}

// Surrogate contact forces (the force law of Sec. 2 with tau = delta_a +
// delta_b + 2 eps in place of 2 eps, times the weight), FP64 atomics into
// the per-particle sums.
__global__ void __launch_bounds__(kAsThreads) k_sur_forces(
    HierDev H, int64_t n_pairs, const int32_t* __restrict__ ab, const double* __restrict__ eps,
    const double* __restrict__ poses, mrdem_contacts sur, const double* __restrict__ mass,
    const double* __restrict__ com, double k_s, double weight, double* ft, double* energy) {
  int64_t n = *sur.count;
  if (n > sur.capacity) n = sur.capacity;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += step) {
    const int p = sur.pair[k], a = sur.tri_a[k], b = sur.tri_b[k];
    if (p < 0 || p >= n_pairs || a < 0 || b < 0 || a >= H.n_nodes || b >= H.n_nodes) continue;
    const int A = ab[2 * p], B = ab[2 * p + 1];
    if (A < 0 || B < 0 || A >= H.n_particles || B >= H.n_particles) continue;
    const double mu = 1.0 / (1.0 / mass[A] + 1.0 / mass[B]);
    const double ks = weight * k_s * sqrt(mu);
    const double tau = (double)H.node_geo[3 * a].w + (double)H.node_geo[3 * b].w + 2.0 * eps[p];
    const double d = sur.dist[k];
    const D3 pa = {sur.point_a[3 * k], sur.point_a[3 * k + 1], sur.point_a[3 * k + 2]};
    const D3 pb = {sur.point_b[3 * k], sur.point_b[3 * k + 1], sur.point_b[3 * k + 2]};
    const double* PA = poses + 7 * (int64_t)A;
    const double* PB = poses + 7 * (int64_t)B;
    double RA[9], RB[9];
    quat_matrix(PA[3], PA[4], PA[5], PA[6], RA);
    quat_matrix(PB[3], PB[4], PB[5], PB[6], RB);
    D3 u;
    if (d > 0.0) {
      u = (1.0 / d) * (pa - pb);
    } else {
      const float4 nb = H.node_nrm[a];
      const double zero[3] = {0.0, 0.0, 0.0};
      const D3 nw = xf_point64(RA, zero, D3{(double)nb.x, (double)nb.y, (double)nb.z});
      const double l = sqrt(dot(nw, nw));
      u = l > 0.0 ? (-1.0 / l) * nw : D3{0.0, 0.0, 0.0};
    }
    const double sgap = fmax(0.0, 1.0 - d / tau);
    const D3 F = (ks * sgap) * u;
    const D3 xc = 0.5 * (pa + pb);
    const D3 tA = {PA[0], PA[1], PA[2]}, tB = {PB[0], PB[1], PB[2]};
    const D3 cA = xf_point64(RA, &tA.x, D3{com[3 * A], com[3 * A + 1], com[3 * A + 2]});
    const D3 cB = xf_point64(RB, &tB.x, D3{com[3 * B], com[3 * B + 1], com[3 * B + 2]});
    const D3 mA = cross(xc - cA, F), mB = cross(xc - cB, -1.0 * F);
    double* fa = ft + 6 * (int64_t)A;
    double* fb = ft + 6 * (int64_t)B;
    atomicAdd(fa + 0, F.x); atomicAdd(fa + 1, F.y); atomicAdd(fa + 2, F.z);
    atomicAdd(fa + 3, mA.x); atomicAdd(fa + 4, mA.y); atomicAdd(fa + 5, mA.z);
    atomicAdd(fb + 0, -F.x); atomicAdd(fb + 1, -F.y); atomicAdd(fb + 2, -F.z);
    atomicAdd(fb + 3, mB.x); atomicAdd(fb + 4, mB.y); atomicAdd(fb + 5, mB.z);
    if (energy) atomicAdd(energy, ks * 0.5 * tau * sgap * sgap);
  }
}

// Per-item scratch (outcome, count / offset), four counters and the scan's
// chunk sums.
size_t active_off_bytes(int64_t n) { return (size_t)(n + 255) / 256 * 256; }
size_t active_cnt_bytes(int64_t n) {
  return (active_off_bytes(n) + sizeof(int32_t) * (size_t)n + 15) / 16 * 16;
}
int ensure_active(mrdem_ctx* c, int64_t cap) {
  if (cap <= c->cap_active && c->as_status) return MRDEM_OK;
  cudaFree(c->as_status);
  c->as_status = nullptr;
  c->as_off = nullptr;
  c->cap_active = 0;
  const int64_t n = std::max<int64_t>(cap, 1);
  char* mem = nullptr;
  const size_t bytes = active_cnt_bytes(n) + sizeof(int64_t) * (4 + kScanMaxBlocks);
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_OOM;
  }
  c->as_status = reinterpret_cast<int8_t*>(mem);
  c->as_off = reinterpret_cast<int32_t*>(mem + active_off_bytes(n));
  c->cap_active = n;
  return MRDEM_OK;
}
int64_t* active_counts(mrdem_ctx* c) {
  return reinterpret_cast<int64_t*>(reinterpret_cast<char*>(c->as_status) +
                                    active_cnt_bytes(c->cap_active));
}

}  // namespace

int launch_active_init(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs,
                       const int32_t* ab, const mrdem_active_set* out, cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n_pairs + kAsThreads - 1) / kAsThreads,
                                                                 (int64_t)c->n_sms * 8));
  k_as_init<<<blocks, kAsThreads, 0, s>>>(hier->dev, n_pairs, ab, *out);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_active_step(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs,
                       const int32_t* ab, const double* eps, const double* poses, int precision,
                       const mrdem_active_set* in, const mrdem_active_set* out,
                       const mrdem_contacts* contacts, const mrdem_contacts* sur,
                       int64_t* counts, cudaStream_t s) {
  int st = ensure_pairs(c, n_pairs);
  if (st) return st;
  mrdem_contacts tmp;
  st = ensure_tmp(c, contacts->capacity, &tmp);
  if (st) return st;
  st = ensure_active(c, in->capacity);
  if (st) return st;
  int64_t* cnt4 = active_counts(c);
  cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * CNT_TOTAL, s);
  cudaMemsetAsync(contacts->count, 0, sizeof(int64_t), s);
  cudaMemsetAsync(tmp.count, 0, sizeof(int64_t), s);
  cudaMemsetAsync(sur->count, 0, sizeof(int64_t), s);
  cudaMemsetAsync(out->count, 0, sizeof(int64_t), s);
  cudaMemsetAsync(cnt4, 0, 4 * sizeof(int64_t), s);
  if (n_pairs > 0) {
    cudaMemsetAsync(c->pair_cnt, 0, sizeof(int32_t) * n_pairs, s);
    st = launch_setup_transforms(c, hier, n_pairs, ab, eps, poses, s);
    if (st) return st;
    const HierDev& H = hier->dev;
    const int blocks = c->n_sms * (2048 / kAsThreads);
    {
      ProfScope ps(c, K_LEVEL, s);
      const AsTestArgs ta = {H,
                             c->xf,
                             c->xf64,
                             sweep_const(c->params),
                             c->params.conv_c,
                             eps,
                             reinterpret_cast<const int4*>(in->item),
                             c->as_status,
                             c->as_off,
                             c->tiles,
                             c->counters,
                             c->status,
                             c->cap_tiles,
                             *sur};
      launch_after(k_as_test, blocks, kAsThreads, 0, s, ta, n_pairs, *in);
      launch_after(k_as_narrow, blocks, kAsThreads, 0, s, H, n_pairs, *in, c->as_status,
                   c->as_off, cnt4);
      const int sb = std::min(kScanMaxBlocks, c->n_sms * 4);
      int64_t* bsum = cnt4 + 4;
      launch_after(k_as_scan_part, sb, kAsThreads, 0, s, *in, (const int32_t*)c->as_off, bsum);
      launch_after(k_as_scan_top, 1, kScanMaxBlocks, 0, s, bsum, sb, out->count);
      launch_after(k_as_scan_apply, sb, kAsThreads, 0, s, *in, c->as_off, (const int64_t*)bsum);
      launch_after(k_as_emit, blocks, kAsThreads, 0, s, H, *in, (const int8_t*)c->as_status,
                   (const int32_t*)c->as_off, *out, cnt4, c->status);
    }
    st = launch_fine_tail(c, hier, n_pairs, eps, precision, &tmp, contacts,
                          shape_for(c, n_pairs), s);
    if (st) return st;
  }
  cudaMemcpyAsync(cnt4 + 2, c->counters + CNT_TILES, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(cnt4 + 3, sur->count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  if (counts) cudaMemcpyAsync(counts, cnt4, 4 * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_surrogate_forces(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs,
                            const int32_t* ab, const double* eps, const double* poses,
                            const mrdem_contacts* sur, const double* mass, const double* com,
                            double k_s, double weight, double* ft, double* energy,
                            cudaStream_t s) {
  const int blocks = c->n_sms * 2;
  ProfScope ps(c, K_FORCES, s);
  k_sur_forces<<<blocks, kAsThreads, 0, s>>>(hier->dev, n_pairs, ab, eps, poses, *sur, mass, com,
                                             k_s, weight, ft, energy);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
