// mrdem_device.cuh -- device helpers shared by the kernels: lane utilities,
// warp-aggregated list appends and output queues, statistics counters, the
// pair transforms, the loads of the fine triangles' 48-B records and the
// double-float candidate geometry.
#pragma once

#include <utility>

#include <cuda_runtime.h>

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
template <typename Item>
__device__ __forceinline__ void warp_append(bool pred, const Item& item, Item* list,
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

// Programmatic dependent launch: a kernel started with launch_after may be
// scheduled while the previous kernel of the stream drains; it waits in
// wait_prior_grid(), its first statement, until that kernel has completed
// and its writes are visible, so the stream order of the work is kept and
// only launch latency and the previous kernel's tail overlap.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... Exp, typename... Act>
inline cudaError_t launch_after(void (*kernel)(Exp...), dim3 grid, dim3 block, size_t smem,
                                cudaStream_t s, Act&&... args) {
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Act>(args)...);
}

// Inclusive warp prefix sum.
__device__ __forceinline__ int warp_scan(int v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane_id() >= o) v += y;
  }
  return v;
}

// Per-warp output queue in shared memory: items are collected with a ballot
// per round and written out in batches, one global atomic per batch instead
// of one per round.  All calls must be made by all 32 lanes.
template <typename Item, int CAP>
struct WarpQueue {
  Item* buf;  // shared memory, CAP items
  int n = 0;  // warp-uniform fill level
  __device__ __forceinline__ void flush(Item* list, unsigned long long* counter, int64_t cap,
                                        unsigned long long* req) {
    __syncwarp();
    if (n == 0) return;
    unsigned long long base = 0;
    if (lane_id() == 0) base = atomicAdd(counter, (unsigned long long)n);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int k = lane_id(); k < n; k += 32) {
      unsigned long long idx = base + k;
      if ((int64_t)idx < cap) list[idx] = buf[k];
      else atomicMax(req, idx + 1);
    }
    n = 0;
    __syncwarp();
  }
  __device__ __forceinline__ void push(bool pred, const Item& item, Item* list,
                                       unsigned long long* counter, int64_t cap,
                                       unsigned long long* req) {
    unsigned m = __ballot_sync(0xffffffffu, pred);
    if (pred) buf[n + __popc(m & ((1u << lane_id()) - 1u))] = item;
    n += __popc(m);
    if (n > CAP - 32) flush(list, counter, cap, req);
  }
};

// Tile item of a pair of leaves (ia, ib: their child records, slot ranges).
__device__ __forceinline__ TileItem make_tile(int pair, int na_node, int nb_node, int2 ia, int2 ib) {
  TileItem t;
  t.pair = pair;
  t.node_a = na_node;
  t.node_b = nb_node;
  t.slot_a = ia.x;
  t.slot_b = ib.x;
  t.counts = (-ia.y) | ((-ib.y) << 8);
  t.pad0 = t.pad1 = 0;
  return t;
}
__device__ __forceinline__ F3 xf_point(const PairXf& X, F3 v) {
  return {fmaf(X.R[0], v.x, fmaf(X.R[1], v.y, fmaf(X.R[2], v.z, X.t[0]))),
          fmaf(X.R[3], v.x, fmaf(X.R[4], v.y, fmaf(X.R[5], v.z, X.t[1]))),
          fmaf(X.R[6], v.x, fmaf(X.R[7], v.y, fmaf(X.R[8], v.z, X.t[2])))};
}
// A node's oriented box (body frame): centre, unit axes (rows), half
// extents; it holds every fine vertex below the node (built on the host).
struct NodeBox {
  F3 c;
  F3 u[3];
  float h[3];
};
__device__ __forceinline__ NodeBox load_box(const HierDev& H, int node) {
  const float4* b = H.node_box + 4 * (int64_t)node;
  const float4 a = __ldg(b), x = __ldg(b + 1), y = __ldg(b + 2), z = __ldg(b + 3);
  NodeBox o;
  o.c = {a.x, a.y, a.z};
  o.u[0] = {x.x, x.y, x.z};
  o.u[1] = {y.x, y.y, y.z};
  o.u[2] = {z.x, z.y, z.z};
  o.h[0] = a.w;
  o.h[1] = x.w;
  o.h[2] = y.w;
  return o;
}
// B's box moved into A's frame: centre by the pair transform, axes rotated.
__device__ __forceinline__ NodeBox move_box(const PairXf& X, const NodeBox& b) {
  NodeBox o;
  o.c = xf_point(X, b.c);
  for (int k = 0; k < 3; ++k) {
    const F3 v = b.u[k];
    o.u[k] = {fmaf(X.R[0], v.x, fmaf(X.R[1], v.y, X.R[2] * v.z)),
              fmaf(X.R[3], v.x, fmaf(X.R[4], v.y, X.R[5] * v.z)),
              fmaf(X.R[6], v.x, fmaf(X.R[7], v.y, X.R[8] * v.z))};
    o.h[k] = b.h[k];
  }
  return o;
}
// Separating-axis test of two oriented boxes (same frame: A's box, and B's
// moved into A's frame): along each of the six face axes a, the centres are
// farther apart than the two half widths plus gap (a box's half width along
// a is sum_k h_k |a . u_k|), so no point of one box comes within gap of the
// other.  Each box's half widths along its own axes come from node_boxw
// (wa, wb: rotation-invariant, so B's unmoved values hold; they differ from
// the moved axes' float dot products far inside the pair's rounding
// margin); the nine products of the two axis sets serve both sides' other
// half widths.  True when one face axis separates the boxes by more than
// gap.
__device__ __forceinline__ bool boxes_apart_w(const NodeBox& A, float4 wa, const NodeBox& B,
                                              float4 wb, float gap) {
  const F3 d = {B.c.x - A.c.x, B.c.y - A.c.y, B.c.z - A.c.z};
  float M[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      M[i][k] = fabsf(fmaf(A.u[i].x, B.u[k].x, fmaf(A.u[i].y, B.u[k].y, A.u[i].z * B.u[k].z)));
  const float wA[3] = {wa.x, wa.y, wa.z}, wB[3] = {wb.x, wb.y, wb.z};
  bool apart = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float dist = fabsf(fmaf(A.u[i].x, d.x, fmaf(A.u[i].y, d.y, A.u[i].z * d.z)));
    const float hw = fmaf(B.h[2], M[i][2], fmaf(B.h[1], M[i][1], B.h[0] * M[i][0]));
    apart = apart || dist > wA[i] + hw + gap;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float dist = fabsf(fmaf(B.u[k].x, d.x, fmaf(B.u[k].y, d.y, B.u[k].z * d.z)));
    const float hw = fmaf(A.h[2], M[2][k], fmaf(A.h[1], M[1][k], A.h[0] * M[0][k]));
    apart = apart || dist > hw + wB[k] + gap;
  }
  return apart;
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
  unsigned v = 0;  // per-warp totals stay far below 2^32
  __device__ __forceinline__ void add(bool pred) {
    unsigned m = __ballot_sync(0xffffffffu, pred);
    v += __popc(m);
  }
  __device__ __forceinline__ void flush(unsigned long long* dst) {
    if (lane_id() == 0 && v) atomicAdd(dst, (unsigned long long)v);
  }
};

// Exclusive prefix sum of n int32 counts in place by one block of up to 1024
// threads, each taking a contiguous run of the counts; the sum of all counts
// goes to *total when total is not null.
__device__ __forceinline__ void block_exclusive_scan(int32_t* cnt, int64_t n, int64_t* total) {
  __shared__ int64_t part[1024];
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b = threadIdx.x * per, e = b + per < n ? b + per : n;
  int64_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += cnt[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    int64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - sum;
  for (int64_t i = b; i < e; ++i) {
    int32_t c = cnt[i];
    cnt[i] = (int32_t)run;
    run += c;
  }
  if (total && threadIdx.x == blockDim.x - 1) *total = part[threadIdx.x];
}

// Per-key sums over a warp.  For every distinct key among the lanes with
// `ok` set (the group of lanes holding that key), lane e (e < nq, in strides
// of 32) forms term = val(e) and receives the group's sum of term(l) over its
// lanes l through emit(key, e, sum); then, after a warp barrier, post(key)
// runs on every lane.  Contacts of one particle pair sit mostly next to each
// other in a contact list, so a warp holds few groups and a per-pair output
// gets one atomic per group instead of one per contact.  Sums run in lane
// order, in the type Acc of the terms (double, or double-float).
template <typename Acc, typename Val, typename Emit, typename Post>
__device__ __forceinline__ void warp_group_sums(bool ok, int key, int nq, Val val, Emit emit,
                                                Post post) {
  const int lane = lane_id();
  unsigned pending = __ballot_sync(0xffffffffu, ok);
  while (pending) {
    const int k = __shfl_sync(0xffffffffu, key, __ffs(pending) - 1);
    const unsigned grp = __ballot_sync(0xffffffffu, ok && key == k);
    pending &= ~grp;
    for (int e = lane; e < nq; e += 32) {
      const auto term = val(e);
      Acc acc(0);
      for (unsigned g = grp; g; g &= g - 1) acc = acc + term(__ffs(g) - 1);
      emit(k, e, acc);
    }
    __syncwarp();
    post(k);
    __syncwarp();
  }
}

// A fine triangle's body-frame vertices: one 48-B record, three 16-B loads.
__device__ __forceinline__ void load_tri(const HierDev& H, int slot, F3 v[3]) {
  const float4* r = H.tri + 3 * (int64_t)slot;
  float4 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2);
  v[0] = {a.x, a.y, a.z};
  v[1] = {a.w, b.x, b.y};
  v[2] = {b.z, b.w, c.x};
}

__device__ __forceinline__ void load_tri64(const HierDev& H, int slot, D3 T[3]) {
  F3 v[3];
  load_tri(H, slot, v);
#pragma unroll
  for (int c = 0; c < 3; ++c) T[c] = {(double)v[c].x, (double)v[c].y, (double)v[c].z};
}

__device__ __forceinline__ void cand_geom(const HierDev& H, const PairXf64& X, int3 c, CandGeom& g) {
  D3 Pb[3], Qb[3];
  load_tri64(H, c.y, Pb);
  load_tri64(H, c.z, Qb);
  g.o = Pb[0];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    g.P[v] = Pb[v] - g.o;
    g.Q[v] = xf_point64(X.R, X.t, Qb[v]) - g.o;
  }
  g.tau = 2.0 * X.eps;
}

// FP32 form: a candidate's geometry in double-float (see CandDD).  L is the
// largest float coordinate magnitude relative to A's first vertex (from the
// float stage), which fixes the power-of-two scale.
__device__ __forceinline__ V3<dd> scale_dd(V3<dd> v, float s) {
  // multiplying both words by a power of two is exact
  return {dd(v.x.hi * s, v.x.lo * s), dd(v.y.hi * s, v.y.lo * s), dd(v.z.hi * s, v.z.lo * s)};
}
__device__ __forceinline__ void cand_dd(const HierDev& H, const PairXfDD& X, int3 c, double tau,
                                        float L, CandDD& g) {
  const int k = L > 0.f ? ilogbf(L) : 0;
  const float s = ldexpf(1.f, -k);
  F3 a[3], bq[3];
  load_tri(H, c.y, a);
  load_tri(H, c.z, bq);
  g.o[0] = a[0].x; g.o[1] = a[0].y; g.o[2] = a[0].z;
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    // differences of floats are exact as double-float
    g.P[v] = scale_dd({two_sum(a[v].x, -a[0].x), two_sum(a[v].y, -a[0].y), two_sum(a[v].z, -a[0].z)}, s);
    const F3 b = bq[v];
    dd q[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dd acc = X.t[r] - dd(g.o[r]);
      acc = acc + mul_f(X.R[3 * r], b.x);
      acc = acc + mul_f(X.R[3 * r + 1], b.y);
      q[r] = acc + mul_f(X.R[3 * r + 2], b.z);
    }
    g.Q[v] = scale_dd({q[0], q[1], q[2]}, s);
  }
  g.k = k;
  g.tau = tau;
}
// The two triangles of a candidate record as nine 16-B loads (P then Q, each
// vertex x.hi x.lo y.hi y.lo z.hi z.lo).
__device__ __forceinline__ void load_cand_tris(const AccRec* r, V3<dd> P[3], V3<dd> Q[3]) {
  const float4* s = reinterpret_cast<const float4*>(r);
  float f[36];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    float4 v = __ldg(s + q);
    f[4 * q] = v.x; f[4 * q + 1] = v.y; f[4 * q + 2] = v.z; f[4 * q + 3] = v.w;
  }
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    P[v] = {dd(f[6 * v], f[6 * v + 1]), dd(f[6 * v + 2], f[6 * v + 3]), dd(f[6 * v + 4], f[6 * v + 5])};
    Q[v] = {dd(f[18 + 6 * v], f[18 + 6 * v + 1]), dd(f[18 + 6 * v + 2], f[18 + 6 * v + 3]),
            dd(f[18 + 6 * v + 4], f[18 + 6 * v + 5])};
  }
}
// Store a candidate record as twelve 16-B words.
__device__ __forceinline__ void store_acc(AccRec* dst, const CandDD& g, int entry, int pair,
                                          int pt_begin, int ee_begin, int cx_begin, int counts) {
  float f[48];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const V3<dd>& p = g.P[v];
    const V3<dd>& q = g.Q[v];
    f[6 * v] = p.x.hi; f[6 * v + 1] = p.x.lo; f[6 * v + 2] = p.y.hi;
    f[6 * v + 3] = p.y.lo; f[6 * v + 4] = p.z.hi; f[6 * v + 5] = p.z.lo;
    f[18 + 6 * v] = q.x.hi; f[18 + 6 * v + 1] = q.x.lo; f[18 + 6 * v + 2] = q.y.hi;
    f[18 + 6 * v + 3] = q.y.lo; f[18 + 6 * v + 4] = q.z.hi; f[18 + 6 * v + 5] = q.z.lo;
  }
  f[36] = g.o[0]; f[37] = g.o[1]; f[38] = g.o[2]; f[39] = __int_as_float(g.k);
  f[40] = __int_as_float(__double2loint(g.tau)); f[41] = __int_as_float(__double2hiint(g.tau));
  f[42] = __int_as_float(entry); f[43] = __int_as_float(pair);
  f[44] = __int_as_float(pt_begin); f[45] = __int_as_float(ee_begin);
  f[46] = __int_as_float(cx_begin); f[47] = __int_as_float(counts);
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int q = 0; q < 12; ++q) d[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
}

// World point of a candidate-frame point p (scaled by 2^-k, relative to o).
__device__ __forceinline__ D3 world_point(const PairXfDD& X, V3<dd> p, int k, const float o[3]) {
  V3<dd> b = scale_dd(p, ldexpf(1.f, k));
  b = {b.x + dd(o[0]), b.y + dd(o[1]), b.z + dd(o[2])};
  dd w[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    w[r] = X.tA[r] + X.RA[3 * r] * b.x + X.RA[3 * r + 1] * b.y + X.RA[3 * r + 2] * b.z;
  return {to_double(w[0]), to_double(w[1]), to_double(w[2])};
}

// Append a contact (warp-collective).  pair_cnt, if given, counts the stored
// contacts of each pair (for the ordering by pair that follows).
__device__ __forceinline__ void write_contact(const HierDev& H, const mrdem_contacts& out,
                                              unsigned long long* status, bool hit, int pair,
                                              int sa, int sb, double d, D3 pa, D3 pb,
                                              int32_t* pair_cnt = nullptr) {
  unsigned m = __ballot_sync(0xffffffffu, hit);
  if (!m) return;
  int leader = __ffs(m) - 1;
  unsigned long long b = 0;
  if ((int)lane_id() == leader) b = atomicAdd((unsigned long long*)out.count, (unsigned long long)__popc(m));
  b = __shfl_sync(0xffffffffu, b, leader);
  if (!hit) return;
  unsigned long long idx = b + __popc(m & ((1u << lane_id()) - 1u));
  const bool stored = (int64_t)idx < out.capacity;
  if (stored) {
    out.pair[idx] = pair;
    out.tri_a[idx] = H.slot_tri[sa];
    out.tri_b[idx] = H.slot_tri[sb];
    out.dist[idx] = d;
    out.point_a[3 * idx] = pa.x; out.point_a[3 * idx + 1] = pa.y; out.point_a[3 * idx + 2] = pa.z;
    out.point_b[3 * idx] = pb.x; out.point_b[3 * idx + 1] = pb.y; out.point_b[3 * idx + 2] = pb.z;
  } else {
    atomicMax(status + ST_REQ_CONTACTS, idx + 1);
  }
  // per-pair counts: one atomic per group of stored lanes holding one pair
  // (the contacts of a warp mostly share their pair)
  if (pair_cnt) {
    const unsigned sm = __ballot_sync(m, stored);
    if (stored) {
      const unsigned g = __match_any_sync(sm, pair);
      if ((int)lane_id() == __ffs(g) - 1) atomicAdd(pair_cnt + pair, __popc(g));
    }
  }
}

}  // namespace mrdem
