// mrdem_closest.cu -- closest points of many triangle pairs, finished in
// double precision with uniform work per lane.
//
// Used by the FP32 form of the exact distance (Sec. 3, comparison-based
// method, the final test of Algorithm 4).  Three steps:
//   k_cp_float   one thread per candidate: the fifteen sub-tests in float on
//                coordinates relative to A's first vertex; a pair clearly
//                beyond 2 eps is dropped; every other pair is accepted: its
//                double-float geometry is stored and one work item per
//                sub-test within 2 err of the float minimum is appended to the
//                point-triangle or the edge-edge list; a crossing or nearly
//                touching pair gets all fifteen sub-tests and the six
//                edge-against-triangle crossing tests as items;
//   k_cp_items   one thread per work item, one list (and one routine) per
//                launch, so the lanes of a warp run the same code, in
//                double-float arithmetic;
//   k_select_exact one thread per accepted pair: the first crossing in the
//                fixed order, else the smallest item, is the distance (the
//                true minimiser is always among them); the contact is
//                written.
#include <cuda_runtime.h>

#include <algorithm>

#include "mrdem_device.cuh"

namespace mrdem {

// Reserve `n` consecutive slots per lane in a list; returns this lane's
// first slot, or -1 on overflow (latched in *req); the slots of a range that
// crosses the capacity that do lie below it get the empty item -1, so that
// every slot the readers see is written.
__device__ __forceinline__ int64_t warp_reserve(int n, int* list, unsigned long long* counter,
                                                int64_t cap, unsigned long long* req) {
  int incl = warp_scan(n);
  int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane_id() == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 31);
  int64_t first = (int64_t)base + incl - n;
  if (n && first + n > cap) {
    atomicMax(req, (unsigned long long)(first + n));
    for (int64_t q = first; q < cap; ++q) list[q] = -1;
    return -1;
  }
  return first;
}

__global__ void __launch_bounds__(256) k_cp_float(HierDev H, const PairXf* __restrict__ xf,
                                                  const PairXf64* __restrict__ xf64,
                                                  const PairXfDD* __restrict__ xfdd,
                                                  const int3* __restrict__ cands,
                                                  AccRec* acc, int64_t cap_acc, int* items_pt,
                                                  int* items_ee, int* items_cx, int64_t cap_items,
                                                  unsigned long long* cnt,
                                                  unsigned long long* status) {
  wait_prior_grid();
  int64_t n = (int64_t)cnt[CNT_CANDS];
  if (n > cap_acc) n = cap_acc;  // the accepted list has the candidate list's capacity
  unsigned n_pt = 0, n_ee = 0;
  WarpCount nfull;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    int res = 0;
    unsigned mask = 0;
    int3 e = make_int3(0, 0, 0);
    float L = 0.f;
    if (k < n) {
      e = cands[k];
      PairXf X;
      load_pairxf(xf, e.x, X);
      F3 a[3], b[3];
      load_tri(H, e.y, a);
      load_tri(H, e.z, b);
      F3 Pf[3] = {{0.f, 0.f, 0.f}, a[1] - a[0], a[2] - a[0]};
      F3 Qf[3] = {xf_point(X, b[0]) - a[0], xf_point(X, b[1]) - a[0], xf_point(X, b[2]) - a[0]};
      res = cand_float_stage(Pf, Qf, (double)X.tau, X.margin, &mask);
#pragma unroll
      for (int v = 0; v < 3; ++v)
        L = fmaxf(L, fmaxf(fmaxf(fabsf(Pf[v].x), fabsf(Pf[v].y)),
                           fmaxf(fmaxf(fabsf(Pf[v].z), fabsf(Qf[v].x)), fmaxf(fabsf(Qf[v].y), fabsf(Qf[v].z)))));
    }
    // accepted pairs: double-float geometry and work items; a crossing or
    // nearly touching pair (res < 0) takes every sub-test and the crossings
    const bool full = res < 0;
    if (full) mask = 0x7fffu;
    nfull.add(full);
    bool accept = res != 0;
    unsigned am = __ballot_sync(0xffffffffu, accept);
    unsigned long long abase = 0;
    if (am) {
      int leader = __ffs(am) - 1;
      if ((int)lane_id() == leader) abase = atomicAdd(cnt + CNT_ACC, (unsigned long long)__popc(am));
      abase = __shfl_sync(0xffffffffu, abase, leader);
    }
    int64_t ai = accept ? (int64_t)abase + __popc(am & ((1u << lane_id()) - 1u)) : -1;
    if (accept && ai >= cap_acc) {
      atomicMax(status + ST_REQ_CANDS, (unsigned long long)(ai + 1));
      accept = false;
    }
    int npt = accept ? __popc(mask & 0x3fu) : 0;
    int nee = accept ? __popc(mask >> 6) : 0;
    int ncx = accept && full ? 6 : 0;
    int64_t pt0 = warp_reserve(npt, items_pt, cnt + CNT_PT, cap_items, status + ST_REQ_CANDS);
    int64_t ee0 = warp_reserve(nee, items_ee, cnt + CNT_EE, cap_items, status + ST_REQ_CANDS);
    int64_t cx0 = warp_reserve(ncx, items_cx, cnt + CNT_CX, cap_items, status + ST_REQ_CANDS);
    // Every slot below a list's capacity that a lane reserved is written,
    // since the next kernels read each of them: when one of the three lists
    // overflows (latched above; the call reports ERR_CAPACITY), the record
    // keeps no items and the slots reserved in the other lists get the
    // empty item -1.
    const bool items_ok = pt0 >= 0 && ee0 >= 0 && cx0 >= 0;
    if (accept && !items_ok) {
      if (pt0 >= 0) for (int q = 0; q < npt; ++q) items_pt[pt0 + q] = -1;
      if (ee0 >= 0) for (int q = 0; q < nee; ++q) items_ee[ee0 + q] = -1;
      if (cx0 >= 0) for (int q = 0; q < ncx; ++q) items_cx[cx0 + q] = -1;
      npt = nee = ncx = 0;
    }
    n_pt += accept ? (unsigned)npt : 0u;
    n_ee += accept ? (unsigned)nee : 0u;
    if (accept) {
      CandDD g;
      cand_dd(H, xfdd[e.x], e, 2.0 * xf64[e.x].eps, L, g);
      store_acc(acc + ai, g, (int)k, e.x, (int)pt0, (int)ee0, (int)cx0,
                npt | (nee << 8) | (ncx << 16));
      if (items_ok) {
        int ip = (int)pt0, ie = (int)ee0;
        for (int f = 0; f < 15; ++f) {
          if (!((mask >> f) & 1u)) continue;
          int item = (int)(ai << 4) | f;
          if (f < 6) items_pt[ip++] = item;
          else items_ee[ie++] = item;
        }
        for (int f = 0; f < ncx; ++f) items_cx[cx0 + f] = (int)(ai << 4) | f;
      }
    }
  }
  n_pt = __reduce_add_sync(0xffffffffu, n_pt);
  n_ee = __reduce_add_sync(0xffffffffu, n_ee);
  if (lane_id() == 0) {
    if (n_pt) atomicAdd(cnt + CNT_STATS + MRDEM_STAT_ITEMS_PT, (unsigned long long)n_pt);
    if (n_ee) atomicAdd(cnt + CNT_STATS + MRDEM_STAT_ITEMS_EE, (unsigned long long)n_ee);
  }
  nfull.flush(cnt + CNT_STATS + MRDEM_STAT_FP64);
}

// One work item per thread in double-float; KIND 0: point-triangle, 1:
// edge-edge, 2: edge-against-triangle crossing (one list per launch, so the
// lanes of a warp run one routine and the kernel holds only that code).
template <int KIND>
__global__ void __launch_bounds__(256) k_cp_items(const AccRec* __restrict__ acc,
                                                  const int* __restrict__ items, int count_slot,
                                                  int64_t cap_items, ItemRes* res, dd* d2_out,
                                                  const unsigned long long* cnt) {
  wait_prior_grid();
  int64_t n = (int64_t)cnt[count_slot];
  if (n > cap_items) n = cap_items;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    int it = items[k];
    if (it < 0) continue;  // an empty slot left by an overflow
    V3<dd> P[3], Q[3];
    load_cand_tris(acc + (it >> 4), P, Q);
    const int f = it & 15;
    V3<dd> pa, pb;
    dd d2;
    if (KIND == 2) {
      // edge (i, i+1) of P through Q for f < 3, of Q through P otherwise
      const int i = f < 3 ? f : f - 3, i1 = i == 2 ? 0 : i + 1;
      V3<dd> s0 = f < 3 ? pick3(P, i) : pick3(Q, i), s1 = f < 3 ? pick3(P, i1) : pick3(Q, i1);
      dd t, w[3];
      bool cross = f < 3 ? segment_crosses(s0, s1, Q[0], Q[1], Q[2], &t, w)
                         : segment_crosses(s0, s1, P[0], P[1], P[2], &t, w);
      if (cross) {
        pa = s0 + t * (s1 - s0);
        d2 = dd(0.f, 0.f);
      } else {
        pa = s0;
        d2 = dd(INFINITY);
      }
      pb = pa;
    } else if (KIND == 0) {
      // vertex f of P against Q, or vertex f - 3 of Q against P, without
      // branches on the Voronoi region (the lanes of a warp stay together)
      if (f < 3) {
        pa = pick3(P, f);
        pb = closest_on_triangle_flat(pa, Q[0], Q[1], Q[2]);
      } else {
        pb = pick3(Q, f - 3);
        pa = closest_on_triangle_flat(pb, P[0], P[1], P[2]);
      }
      V3<dd> dv = pa - pb;
      d2 = dot(dv, dv);
    } else {
      dd wa[3], wb[3];
      d2 = eval_subtest(P, Q, f >= 6 ? f : 6, &pa, &pb, wa, wb);
    }
    float4* o = reinterpret_cast<float4*>(res + k);
    o[0] = make_float4(d2.hi, d2.lo, pa.x.hi, pa.x.lo);
    o[1] = make_float4(pa.y.hi, pa.y.lo, pa.z.hi, pa.z.lo);
    o[2] = make_float4(pb.x.hi, pb.x.lo, pb.y.hi, pb.y.lo);
    o[3] = make_float4(pb.z.hi, pb.z.lo, 0.f, 0.f);
    d2_out[k] = d2;
  }
}

// Exact pass: contacts of the accepted candidates.  One thread per accepted
// pair reads its items' squared distances from the packed arrays (a pair's
// items are contiguous, so a warp's reads share sectors) in the fixed order
// (crossings, then point-triangle, then edge-edge items) and takes the first
// crossing that crossed, else the first smallest squared distance: the
// choice of tri_tri_distance.  Only the chosen item's full record (its
// closest points) is read.
__global__ void __launch_bounds__(256) k_select_exact(HierDev H, const PairXfDD* __restrict__ xfdd,
                                                      const AccRec* __restrict__ acc,
                                                      const ItemRes* __restrict__ res_pt,
                                                      const ItemRes* __restrict__ res_ee,
                                                      const ItemRes* __restrict__ res_cx,
                                                      const dd* __restrict__ d2_pt,
                                                      const dd* __restrict__ d2_ee,
                                                      const dd* __restrict__ d2_cx,
                                                      const int3* __restrict__ cands,
                                                      unsigned long long* cnt, int64_t cap_acc,
                                                      unsigned long long* status,
                                                      mrdem_contacts out, int32_t* pair_cnt) {
  wait_prior_grid();
  int64_t n = (int64_t)cnt[CNT_ACC];
  if (n > cap_acc) n = cap_acc;
  WarpCount ncon;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t k = base + threadIdx.x;
    bool hit = false;
    int3 c = make_int3(0, 0, 0);
    double d = 0;
    D3 pa = {0, 0, 0}, pb = {0, 0, 0};
    if (k < n) {
      const AccRec& r = acc[k];
      const int npt = r.counts & 0xff, nee = (r.counts >> 8) & 0xff;
      const int ncx = (r.counts >> 16) & 0xff;
      const ItemRes* b = nullptr;
      for (int q = 0; q < ncx && !b; ++q)
        if (d2_cx[r.cx_begin + q].hi == 0.f) b = res_cx + r.cx_begin + q;
      if (!b) {
        int best = -1;
        dd bd = dd(INFINITY);
#pragma unroll 2
        for (int q = 0; q < npt; ++q) {
          const dd v = d2_pt[r.pt_begin + q];
          if (best < 0 || v < bd) { bd = v; best = q; }
        }
#pragma unroll 3
        for (int q = 0; q < nee; ++q) {
          const dd v = d2_ee[r.ee_begin + q];
          if (best < 0 || v < bd) { bd = v; best = npt + q; }
        }
        if (best >= 0) b = best < npt ? res_pt + r.pt_begin + best : res_ee + r.ee_begin + (best - npt);
      }
      if (b) {
        d = ldexp(to_double(dd_sqrt(b->d2)), r.g.k);
        hit = d <= r.g.tau;
        if (hit) {
          c = cands[r.entry];
          const PairXfDD& X = xfdd[r.pair];
          pa = world_point(X, b->pa, r.g.k, r.g.o);
          pb = world_point(X, b->pb, r.g.k, r.g.o);
        }
      }
    }
    ncon.add(hit);
    write_contact(H, out, status, hit, c.x, c.y, c.z, d, pa, pb, pair_cnt);
  }
  ncon.flush(cnt + CNT_STATS + MRDEM_STAT_CONTACTS);
}

// ---------------------------------------------------------------------------
// launchers

int launch_exact_fp32(mrdem_ctx* c, const mrdem_hier* hier, const mrdem_contacts* out,
                      int threads, cudaStream_t s) {
  ProfScope ps(c, K_EXACT, s);
  // blocks: 8 per SM at 128 threads, the same threads per SM otherwise
  const int eb = c->n_sms * 8 * 128 / threads;
  // the accepted pairs and the three item lists start empty (counters zeroed by detect)
  launch_after(k_cp_float, eb, threads, 0, s, hier->dev, c->xf, c->xf64, c->xfdd, c->cands,
               c->acc, c->cap_cands, c->items_pt, c->items_ee, c->items_cx, c->cap_items,
               c->counters, c->status);
  int ib = c->n_sms * 8;
  launch_after(k_cp_items<0>, ib, 256, 0, s, c->acc, c->items_pt, (int)CNT_PT, c->cap_items,
               c->res_pt, c->d2_pt, c->counters);
  launch_after(k_cp_items<1>, ib, 256, 0, s, c->acc, c->items_ee, (int)CNT_EE, c->cap_items,
               c->res_ee, c->d2_ee, c->counters);
  launch_after(k_cp_items<2>, ib, 256, 0, s, c->acc, c->items_cx, (int)CNT_CX, c->cap_items,
               c->res_cx, c->d2_cx, c->counters);
  launch_after(k_select_exact, eb, threads, 0, s, hier->dev, c->xfdd, c->acc, c->res_pt,
               c->res_ee, c->res_cx, (const dd*)c->d2_pt, (const dd*)c->d2_ee,
               (const dd*)c->d2_cx, c->cands, c->counters, c->cap_cands, c->status, *out,
               c->pair_cnt);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
