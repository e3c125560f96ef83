// mrdem_closest.cu -- closest points of many triangle pairs, finished in
// double precision with uniform work per lane.
//
// Used by the FP32 form of the exact distance (Sec. 3, comparison-based
// method, the final test of Algorithm 4).  Three steps:
//   k_cp_float   one thread per pair: the fifteen sub-tests in float on
//                coordinates relative to A's first vertex; a pair clearly
//                beyond 2 eps is dropped, a crossing or nearly touching pair
//                goes to a fallback list (full double test), and every other
//                pair is accepted: its double geometry is stored and one work
//                item per sub-test within 2 err of the float minimum is
//                appended to the point-triangle or the edge-edge list;
//   k_cp_items   one thread per work item, one list at a time, so the lanes
//                of a warp run the same double routine;
//   k_select_exact one thread per accepted pair: the smallest of its items
//                is the distance (the true minimiser is always among them)
//                and the pair's contact is written.
#include <cuda_runtime.h>

#include <algorithm>

#include "mrdem_device.cuh"

namespace mrdem {

// Reserve `n` consecutive slots per lane in a list; returns this lane's
// first slot (or -1 on overflow, latched in *req).
__device__ __forceinline__ int64_t warp_reserve(int n, unsigned long long* counter, int64_t cap,
                                                unsigned long long* req) {
  int incl = warp_scan(n);
  int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane_id() == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 31);
  int64_t first = (int64_t)base + incl - n;
  if (n && first + n > cap) {
    atomicMax(req, (unsigned long long)(first + n));
    return -1;
  }
  return first;
}

__global__ void __launch_bounds__(128) k_cp_float(HierDev H, const PairXf* __restrict__ xf,
                                                  const PairXf64* __restrict__ xf64,
                                                  const int3* __restrict__ cands,
                                                  AccRec* acc, int64_t cap_acc, int* items_pt,
                                                  int* items_ee, int64_t cap_items,
                                                  int* fallback, int64_t cap_fallback,
                                                  unsigned long long* cnt,
                                                  unsigned long long* status) {
  int64_t n = (int64_t)cnt[CNT_CANDS];
  if (n > cap_acc) n = cap_acc;  // the accepted list has the candidate list's capacity
  unsigned n_pt = 0, n_ee = 0;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    int res = 0;
    unsigned mask = 0;
    int3 e = make_int3(0, 0, 0);
    if (k < n) {
      e = cands[k];
      PairXf X;
      load_pairxf(xf, e.x, X);
      F3 a0 = load_vertex(H, e.y, 0), a1 = load_vertex(H, e.y, 1), a2 = load_vertex(H, e.y, 2);
      F3 Pf[3] = {{0.f, 0.f, 0.f}, a1 - a0, a2 - a0};
      F3 Qf[3] = {xf_point(X, load_vertex(H, e.z, 0)) - a0, xf_point(X, load_vertex(H, e.z, 1)) - a0,
                  xf_point(X, load_vertex(H, e.z, 2)) - a0};
      res = cand_float_stage(Pf, Qf, (double)X.tau, X.margin, &mask);
    }
    // accepted pairs: double geometry and work items
    bool accept = res == 1;
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
    int64_t pt0 = warp_reserve(npt, cnt + CNT_PT, cap_items, status + ST_REQ_CANDS);
    int64_t ee0 = warp_reserve(nee, cnt + CNT_EE, cap_items, status + ST_REQ_CANDS);
    if (accept && (pt0 < 0 || ee0 < 0)) accept = false;
    n_pt += accept ? (unsigned)npt : 0u;
    n_ee += accept ? (unsigned)nee : 0u;
    if (accept) {
      AccRec& r = acc[ai];
      const PairXf64& X64 = xf64[e.x];
      CandGeom g;
      cand_geom(H, X64, e, g);
      r.g = g;
      r.entry = (int)k;
      r.pair = e.x;
      r.pt_begin = (int)pt0;
      r.ee_begin = (int)ee0;
      r.counts = npt | (nee << 8);
      int ip = (int)pt0, ie = (int)ee0;
      for (int f = 0; f < 15; ++f) {
        if (!((mask >> f) & 1u)) continue;
        int item = (int)(ai << 4) | f;
        if (f < 6) items_pt[ip++] = item;
        else items_ee[ie++] = item;
      }
    }
    warp_append(res < 0, (int)k, fallback, cnt + CNT_FALLBACK, cap_fallback, status + ST_REQ_CANDS);
  }
  n_pt = __reduce_add_sync(0xffffffffu, n_pt);
  n_ee = __reduce_add_sync(0xffffffffu, n_ee);
  if (lane_id() == 0) {
    if (n_pt) atomicAdd(cnt + CNT_STATS + MRDEM_STAT_ITEMS_PT, (unsigned long long)n_pt);
    if (n_ee) atomicAdd(cnt + CNT_STATS + MRDEM_STAT_ITEMS_EE, (unsigned long long)n_ee);
  }
}

// One sub-test in double per thread; the lanes of a warp run the same
// routine (point-triangle or edge-edge list).
__global__ void __launch_bounds__(256) k_cp_items(const AccRec* __restrict__ acc,
                                                  const int* __restrict__ items, int count_slot,
                                                  int64_t cap_items, ItemRes* res,
                                                  const unsigned long long* cnt) {
  int64_t n = (int64_t)cnt[count_slot];
  if (n > cap_items) n = cap_items;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    int it = items[k];
    const CandGeom& g = acc[it >> 4].g;
    CandGeom G = g;
    D3 pa, pb;
    double wa[3], wb[3];
    double d2 = eval_subtest(G.P, G.Q, it & 15, &pa, &pb, wa, wb);
    ItemRes& r = res[k];
    r.d2 = d2;
    r.pa[0] = pa.x; r.pa[1] = pa.y; r.pa[2] = pa.z;
    r.pb[0] = pb.x; r.pb[1] = pb.y; r.pb[2] = pb.z;
    for (int q = 0; q < 3; ++q) { r.wa[q] = wa[q]; r.wb[q] = wb[q]; }
  }
}

// The smallest item of an accepted pair.
__device__ __forceinline__ const ItemRes* best_item(const AccRec& r, const ItemRes* res_pt,
                                                    const ItemRes* res_ee) {
  const ItemRes* best = nullptr;
  int npt = r.counts & 0xff, nee = (r.counts >> 8) & 0xff;
  for (int q = 0; q < npt; ++q) {
    const ItemRes* x = res_pt + r.pt_begin + q;
    if (!best || x->d2 < best->d2) best = x;
  }
  for (int q = 0; q < nee; ++q) {
    const ItemRes* x = res_ee + r.ee_begin + q;
    if (!best || x->d2 < best->d2) best = x;
  }
  return best;
}

// Exact pass: contacts of the accepted candidates.
__global__ void __launch_bounds__(128) k_select_exact(HierDev H, const PairXf64* __restrict__ xf64,
                                                      const AccRec* __restrict__ acc,
                                                      const ItemRes* __restrict__ res_pt,
                                                      const ItemRes* __restrict__ res_ee,
                                                      const int3* __restrict__ cands,
                                                      unsigned long long* cnt, int64_t cap_acc,
                                                      unsigned long long* status,
                                                      mrdem_contacts out) {
  int64_t n = (int64_t)cnt[CNT_ACC];
  if (n > cap_acc) n = cap_acc;
  WarpCount ncon;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    bool hit = false;
    int3 c = make_int3(0, 0, 0);
    double d = 0;
    D3 pa = {0, 0, 0}, pb = {0, 0, 0};
    if (k < n) {
      const AccRec& r = acc[k];
      const ItemRes* b = best_item(r, res_pt, res_ee);
      if (b) {
        d = sqrt(b->d2);
        hit = d <= r.g.tau;
        if (hit) {
          c = cands[r.entry];
          const PairXf64& X = xf64[r.pair];
          pa = xf_point64(X.RA, X.tA, D3{b->pa[0], b->pa[1], b->pa[2]} + r.g.o);
          pb = xf_point64(X.RA, X.tA, D3{b->pb[0], b->pb[1], b->pb[2]} + r.g.o);
        }
      }
    }
    ncon.add(hit);
    write_contact(H, out, status, hit, c.x, c.y, c.z, d, pa, pb);
  }
  ncon.flush(cnt + CNT_STATS + MRDEM_STAT_CONTACTS);
}

// Full double test of the fallback entries (indices into the candidates).
__global__ void __launch_bounds__(128) k_exact64_idx(HierDev H, const PairXf64* __restrict__ xf64,
                                                     const int3* __restrict__ cands,
                                                     const int* __restrict__ list,
                                                     unsigned long long* cnt, int64_t cap,
                                                     unsigned long long* status,
                                                     mrdem_contacts out) {
  int64_t n = (int64_t)cnt[CNT_FALLBACK];
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
      c = cands[list[k]];
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
    write_contact(H, out, status, hit, c.x, c.y, c.z, d, pa, pb);
  }
  ncon.flush(cnt + CNT_STATS + MRDEM_STAT_CONTACTS);
  nall.flush(cnt + CNT_STATS + MRDEM_STAT_FP64);
}

// ---------------------------------------------------------------------------
// launchers

// The float stage over the candidate list and the two double item lists.
static int closest_float_stage(mrdem_ctx* c, const mrdem_hier* hier, int* fallback,
                               int64_t cap_fallback, cudaStream_t s) {
  cudaMemsetAsync(c->counters + CNT_ACC, 0, sizeof(unsigned long long) * 3, s);
  cudaMemsetAsync(c->counters + CNT_FALLBACK, 0, sizeof(unsigned long long), s);
  k_cp_float<<<c->n_sms * 8, 128, 0, s>>>(hier->dev, c->xf, c->xf64, c->cands, c->acc,
                                          c->cap_cands, c->items_pt, c->items_ee, c->cap_items,
                                          fallback, cap_fallback, c->counters, c->status);
  int ib = c->n_sms * 8;
  k_cp_items<<<ib, 256, 0, s>>>(c->acc, c->items_pt, CNT_PT, c->cap_items, c->res_pt, c->counters);
  k_cp_items<<<ib, 256, 0, s>>>(c->acc, c->items_ee, CNT_EE, c->cap_items, c->res_ee, c->counters);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_exact_fp32(mrdem_ctx* c, const mrdem_hier* hier, const mrdem_contacts* out,
                      cudaStream_t s) {
  int* fallback = reinterpret_cast<int*>(c->level_list[0]);  // free once the tiles are done
  int st;
  {
    ProfScope ps(c, K_EXACT, s);
    st = closest_float_stage(c, hier, fallback, c->cap_level, s);
    if (st) return st;
    k_select_exact<<<c->n_sms * 8, 128, 0, s>>>(hier->dev, c->xf64, c->acc, c->res_pt, c->res_ee,
                                                 c->cands, c->counters, c->cap_cands, c->status,
                                                 *out);
  }
  ProfScope ps(c, K_EXACT64, s);
  launch_exact64_list(c, hier, fallback, out, s);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_exact64_list(mrdem_ctx* c, const mrdem_hier* hier, const int* fallback,
                        const mrdem_contacts* out, cudaStream_t s) {
  k_exact64_idx<<<c->n_sms * 4, 128, 0, s>>>(hier->dev, c->xf64, c->cands, fallback, c->counters,
                                              c->cap_level, c->status, *out);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
