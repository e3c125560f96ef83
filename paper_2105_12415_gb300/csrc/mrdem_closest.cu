// mrdem_closest.cu -- closest points of many triangle pairs, finished in
// double precision with uniform work per lane.
//
// Used by the FP32 form of the exact distance (Sec. 3, comparison-based
// method, the final test of Algorithm 4) and by the adjoint, which recomputes
// each contact's closest points.  Three steps:
//   k_cp_float   one thread per pair: the fifteen sub-tests in float on
//                coordinates relative to A's first vertex; a pair clearly
//                beyond 2 eps is dropped, a crossing or nearly touching pair
//                goes to a fallback list (full double test), and every other
//                pair is accepted: its double geometry is stored and one work
//                item per sub-test within 2 err of the float minimum is
//                appended to the point-triangle or the edge-edge list;
//   k_cp_items   one thread per work item, one list at a time, so the lanes
//                of a warp run the same double routine;
//   k_select_*   one thread per accepted pair: the smallest of its items is
//                the distance (the true minimiser is always among them);
//                the exact pass writes the contact, the adjoint scatters the
//                gradient.
#include <cuda_runtime.h>

#include <algorithm>

#include "mrdem_device.cuh"

namespace mrdem {

// Entries of the float stage come from the candidate list (detection) or
// from the caller's contact list (adjoint).
struct EntrySrc {
  const int3* cands;      // (pair, slot_a, slot_b), or nullptr
  mrdem_contacts con;     // used when cands == nullptr
  int count_slot;         // counter holding the candidate count
  int64_t cap;
};

__device__ __forceinline__ bool load_entry(const HierDev& H, const EntrySrc& src, int64_t k,
                                           const int32_t* ab, int64_t n_pairs, int3& e) {
  if (src.cands) {
    e = src.cands[k];
    return true;
  }
  int p = src.con.pair[k];
  if (p < 0 || p >= n_pairs) return false;
  int A = ab[2 * p], B = ab[2 * p + 1];
  e = make_int3(p, H.tri_slot[H.tri_off[A] + src.con.tri_a[k]],
                H.tri_slot[H.tri_off[B] + src.con.tri_b[k]]);
  return true;
}

__device__ __forceinline__ int64_t entry_count(const EntrySrc& src, const unsigned long long* cnt) {
  int64_t n = src.cands ? (int64_t)cnt[src.count_slot] : (int64_t)*src.con.count;
  return n > src.cap ? src.cap : n;
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
                                                  EntrySrc src, const int32_t* __restrict__ ab,
                                                  int64_t n_pairs, double tau_override,
                                                  AccRec* acc, int64_t cap_acc, int* items_pt,
                                                  int* items_ee, int64_t cap_items,
                                                  int* fallback, int64_t cap_fallback,
                                                  unsigned long long* cnt,
                                                  unsigned long long* status) {
  int64_t n = entry_count(src, cnt);
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    int res = 0;
    unsigned mask = 0;
    int3 e = make_int3(0, 0, 0);
    if (k < n && load_entry(H, src, k, ab, n_pairs, e)) {
      PairXf X;
      load_pairxf(xf, e.x, X);
      F3 a0 = load_vertex(H, e.y, 0), a1 = load_vertex(H, e.y, 1), a2 = load_vertex(H, e.y, 2);
      F3 Pf[3] = {{0.f, 0.f, 0.f}, a1 - a0, a2 - a0};
      F3 Qf[3] = {xf_point(X, load_vertex(H, e.z, 0)) - a0, xf_point(X, load_vertex(H, e.z, 1)) - a0,
                  xf_point(X, load_vertex(H, e.z, 2)) - a0};
      double tau = tau_override > 0 ? tau_override : (double)X.tau;
      res = cand_float_stage(Pf, Qf, tau, X.margin, &mask);
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
    if (accept) {
      AccRec& r = acc[ai];
      const PairXf64& X64 = xf64[e.x];
      CandGeom g;
      cand_geom(H, X64, e, g);
      if (tau_override > 0) g.tau = tau_override;
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
// Adjoint on top of the closest points (see mrdem_forces.cu for the formulas).
// Scatter of one contact's gradient; must be called by all 32 lanes (the
// Gauss-Newton blocks are summed per pair within the warp).
constexpr int kGradThreads = 128;
__device__ __forceinline__ void grad_scatter(bool ok, const HierDev& H, const PairXf64& X64,
                                             int p, int sa, int sb, double d, D3 pa, D3 pb,
                                             const double* wa, const double* wb, const CandGeom& g,
                                             const double* __restrict__ poses,
                                             const double* __restrict__ mass, double k_s,
                                             double scale, float* dverts, double* dpose,
                                             double* jac, double (*sJ)[13]) {
  const int lane = lane_id();
  double J[12], h = 0.0;
  ok = ok && d <= 2.0 * X64.eps;
  if (ok) {
    const int A = X64.A, B = X64.B;
    const double e = X64.eps;
    double mu = 1.0 / (1.0 / mass[A] + 1.0 / mass[B]);
    double ks = k_s * sqrt(mu);
    D3 uA;
    if (d > 0.0) {
      uA = (1.0 / d) * (pa - pb);
    } else {
      D3 nn = cross(g.P[1] - g.P[0], g.P[2] - g.P[0]);
      uA = (-1.0 / sqrt(dot(nn, nn))) * nn;
    }
    const double* RA = X64.RA;
    auto mulA = [&](D3 v) {
      return D3{RA[0] * v.x + RA[1] * v.y + RA[2] * v.z, RA[3] * v.x + RA[4] * v.y + RA[5] * v.z,
                RA[6] * v.x + RA[7] * v.y + RA[8] * v.z};
    };
    D3 paw = mulA(pa + g.o), pbw = mulA(pb + g.o);
    paw = {paw.x + X64.tA[0], paw.y + X64.tA[1], paw.z + X64.tA[2]};
    pbw = {pbw.x + X64.tA[0], pbw.y + X64.tA[1], pbw.z + X64.tA[2]};
    D3 u = mulA(uA);
    double de = -ks * (1.0 - d / (2.0 * e)) * scale;
    D3 gv = de * u;
    if (dverts) {
      // A's body frame: R_A^T g = de uA; B's body frame: R_rel^T of that
      D3 gA = de * uA;
      const double* R = X64.R;
      D3 gB = {R[0] * gA.x + R[3] * gA.y + R[6] * gA.z, R[1] * gA.x + R[4] * gA.y + R[7] * gA.z,
               R[2] * gA.x + R[5] * gA.y + R[8] * gA.z};
      for (int v = 0; v < 3; ++v) {
        int ia = H.vid[v * H.stride + sa], ib = H.vid[v * H.stride + sb];
        atomicAdd(dverts + 3 * (int64_t)ia, (float)(wa[v] * gA.x));
        atomicAdd(dverts + 3 * (int64_t)ia + 1, (float)(wa[v] * gA.y));
        atomicAdd(dverts + 3 * (int64_t)ia + 2, (float)(wa[v] * gA.z));
        atomicAdd(dverts + 3 * (int64_t)ib, (float)(-wb[v] * gB.x));
        atomicAdd(dverts + 3 * (int64_t)ib + 1, (float)(-wb[v] * gB.y));
        atomicAdd(dverts + 3 * (int64_t)ib + 2, (float)(-wb[v] * gB.z));
      }
    }
    const double* tB = poses + 7 * (int64_t)B;
    D3 ra = paw - D3{X64.tA[0], X64.tA[1], X64.tA[2]};
    D3 rb = pbw - D3{tB[0], tB[1], tB[2]};
    if (dpose) {
      D3 t1 = cross(ra, gv), t2 = cross(rb, -1.0 * gv);
      double* oa = dpose + 6 * (int64_t)A;
      double* ob = dpose + 6 * (int64_t)B;
      atomicAdd(oa, gv.x); atomicAdd(oa + 1, gv.y); atomicAdd(oa + 2, gv.z);
      atomicAdd(oa + 3, t1.x); atomicAdd(oa + 4, t1.y); atomicAdd(oa + 5, t1.z);
      atomicAdd(ob, -gv.x); atomicAdd(ob + 1, -gv.y); atomicAdd(ob + 2, -gv.z);
      atomicAdd(ob + 3, t2.x); atomicAdd(ob + 4, t2.y); atomicAdd(ob + 5, t2.z);
    }
    D3 c1 = cross(ra, u), c2 = cross(rb, u);
    J[0] = u.x; J[1] = u.y; J[2] = u.z; J[3] = c1.x; J[4] = c1.y; J[5] = c1.z;
    J[6] = -u.x; J[7] = -u.y; J[8] = -u.z; J[9] = -c2.x; J[10] = -c2.y; J[11] = -c2.z;
    h = ks / (2.0 * e) * scale;
  }
  if (jac) {
    // group the warp's contacts by pair; each group's 78 distinct block
    // entries are summed by the lanes in turn and added once
    for (int q = 0; q < 12; ++q) sJ[lane][q] = ok ? J[q] : 0.0;
    sJ[lane][12] = ok ? h : 0.0;
    __syncwarp();
    unsigned pending = __ballot_sync(0xffffffffu, ok);
    int mykey = ok ? p : -1;
    while (pending) {
      int leader = __ffs(pending) - 1;
      int key = __shfl_sync(0xffffffffu, mykey, leader);
      unsigned grp = __ballot_sync(0xffffffffu, ok && mykey == key);
      pending &= ~grp;
      for (int e2 = lane; e2 < 78; e2 += 32) {
        int r = 0, rem = e2;
        while (rem >= 12 - r) { rem -= 12 - r; ++r; }
        int q = r + rem;
        double acc = 0.0;
        unsigned gm = grp;
        while (gm) {
          int l = __ffs(gm) - 1;
          gm &= gm - 1;
          acc += sJ[l][12] * sJ[l][r] * sJ[l][q];
        }
        double* o = jac + 144 * (int64_t)key;
        atomicAdd(o + 12 * r + q, acc);
        if (q != r) atomicAdd(o + 12 * q + r, acc);
      }
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kGradThreads) k_grad_select(
    HierDev H, const PairXf64* __restrict__ xf64, const AccRec* __restrict__ acc,
    const ItemRes* __restrict__ res_pt, const ItemRes* __restrict__ res_ee, mrdem_contacts con,
    const int32_t* __restrict__ ab, const double* __restrict__ poses,
    const double* __restrict__ mass, double k_s, double scale, float* dverts, double* dpose,
    double* jac, unsigned long long* cnt, int64_t cap_acc) {
  __shared__ double sJ[kGradThreads / 32][32][13];
  const int w = threadIdx.x >> 5;
  int64_t n = (int64_t)cnt[CNT_ACC];
  if (n > cap_acc) n = cap_acc;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    bool ok = false;
    int p = 0, sa = 0, sb = 0;
    double d = 0, wa[3] = {0, 0, 0}, wb[3] = {0, 0, 0};
    D3 pa = {0, 0, 0}, pb = {0, 0, 0};
    const AccRec* r = nullptr;
    if (k < n) {
      r = acc + k;
      const ItemRes* b = best_item(*r, res_pt, res_ee);
      if (b) {
        ok = true;
        d = sqrt(b->d2);
        pa = {b->pa[0], b->pa[1], b->pa[2]};
        pb = {b->pb[0], b->pb[1], b->pb[2]};
        for (int q = 0; q < 3; ++q) { wa[q] = b->wa[q]; wb[q] = b->wb[q]; }
        p = r->pair;
        int e = r->entry;
        int A = ab[2 * p], B = ab[2 * p + 1];
        sa = H.tri_slot[H.tri_off[A] + con.tri_a[e]];
        sb = H.tri_slot[H.tri_off[B] + con.tri_b[e]];
      }
    }
    CandGeom g;
    if (r) g = r->g;
    grad_scatter(ok, H, xf64[ok ? p : 0], p, sa, sb, d, pa, pb, wa, wb, g, poses, mass, k_s, scale,
                 dverts, dpose, jac, sJ[w]);
  }
}

// Full double test for the contacts the float stage left (crossing or nearly
// touching triangles).
__global__ void __launch_bounds__(kGradThreads) k_grad_fallback(
    HierDev H, const PairXf64* __restrict__ xf64, const int* __restrict__ list, mrdem_contacts con,
    const int32_t* __restrict__ ab, int64_t n_pairs, const double* __restrict__ poses,
    const double* __restrict__ mass, double k_s, double scale, float* dverts, double* dpose,
    double* jac, unsigned long long* cnt, int64_t cap) {
  __shared__ double sJ[kGradThreads / 32][32][13];
  const int w = threadIdx.x >> 5;
  int64_t n = (int64_t)cnt[CNT_FALLBACK];
  if (n > cap) n = cap;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    bool ok = false;
    int p = 0, sa = 0, sb = 0;
    double d = 0, wa[3] = {0, 0, 0}, wb[3] = {0, 0, 0};
    D3 pa = {0, 0, 0}, pb = {0, 0, 0};
    CandGeom g;
    if (k < n) {
      int e = list[k];
      p = con.pair[e];
      if (p >= 0 && p < n_pairs) {
        int A = ab[2 * p], B = ab[2 * p + 1];
        sa = H.tri_slot[H.tri_off[A] + con.tri_a[e]];
        sb = H.tri_slot[H.tri_off[B] + con.tri_b[e]];
        cand_geom(H, xf64[p], make_int3(p, sa, sb), g);
        TriTriResult<double> r = tri_tri_distance(g.P, g.Q);
        d = r.d; pa = r.pa; pb = r.pb;
        for (int q = 0; q < 3; ++q) { wa[q] = r.wa[q]; wb[q] = r.wb[q]; }
        ok = true;
      }
    }
    grad_scatter(ok, H, xf64[ok ? p : 0], p, sa, sb, d, pa, pb, wa, wb, g, poses, mass, k_s, scale,
                 dverts, dpose, jac, sJ[w]);
  }
}

// ---------------------------------------------------------------------------
// launchers

int closest_float_stage(mrdem_ctx* c, const mrdem_hier* hier, const EntrySrc& src,
                        const int32_t* ab, int64_t n_pairs, double tau_override, int* fallback,
                        int64_t cap_fallback, cudaStream_t s) {
  cudaMemsetAsync(c->counters + CNT_ACC, 0, sizeof(unsigned long long) * 3, s);
  cudaMemsetAsync(c->counters + CNT_FALLBACK, 0, sizeof(unsigned long long), s);
  k_cp_float<<<c->n_sms * 8, 128, 0, s>>>(hier->dev, c->xf, c->xf64, src, ab, n_pairs,
                                          tau_override, c->acc, c->cap_cands, c->items_pt,
                                          c->items_ee, c->cap_items, fallback, cap_fallback,
                                          c->counters, c->status);
  int ib = c->n_sms * 8;
  k_cp_items<<<ib, 256, 0, s>>>(c->acc, c->items_pt, CNT_PT, c->cap_items, c->res_pt, c->counters);
  k_cp_items<<<ib, 256, 0, s>>>(c->acc, c->items_ee, CNT_EE, c->cap_items, c->res_ee, c->counters);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_exact_fp32(mrdem_ctx* c, const mrdem_hier* hier, const mrdem_contacts* out,
                      cudaStream_t s) {
  EntrySrc src{};
  src.cands = c->cands;
  src.count_slot = CNT_CANDS;
  src.cap = c->cap_cands;
  int* fallback = reinterpret_cast<int*>(c->level_list[0]);  // free once the tiles are done
  int st;
  {
    ProfScope ps(c, K_EXACT, s);
    st = closest_float_stage(c, hier, src, nullptr, 0, -1.0, fallback, c->cap_level, s);
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

int launch_grad_closest(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                        const double* poses, const mrdem_contacts* con, const double* mass,
                        double k_s, double scale, float* dverts, double* dpose, double* jac,
                        cudaStream_t s) {
  EntrySrc src{};
  src.cands = nullptr;
  src.con = *con;
  src.cap = con->capacity;
  int* fallback = reinterpret_cast<int*>(c->level_list[1]);
  ProfScope ps(c, K_GRAD, s);
  int st = closest_float_stage(c, hier, src, ab, n_pairs, 1e300, fallback, c->cap_level, s);
  if (st) return st;
  k_grad_select<<<c->n_sms * 8, kGradThreads, 0, s>>>(hier->dev, c->xf64, c->acc, c->res_pt,
                                                       c->res_ee, *con, ab, poses, mass, k_s,
                                                       scale, dverts, dpose, jac, c->counters,
                                                       c->cap_cands);
  k_grad_fallback<<<c->n_sms * 2, kGradThreads, 0, s>>>(hier->dev, c->xf64, fallback, *con, ab,
                                                         n_pairs, poses, mass, k_s, scale, dverts,
                                                         dpose, jac, c->counters, c->cap_level);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
