// mrdem_step.cu -- kernels of the implicit time step (Algorithm 3) around the
// contact detection and forces: the uniform-grid broad phase that lists the
// candidate particle pairs, the rigid-body pose update, and the Picard update
// of the velocities with its convergence measure.
//
// Broad phase, one call:
//   k_bp_bounds   one block: smallest centre per axis, largest and smallest
//                 bounding radius -> size classes and their cell sides;
//                 flags non-finite input;
//   k_bp_cells    class, cell and bucket of every particle; bucket and
//                 class sizes;
//   k_bp_scan     exclusive scans of the bucket and class sizes -> starts;
//   k_bp_scatter  particles grouped by bucket and by class (the starts end
//                 as the ends);
//   k_bp_count    a thread per particle: its candidates j > i, class by
//                 class, in the cells of that class's grid that its search
//                 box meets (or the class's particles, when fewer);
//   k_bp_scan     exclusive scan of the counts -> output offsets and the total;
//   k_bp_write    if the total fits: each particle writes its candidates at its
//                 offset and sorts them by j, so the list is ordered by (i, j)
//                 whatever order the atomics grouped the buckets in.
// The particles' own FP64 arithmetic lives in mrdem_step.cuh.
#include <cooperative_groups.h>
#include <cstddef>
#include <cuda_runtime.h>

#include "mrdem_device.cuh"
#include "mrdem_split.cuh"
#include "mrdem_step.cuh"

namespace cg = cooperative_groups;

namespace mrdem {

namespace {

constexpr int kBoundsThreads = 1024;
constexpr int kThreads = 256;

__device__ __forceinline__ double dmax_nan(double a, double b) {
  if (a != a) return a;
  if (b != b) return b;
  return a > b ? a : b;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = dmax_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(kBoundsThreads) k_bp_bounds(BroadIn in, BroadGrid* grid,
                                                              unsigned long long* status) {
  wait_prior_grid();
  __shared__ double part[5][32];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, rb = 0.0, rmin = INFINITY;
  bool bad = false;
  for (int32_t i = threadIdx.x; i < in.n; i += blockDim.x) {
    const double* c = in.poses + (int64_t)7 * i;
    for (int k = 0; k < 3; ++k) {
      const double x = c[k];
      if (!isfinite(x)) bad = true;
      lo[k] = fmin(lo[k], x);
    }
    const double R = in.bound[i], r = in.radius[i];
    if (!(R >= 0.0) || !isfinite(R) || !(r >= 0.0) || !isfinite(r)) bad = true;
    rb = fmax(rb, R);
    rmin = fmin(rmin, R);
  }
  // mins of the three coordinates and of R, max of R
  double v[5] = {warp_min(lo[0]), warp_min(lo[1]), warp_min(lo[2]), warp_max(rb), warp_min(rmin)};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 5; ++k) part[k][warp] = v[k];
  bad = __syncthreads_or(bad) != 0;
  if (warp == 0) {
    for (int k = 0; k < 5; ++k) {
      const bool is_max = k == 3;
      double x = lane < nw ? part[k][lane] : (is_max ? 0.0 : INFINITY);
      v[k] = is_max ? warp_max(x) : warp_min(x);
    }
    if (lane == 0) {
      BroadGrid g;
      g.lo[0] = v[0];
      g.lo[1] = v[1];
      g.lo[2] = v[2];
      g.r_max = v[3];
      g.classes = bp_classes(v[3], v[4]);
      bool ok = !bad && isfinite(g.r_max);
      for (int k = 0; k < kMaxClasses; ++k) {
        g.h[k] = bp_cell_side(g.r_max, k);
        g.inv_h[k] = 1.0 / g.h[k];
        ok = ok && isfinite(g.h[k]) && g.h[k] > 0.0;
      }
      g.bad = ok ? 0 : 1;
      *grid = g;
      if (g.bad) atomicExch(status + ST_NONFINITE, 1ull);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_bp_cells(BroadIn in, const BroadGrid* grid,
                                                       BroadWork w) {
  wait_prior_grid();
  const BroadGrid g = *grid;
  if (g.bad) return;
  const int32_t step = gridDim.x * blockDim.x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < in.n; i += step) {
    const BroadCell cl = bp_cell_of(in, g, i, w.log2_t);
    w.cell[i] = cl;
    atomicAdd(w.bucket_end + cl.b, 1);
    atomicAdd(w.class_end + cl.k, 1);
  }
}

__global__ void __launch_bounds__(1024) k_bp_scan(int32_t* cnt, int64_t n, int64_t* total) {
  wait_prior_grid();
  block_exclusive_scan(cnt, n, total);
}

__global__ void __launch_bounds__(kThreads) k_bp_scatter(BroadIn in, const BroadGrid* grid,
                                                         BroadWork w) {
  wait_prior_grid();
  if (grid->bad) return;
  const int32_t step = gridDim.x * blockDim.x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < in.n; i += step) {
    const BroadCell cl = w.cell[i];
    w.order[atomicAdd(w.bucket_end + cl.b, 1)] = i;
    w.class_order[atomicAdd(w.class_end + cl.k, 1)] = i;
  }
}

// Candidates per particle: a warp per particle, its lanes sharing the
// particle's cells (a big particle's search box holds many cells of the
// small particles' grids).
__global__ void __launch_bounds__(kThreads) k_bp_count(BroadIn in, const BroadGrid* grid,
                                                       BroadWork w, int32_t* cnt) {
  wait_prior_grid();
  const BroadGrid g = *grid;
  const int lane = threadIdx.x & 31;
  const int32_t warps = gridDim.x * (blockDim.x >> 5);
  for (int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < in.n; i += warps) {
    int32_t c = g.bad ? 0 : bp_visit_lane(in, g, w, i, lane, 32, [](int32_t, double) {});
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) cnt[i] = c;
  }
}

// The pairs (i, j), j > i, of each particle at its offset, in increasing j:
// a warp per particle; each lane writes its candidates after those of the
// lanes before it, then the warp puts them in order by rank (a particle has
// a few dozen candidates in a packing; more than kBpSortMax are ordered by
// one lane).
constexpr int kBpSortMax = 256;
__global__ void __launch_bounds__(kThreads) k_bp_write(BroadIn in, const BroadGrid* grid,
                                                       BroadWork w, const int32_t* off,
                                                       const int64_t* count, int64_t cap,
                                                       int32_t* pairs, double* pair_eps) {
  wait_prior_grid();
  __shared__ int32_t sj[kThreads / 32][kBpSortMax];
  __shared__ double se[kThreads / 32][kBpSortMax];
  const int64_t total = *count;
  const BroadGrid g = *grid;
  if (g.bad || total > cap) return;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int32_t warps = gridDim.x * (blockDim.x >> 5);
  for (int32_t i = blockIdx.x * (blockDim.x >> 5) + wq; i < in.n; i += warps) {
    const int64_t o = off[i];
    const int64_t m = (i + 1 < in.n ? (int64_t)off[i + 1] : total) - o;
    // this lane's share, then its place after the lanes before it
    const int32_t mine = bp_visit_lane(in, g, w, i, lane, 32, [](int32_t, double) {});
    int32_t incl = mine;
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const int32_t got_all = __shfl_sync(0xffffffffu, incl, 31);
    int64_t k = incl - mine;
    bp_visit_lane(in, g, w, i, lane, 32, [&](int32_t j, double e) {
      if (k < m) {
        pairs[2 * (o + k) + 1] = j;
        pair_eps[o + k] = e;
      }
      ++k;
    });
    const int64_t got = got_all < m ? got_all : m;
    __syncwarp();
    if (got <= kBpSortMax) {
      // order by j: each entry goes to its rank (the j are distinct)
      for (int64_t a = lane; a < got; a += 32) {
        sj[wq][a] = pairs[2 * (o + a) + 1];
        se[wq][a] = pair_eps[o + a];
      }
      __syncwarp();
      for (int64_t a = lane; a < got; a += 32) {
        const int32_t j = sj[wq][a];
        int32_t r = 0;
        for (int64_t q = 0; q < got; ++q) r += sj[wq][q] < j;
        pairs[2 * (o + r)] = i;
        pairs[2 * (o + r) + 1] = j;
        pair_eps[o + r] = se[wq][a];
      }
      __syncwarp();
    } else if (lane == 0) {
      for (int64_t a = o + 1; a < o + got; ++a) {
        const int32_t j = pairs[2 * a + 1];
        const double e = pair_eps[a];
        int64_t b = a - 1;
        while (b >= o && pairs[2 * b + 1] > j) {
          pairs[2 * (b + 1) + 1] = pairs[2 * b + 1];
          pair_eps[b + 1] = pair_eps[b];
          --b;
        }
        pairs[2 * (b + 1) + 1] = j;
        pair_eps[b + 1] = e;
      }
      for (int64_t a = o; a < o + got; ++a) pairs[2 * a] = i;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kThreads) k_move_poses(int32_t n, const double* poses0,
                                                         const double* vel, double dt,
                                                         double* poses) {
  wait_prior_grid();
  const int32_t step = gridDim.x * blockDim.x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    double p0[7], v[6], out[7];
    for (int k = 0; k < 7; ++k) p0[k] = poses0[(int64_t)7 * i + k];
    for (int k = 0; k < 6; ++k) v[k] = vel[(int64_t)6 * i + k];
    move_pose(p0, v, dt, out);
    for (int k = 0; k < 7; ++k) poses[(int64_t)7 * i + k] = out[k];
  }
}

__global__ void __launch_bounds__(kThreads) k_twist_grad(int32_t n, const double* twist,
                                                         const double* g, double* out) {
  wait_prior_grid();
  const int32_t step = gridDim.x * blockDim.x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    double tw[6], gi[6], o[6];
    for (int k = 0; k < 6; ++k) {
      tw[k] = twist[(int64_t)6 * i + k];
      gi[k] = g[(int64_t)6 * i + k];
    }
    twist_gradient(tw, gi, o);
    for (int k = 0; k < 6; ++k) out[(int64_t)6 * i + k] = o[k];
  }
}

struct Gravity {
  double g[3];
};

__global__ void __launch_bounds__(kThreads) k_picard(int32_t n, const double* vel0,
                                                     const double* ft, const double* mass,
                                                     const double* inertia, Gravity grav,
                                                     double dt, double* vel,
                                                     unsigned long long* norms) {
  wait_prior_grid();
  double cmax = 0.0, smax = 0.0;
  const int32_t step = gridDim.x * blockDim.x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    double v0[6], f[6], guess[6], out[6], c, s;
    for (int k = 0; k < 6; ++k) {
      v0[k] = vel0[(int64_t)6 * i + k];
      f[k] = ft[(int64_t)6 * i + k];
      guess[k] = vel[(int64_t)6 * i + k];
    }
    picard_velocity(v0, f, mass[i], inertia[i], grav.g, dt, guess, out, &c, &s);
    for (int k = 0; k < 6; ++k) vel[(int64_t)6 * i + k] = out[k];
    cmax = dmax_nan(cmax, c);
    smax = dmax_nan(smax, s);
  }
  cmax = warp_max(cmax);
  smax = warp_max(smax);
  if ((threadIdx.x & 31) == 0) {
    // non-negative doubles (and NaN, with its sign cleared) order like their bits
    atomicMax(norms, (unsigned long long)__double_as_longlong(fabs(cmax)));
    atomicMax(norms + 1, (unsigned long long)__double_as_longlong(fabs(smax)));
  }
}

// World FP64 corners of fine triangle `tri` of particle i.
__device__ __forceinline__ bool world_triangle(const HierDev& H, const double* poses, int i,
                                               int tri, V3<double> T[3], V3<double>* t) {
  if (tri < 0 || tri >= H.tri_off[i + 1] - H.tri_off[i]) return false;
  const int slot = H.tri_slot[H.tri_off[i] + tri];
  V3<double> V[3];
  load_tri64(H, slot, V);
  const double* p = poses + (int64_t)7 * i;
  double R[9];
  quat_matrix(p + 3, R);
  *t = {p[0], p[1], p[2]};
  for (int k = 0; k < 3; ++k) T[k] = pose_point(R, p, V[k]);
  return true;
}

// Contact Hessian blocks: a warp takes 32 contacts; each lane finds its
// contact's closest points (screened in float, FP64 where it decides) and
// stores the block in compact form (HessRep, mrdem_step.cuh) in shared
// memory; then each half-warp forms the reduced 9x9 block (45 entries of
// the upper triangle, three per lane) of its 16 contacts, summing runs of
// contacts of the same pair (detection lists a pair's contacts together) in
// registers, and adds each run's sums to the pair's 12x12 block, signed,
// with one atomic per entry.
constexpr int kHessWarps = 2;
// The reduced block H9 is symmetric: its 45 entries (p <= q) as (p << 4) | q,
// row by row (entry e of row p at p*9 - p(p-1)/2 + q - p).
__constant__ unsigned char kHessUpper9[45] = {
    0x00, 0x01, 0x02, 0x03, 0x04, 0x05, 0x06, 0x07, 0x08,
    0x11, 0x12, 0x13, 0x14, 0x15, 0x16, 0x17, 0x18,
    0x22, 0x23, 0x24, 0x25, 0x26, 0x27, 0x28,
    0x33, 0x34, 0x35, 0x36, 0x37, 0x38,
    0x44, 0x45, 0x46, 0x47, 0x48,
    0x55, 0x56, 0x57, 0x58,
    0x66, 0x67, 0x68,
    0x77, 0x78,
    0x88};
__device__ __forceinline__ int hess9_index(int p, int q) {
  if (p > q) { const int t = p; p = q; q = t; }
  return p * 9 - (p * (p - 1)) / 2 + (q - p);
}

// The compact block in double-float: the same layout as HessRep with a
// double-float (two floats, 8 bytes) in place of each double, so that the
// lane that built a contact's HessRep in shared memory converts it field by
// field in place (integer split of each double, mrdem_split.cuh).  The
// entries are then formed in double-float on the FP32 units: the FP64 rate
// of this part is about 1/61 of its FP32 rate (measured), and the entry
// phase was bound by it.
struct HessRepDD {
  dd u[3], r[3];
  dd rA[3], rB[3];
  dd G[2][3];
  dd K[3];
  dd a, b;
  dd g[3];
  dd zu[9];
  dd N[2][9];
  int nq;
  int own[2];
};
union HessSlot {
  HessRep d;
  HessRepDD f;
};
static_assert(sizeof(dd) == sizeof(double), "double-float slot size");
static_assert(offsetof(HessRep, N) == offsetof(HessRepDD, N), "HessRepDD layout");
static_assert(offsetof(HessRep, nq) == offsetof(HessRepDD, nq), "HessRepDD layout");
__device__ __forceinline__ void hess_rep_to_dd(HessSlot& s) {
  // each slot read as a double, then written back as a double-float
#define MRDEM_SPLIT_FIELD(x) s.f.x = split_double(s.d.x)
  for (int k = 0; k < 3; ++k) {
    MRDEM_SPLIT_FIELD(rA[k]);
    MRDEM_SPLIT_FIELD(rB[k]);
    MRDEM_SPLIT_FIELD(K[k]);
    MRDEM_SPLIT_FIELD(g[k]);
  }
  MRDEM_SPLIT_FIELD(a);
  MRDEM_SPLIT_FIELD(b);
  for (int k = 0; k < 9; ++k) {
    MRDEM_SPLIT_FIELD(zu[k]);
    MRDEM_SPLIT_FIELD(N[0][k]);
    MRDEM_SPLIT_FIELD(N[1][k]);
  }
#undef MRDEM_SPLIT_FIELD
}

// Entry (p, q) of the reduced block (the formula of hessian_entry9) with
// value selects in place of its branches on the row kind, since the lanes
// of a warp hold different entries.
__device__ __forceinline__ void hess9_zrow_sel(const HessRepDD& h, int p, dd z[3]) {
  const int blk = p / 3, c = p % 3;
  const bool a = blk == 1;
  const dd q0 = a ? h.rA[0] : h.rB[0], q1 = a ? h.rA[1] : h.rB[1];
  const dd q2 = a ? h.rA[2] : h.rB[2];
  const dd zero(0.f, 0.f), one(1.f, 0.f);
  const dd x0 = c == 0 ? zero : (c == 1 ? q2 : -q1);
  const dd x1 = c == 0 ? -q2 : (c == 1 ? zero : q0);
  const dd x2 = c == 0 ? q1 : (c == 1 ? -q0 : zero);
  const bool t = blk == 0;
  z[0] = t ? (c == 0 ? one : zero) : x0;
  z[1] = t ? (c == 1 ? one : zero) : x1;
  z[2] = t ? (c == 2 ? one : zero) : x2;
}
__device__ __forceinline__ dd hess9_entry_sel(const HessRepDD& h, int p, int q) {
  dd zp[3], zq[3];
  hess9_zrow_sel(h, p, zp);
  hess9_zrow_sel(h, q, zq);
  dd v = h.a * h.zu[p] * h.zu[q] + h.b * (zp[0] * zq[0] + zp[1] * zq[1] + zp[2] * zq[2]);
  if (h.nq > 0) {  // the same for every lane of a contact
    const dd np0 = h.N[0][p], nq0 = h.N[0][q];
    const dd np1 = h.N[1][p], nq1 = h.N[1][q];  // zero beyond nq
    v = v - h.b * (np0 * h.K[0] * nq0 + np0 * h.K[1] * nq1 + np1 * h.K[1] * nq0 +
                   np1 * h.K[2] * nq1);
  }
  const int bp = p / 3, ii = p % 3, jj = q % 3;
  const bool rot = bp == q / 3 && bp > 0;
  const bool a = bp == 1;
  const dd r0 = a ? h.rA[0] : h.rB[0], r1 = a ? h.rA[1] : h.rB[1];
  const dd r2 = a ? h.rA[2] : h.rB[2];
  const dd ri = ii == 0 ? r0 : (ii == 1 ? r1 : r2), rj = jj == 0 ? r0 : (jj == 1 ? r1 : r2);
  const dd gi = h.g[ii], gj = h.g[jj];
  const dd gr = h.g[0] * r0 + h.g[1] * r1 + h.g[2] * r2;
  const dd sym = gi * rj + gj * ri;
  const dd corr = dd(0.5f * sym.hi, 0.5f * sym.lo) - (ii == jj ? gr : dd(0.f, 0.f));
  return rot ? v + corr : v;
}

__global__ void __launch_bounds__(kHessWarps * 32, 2) k_hessian(HierDev H, const int32_t* ab,
                                                             const double* eps,
                                                             const double* poses,
                                                             const double* mass, double k_s,
                                                             mrdem_contacts c, int64_t n_pairs,
                                                             double* blocks,
                                                             unsigned long long* skipped) {
  wait_prior_grid();
  __shared__ HessSlot rep[kHessWarps][32];
  __shared__ int rpair[kHessWarps][32];
  __shared__ double sacc[kHessWarps][2][45];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t n = *c.count;
  if (n > c.capacity) n = c.capacity;
  const int64_t step = (int64_t)gridDim.x * kHessWarps * 32;
  unsigned long long parallel = 0;
  for (int64_t base = ((int64_t)blockIdx.x * kHessWarps + w) * 32; base < n; base += step) {
    const int64_t k = base + lane;
    int pr = -1;
    if (k < n) {
      const int p = c.pair[k];
      if (p >= 0 && p < n_pairs) {
        const int A = ab[2 * p], B = ab[2 * p + 1];
        V3<double> TA[3], TB[3], tA, tB;
        if (A >= 0 && A < H.n_particles && B >= 0 && B < H.n_particles &&
            world_triangle(H, poses, A, c.tri_a[k], TA, &tA) &&
            world_triangle(H, poses, B, c.tri_b[k], TB, &tB)) {
          const double mA = mass[A], mB = mass[B];
          const double ks = k_s * sqrt(mA * mB / (mA + mB));
          const int st = contact_hessian_rep(TA, TB, tA, tB, ks, eps[p], &rep[w][lane].d);
          if (st == 0) {
            pr = p;
            hess_rep_to_dd(rep[w][lane]);
          }
          else if (st == 2) ++parallel;
        }
      }
    }
    rpair[w][lane] = pr;
    __syncwarp();
    // each half-warp takes 16 of the warp's contacts in order; a lane holds
    // the reduced entries e = hl, hl + 16, hl + 32 of its half's contacts
    // (45 entries over 16 lanes: three rounds, 94 % of the lanes busy)
    const int half = lane >> 4, hl = lane & 15;
    const unsigned hmask = half ? 0xffff0000u : 0x0000ffffu;
    int ep[3], eq[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int e = hl + 16 * m;
      const int c = e < 45 ? kHessUpper9[e] : 0;
      ep[m] = e < 45 ? c >> 4 : -1;
      eq[m] = c & 15;
    }
    dd acc[3] = {dd(0.f, 0.f), dd(0.f, 0.f), dd(0.f, 0.f)};
    int cur = -1;
    // a pair's run: the 45 sums through shared memory, then the 144 entries
    // of its block, signed (B's translation rows are minus A's)
    auto flush = [&]() {
      double* o = blocks + 144 * (int64_t)cur;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (ep[m] >= 0) sacc[w][half][hl + 16 * m] = to_double(acc[m]);
        acc[m] = dd(0.f, 0.f);
      }
      __syncwarp(hmask);
      for (int x = hl; x < 144; x += 16) {
        int p9, q9;
        double si, sj;
        hess_map(x / 12, &p9, &si);
        hess_map(x % 12, &q9, &sj);
        atomicAdd(o + x, si * sj * sacc[w][half][hess9_index(p9, q9)]);
      }
      __syncwarp(hmask);
    };
    for (int kk = 0; kk < 16; ++kk) {
      const int ci = 16 * half + kk;
      const int p = rpair[w][ci];  // the same on every lane of the half
      if (p != cur) {
        if (cur >= 0) flush();
        cur = p;
      }
      if (p < 0) continue;
      const HessRepDD& h = rep[w][ci].f;
#pragma unroll
      for (int m = 0; m < 3; ++m)
        if (ep[m] >= 0) acc[m] = acc[m] + hess9_entry_sel(h, ep[m], eq[m]);
    }
    if (cur >= 0) flush();
    __syncwarp();
  }
  if (skipped && parallel) atomicAdd(skipped, parallel);
}

// ---- Newton's method: residual, and a Jacobi-preconditioned conjugate
// gradient solve of (M/dt + dt K) x = b with K the pair blocks

__global__ void __launch_bounds__(kThreads) k_residual(int32_t n, const double* vel0,
                                                       const double* vel, const double* ft,
                                                       const double* mass,
                                                       const double* inertia, Gravity grav,
                                                       double dt, double* res,
                                                       unsigned long long* norms) {
  wait_prior_grid();
  double rmax = 0.0, smax = 0.0;
  const int32_t step = gridDim.x * blockDim.x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    double v0[6], v[6], f[6], out[6], a, b;
    for (int k = 0; k < 6; ++k) {
      v0[k] = vel0[(int64_t)6 * i + k];
      v[k] = vel[(int64_t)6 * i + k];
      f[k] = ft[(int64_t)6 * i + k];
    }
    newton_residual(v0, v, f, mass[i], inertia[i], grav.g, dt, out, &a, &b);
    for (int k = 0; k < 6; ++k) res[(int64_t)6 * i + k] = out[k];
    rmax = dmax_nan(rmax, a);
    smax = dmax_nan(smax, b);
  }
  rmax = warp_max(rmax);
  smax = warp_max(smax);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(norms, (unsigned long long)__double_as_longlong(fabs(rmax)));
    atomicMax(norms + 1, (unsigned long long)__double_as_longlong(fabs(smax)));
  }
}

__global__ void __launch_bounds__(kThreads) k_vel_axpy(int64_t m, double a, const double* x,
                                                       const double* y, double* out) {
  wait_prior_grid();
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += step)
    out[i] = y[i] + a * x[i];
}

struct CgState {
  int32_t done, iters, breakdown, pad;
};

// Conjugate-gradient working set: vectors of 6n unknowns (x is the caller's
// output), and per iteration k the scalars rz[k] = r.z, pap[k] = p.Ap and
// rr[k] = r.r, summed with atomics.
struct CgView {
  double *x, *r, *z, *p, *ap, *diag;
  double *rz, *pap, *rr;
  CgState* st;
  const double* mass;
  const double* inertia;
  double dt;
  int32_t n;
};

__device__ __forceinline__ double view_mdt(const CgView& v, int64_t i) {
  return cg_mdt(v.mass, v.inertia, v.dt, i);
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// The whole solve in one cooperative launch (every block resident, grid-wide
// barriers between the phases), so that an iteration costs a few barriers
// instead of six kernel launches, and the loop stops on the device when the
// residual is small enough.  Phases of iteration k: A p (the M/dt part, then
// the pair blocks' share with atomics), p.Ap, the step (x, r, z, r.z, r.r),
// the stopping test (one thread), the next direction.  Sums of one phase are
// taken with atomics into the iteration's own scalar slots.
// Values other blocks wrote in an earlier phase are read past the SM's L1
// (__ldcg), which is not kept coherent with other SMs' writes.
__device__ __forceinline__ double view_precond(const CgView& v, int64_t i) {
  return cg_precond(__ldcg(v.diag + i), view_mdt(v, i));  // an indefinite diagonal: M/dt
}

__device__ __forceinline__ void grid_sum(double* dst, double x) {
  x = warp_sum_d(x);
  if ((threadIdx.x & 31) == 0) atomicAdd(dst, x);
}

__global__ void __launch_bounds__(kThreads) k_cg_coop(CgView v, const double* rhs, int64_t n_pairs,
                                                      const int32_t* ab, const double* blocks,
                                                      int max_iter, double tol2, double* info) {
  cg::grid_group grid = cg::this_grid();
  const int64_t m = (int64_t)6 * v.n;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  volatile CgState* st = v.st;
  // x = 0, r = rhs, diagonal of M/dt + dt K
  for (int64_t i = t0; i < m; i += step) {
    v.x[i] = 0.0;
    v.r[i] = rhs[i];
    v.diag[i] = view_mdt(v, i);
  }
  grid.sync();
  for (int64_t q = t0; q < n_pairs; q += step) {
    const int A = ab[2 * q], B = ab[2 * q + 1];
    if (A < 0 || A >= v.n || B < 0 || B >= v.n) continue;
    double da[6], db[6];
    cg_pair_diag(blocks + 144 * q, v.dt, da, db);
    for (int k = 0; k < 6; ++k) {
      atomicAdd(v.diag + (int64_t)6 * A + k, da[k]);
      atomicAdd(v.diag + (int64_t)6 * B + k, db[k]);
    }
  }
  grid.sync();
  {
    double rz = 0.0, rr = 0.0;
    for (int64_t i = t0; i < m; i += step) {
      const double r = v.r[i], z = r / view_precond(v, i);
      v.z[i] = z;
      v.p[i] = z;
      rz += r * z;
      rr += r * r;
    }
    grid_sum(v.rz, rz);
    grid_sum(v.rr, rr);
  }
  grid.sync();
  if (lead && __ldcg(v.rr) <= 0.0) { st->done = 1; st->iters = 0; }
  grid.sync();
  for (int k = 0; k < max_iter; ++k) {
    if (st->done) break;  // read after a barrier: the same on every thread
    for (int64_t i = t0; i < m; i += step) v.ap[i] = view_mdt(v, i) * v.p[i];
    grid.sync();
    for (int64_t q = t0; q < n_pairs; q += step) {
      const int A = ab[2 * q], B = ab[2 * q + 1];
      if (A < 0 || A >= v.n || B < 0 || B >= v.n) continue;
      double ya[6], yb[6], pa[6], pb[6];
      for (int c = 0; c < 6; ++c) {
        pa[c] = __ldcg(v.p + (int64_t)6 * A + c);
        pb[c] = __ldcg(v.p + (int64_t)6 * B + c);
      }
      cg_pair_apply(blocks + 144 * q, pa, pb, v.dt, ya, yb);
      for (int c = 0; c < 6; ++c) {
        atomicAdd(v.ap + (int64_t)6 * A + c, ya[c]);
        atomicAdd(v.ap + (int64_t)6 * B + c, yb[c]);
      }
    }
    grid.sync();
    {
      double s = 0.0;
      for (int64_t i = t0; i < m; i += step) s += v.p[i] * __ldcg(v.ap + i);
      grid_sum(v.pap + k, s);
    }
    grid.sync();
    const double pap = __ldcg(v.pap + k);
    if (!(pap > 0.0)) {
      // not positive definite along p: stop; negative curvature along the
      // first direction still gives a step along it, so x is not left at 0
      if (k == 0 && pap < 0.0) {
        const double a = __ldcg(v.rz) / -pap;
        for (int64_t i = t0; i < m; i += step) v.x[i] += a * v.p[i];
      }
      if (lead) { st->done = 1; st->breakdown = 1; st->iters = k; }
      break;  // every thread sees the same pap
    }
    {
      const double alpha = __ldcg(v.rz + k) / pap;
      double rz = 0.0, rr = 0.0;
      for (int64_t i = t0; i < m; i += step) {
        v.x[i] += alpha * v.p[i];
        const double r = v.r[i] - alpha * __ldcg(v.ap + i);
        const double z = r / view_precond(v, i);
        v.r[i] = r;
        v.z[i] = z;
        rz += r * z;
        rr += r * r;
      }
      grid_sum(v.rz + k + 1, rz);
      grid_sum(v.rr + k + 1, rr);
    }
    grid.sync();
    if (__ldcg(v.rr + k + 1) <= tol2 * __ldcg(v.rr)) {
      if (lead) { st->done = 1; st->iters = k + 1; }
      break;  // every thread sees the same sums
    }
    const double beta = __ldcg(v.rz + k + 1) / __ldcg(v.rz + k);
    for (int64_t i = t0; i < m; i += step) v.p[i] = v.z[i] + beta * v.p[i];
    grid.sync();
  }
  if (lead) {
    const int it = st->done ? st->iters : max_iter;
    info[0] = (double)it;
    const double r0 = __ldcg(v.rr), ri = __ldcg(v.rr + it);
    info[1] = r0 > 0.0 ? sqrt(ri / r0) : 0.0;
    info[2] = (double)st->breakdown;
    info[3] = sqrt(r0);
  }
}

// ---- contacts of a cached candidate list (the active set kept across the
// iterations of one step): exact FP64 distance of each listed triangle pair
// at the current poses, kept when d <= 2 eps; two passes around a scan so the
// output keeps the list's order.

struct RefineRec {
  double d, pa[3], pb[3];
};

__global__ void __launch_bounds__(kThreads) k_refine(HierDev H, const int32_t* ab,
                                                     const double* eps, const double* poses,
                                                     mrdem_contacts cand, int64_t n_pairs,
                                                     RefineRec* rec, int32_t* keep) {
  wait_prior_grid();
  int64_t n = *cand.count;
  if (n > cand.capacity) n = cand.capacity;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += step) {
    int32_t ok = 0;
    const int p = cand.pair[k];
    if (p >= 0 && p < n_pairs) {
      const int A = ab[2 * p], B = ab[2 * p + 1];
      V3<double> TA[3], TB[3], tA, tB;
      if (A >= 0 && A < H.n_particles && B >= 0 && B < H.n_particles &&
          world_triangle(H, poses, A, cand.tri_a[k], TA, &tA) &&
          world_triangle(H, poses, B, cand.tri_b[k], TB, &tB)) {
        const TriTriResult<double> t = tri_tri_distance<double>(TA, TB);
        if (t.d <= 2.0 * eps[p]) {
          ok = 1;
          RefineRec r;
          r.d = t.d;
          r.pa[0] = t.pa.x; r.pa[1] = t.pa.y; r.pa[2] = t.pa.z;
          r.pb[0] = t.pb.x; r.pb[1] = t.pb.y; r.pb[2] = t.pb.z;
          rec[k] = r;
        }
      }
    }
    keep[k] = ok;
  }
}

__global__ void __launch_bounds__(1024) k_refine_scan(int32_t* keep, const mrdem_contacts cand,
                                                      int64_t* total) {
  wait_prior_grid();
  int64_t n = *cand.count;
  if (n > cand.capacity) n = cand.capacity;
  block_exclusive_scan(keep, n, total);
}

// keep[] now holds exclusive offsets; entry k is kept when the next offset
// (or the total) is larger
__global__ void __launch_bounds__(kThreads) k_refine_write(mrdem_contacts cand,
                                                           const RefineRec* rec,
                                                           const int32_t* off, mrdem_contacts out,
                                                           unsigned long long* status) {
  wait_prior_grid();
  int64_t n = *cand.count;
  if (n > cand.capacity) n = cand.capacity;
  const int64_t total = *out.count;
  if (blockIdx.x == 0 && threadIdx.x == 0 && total > out.capacity)
    atomicMax(status + ST_REQ_CONTACTS, (unsigned long long)total);
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += step) {
    const int64_t o = off[k], next = k + 1 < n ? (int64_t)off[k + 1] : total;
    if (next == o || o >= out.capacity) continue;
    const RefineRec r = rec[k];
    out.pair[o] = cand.pair[k];
    out.tri_a[o] = cand.tri_a[k];
    out.tri_b[o] = cand.tri_b[k];
    out.dist[o] = r.d;
    for (int c = 0; c < 3; ++c) {
      out.point_a[3 * o + c] = r.pa[c];
      out.point_b[3 * o + c] = r.pb[c];
    }
  }
}

// Largest displacement of any point of a particle between two poses: the
// centre's plus the rotation angle times the bounding radius.
__global__ void __launch_bounds__(kThreads) k_motion(int32_t n, const double* ref,
                                                     const double* poses, const double* bound,
                                                     unsigned long long* out) {
  wait_prior_grid();
  double m = 0.0;
  const int32_t step = gridDim.x * blockDim.x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step)
    m = dmax_nan(m, particle_motion(ref + (int64_t)7 * i, poses + (int64_t)7 * i, bound[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0)
    atomicMax(out, (unsigned long long)__double_as_longlong(fabs(m)));
}

int ceil_log2(int64_t v) {
  int k = 0;
  while (((int64_t)1 << k) < v) ++k;
  return k;
}

int blocks_for(const mrdem_ctx* c, int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  const int64_t lim = (int64_t)c->n_sms * 8;
  return (int)(b < 1 ? 1 : (b < lim ? b : lim));
}

}  // namespace

// Broad-phase scratch: the grid record, then cell [n], order [n], class
// order [n], counts / offsets [n], bucket ends [2^log2_t], class ends.
static int ensure_broad(mrdem_ctx* c, int32_t n, BroadWork* w, BroadGrid** grid,
                        int32_t** cnt) {
  const int log2_t = ceil_log2(2 * (int64_t)n) < 6 ? 6 : ceil_log2(2 * (int64_t)n);
  const int64_t t = (int64_t)1 << log2_t;
  static_assert(sizeof(BroadGrid) <= 512, "grid record");
  const size_t bytes = 512 + sizeof(BroadCell) * (size_t)n + sizeof(int32_t) * (size_t)n * 3 +
                       sizeof(int32_t) * ((size_t)t + kMaxClasses) + 64;
  if (bytes > c->cap_broad) {
    cudaFree(c->broad_mem);
    c->broad_mem = nullptr;
    c->cap_broad = 0;
    if (cudaMalloc(&c->broad_mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->broad_mem = nullptr;
      return MRDEM_ERR_OOM;
    }
    c->cap_broad = bytes;
  }
  unsigned char* p = static_cast<unsigned char*>(c->broad_mem);
  *grid = reinterpret_cast<BroadGrid*>(p);
  p += 512;
  w->cell = reinterpret_cast<BroadCell*>(p);
  p += sizeof(BroadCell) * (size_t)n;
  w->order = reinterpret_cast<int32_t*>(p);
  p += sizeof(int32_t) * (size_t)n;
  w->class_order = reinterpret_cast<int32_t*>(p);
  p += sizeof(int32_t) * (size_t)n;
  *cnt = reinterpret_cast<int32_t*>(p);
  p += sizeof(int32_t) * (size_t)n;
  w->bucket_end = reinterpret_cast<int32_t*>(p);
  p += sizeof(int32_t) * (size_t)t;
  w->class_end = reinterpret_cast<int32_t*>(p);
  w->log2_t = log2_t;
  return MRDEM_OK;
}

int launch_broad_phase(mrdem_ctx* c, int32_t n, const double* poses, const double* bound,
                       const double* radius, double eps_rel, int32_t* pairs, double* pair_eps,
                       int64_t cap, int64_t* count, cudaStream_t s) {
  if (n == 0) {
    cudaMemsetAsync(count, 0, sizeof(int64_t), s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
  }
  BroadWork w;
  BroadGrid* grid = nullptr;
  int32_t* cnt = nullptr;
  int st = ensure_broad(c, n, &w, &grid, &cnt);
  if (st) return st;
  const BroadIn in{poses, bound, radius, eps_rel, n};
  const int64_t t = (int64_t)1 << w.log2_t;
  const int nb = blocks_for(c, n);
  ProfScope ps(c, K_BROAD, s);
  // bucket ends and class ends are contiguous
  cudaMemsetAsync(w.bucket_end, 0, sizeof(int32_t) * ((size_t)t + kMaxClasses), s);
  launch_after(k_bp_bounds, 1, kBoundsThreads, 0, s, in, grid, c->status);
  launch_after(k_bp_cells, nb, kThreads, 0, s, in, (const BroadGrid*)grid, w);
  launch_after(k_bp_scan, 1, 1024, 0, s, w.bucket_end, t, (int64_t*)nullptr);
  launch_after(k_bp_scan, 1, 1024, 0, s, w.class_end, (int64_t)kMaxClasses, (int64_t*)nullptr);
  launch_after(k_bp_scatter, nb, kThreads, 0, s, in, (const BroadGrid*)grid, w);
  // a warp per particle
  const int wb = (int)std::min<int64_t>(((int64_t)n + kThreads / 32 - 1) / (kThreads / 32),
                                        (int64_t)c->n_sms * 16);
  launch_after(k_bp_count, wb, kThreads, 0, s, in, (const BroadGrid*)grid, w, cnt);
  launch_after(k_bp_scan, 1, 1024, 0, s, cnt, (int64_t)n, count);
  launch_after(k_bp_write, wb, kThreads, 0, s, in, (const BroadGrid*)grid, w,
               (const int32_t*)cnt, (const int64_t*)count, cap, pairs, pair_eps);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_move_poses(mrdem_ctx* c, int32_t n, const double* poses0, const double* vel, double dt,
                      double* poses, cudaStream_t s) {
  if (n == 0) return MRDEM_OK;
  ProfScope ps(c, K_STEP, s);
  launch_after(k_move_poses, blocks_for(c, n), kThreads, 0, s, n, poses0, vel, dt, poses);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_twist_grad(mrdem_ctx* c, int32_t n, const double* twist, const double* g, double* out,
                      cudaStream_t s) {
  if (n == 0) return MRDEM_OK;
  ProfScope ps(c, K_STEP, s);
  launch_after(k_twist_grad, blocks_for(c, n), kThreads, 0, s, n, twist, g, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_picard_update(mrdem_ctx* c, int32_t n, const double* vel0, const double* ft,
                         const double* mass, const double* inertia, const double* gravity,
                         double dt, double* vel, double* norms, cudaStream_t s) {
  cudaMemsetAsync(norms, 0, 2 * sizeof(double), s);
  if (n > 0) {
    ProfScope ps(c, K_STEP, s);
    Gravity g{{gravity[0], gravity[1], gravity[2]}};
    launch_after(k_picard, blocks_for(c, n), kThreads, 0, s, n, vel0, ft, mass, inertia, g, dt,
                 vel, reinterpret_cast<unsigned long long*>(norms));
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_contact_hessian(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                           const double* eps, const double* poses, const mrdem_contacts* con,
                           const double* mass, double k_s, double* blocks, int64_t* skipped,
                           cudaStream_t s) {
  if (n_pairs == 0 || con->capacity == 0) return MRDEM_OK;
  ProfScope ps(c, K_HESSIAN, s);
  const int hb = kHessWarps * 32;
  const int64_t nb64 = (con->capacity + hb - 1) / hb;
  const int64_t lim = (int64_t)c->n_sms * 16;
  const int nb = (int)(nb64 < lim ? nb64 : lim);
  launch_after(k_hessian, nb, hb, 0, s, h->dev, ab, eps, poses, mass, k_s, *con, n_pairs,
               blocks, reinterpret_cast<unsigned long long*>(skipped));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_newton_residual(mrdem_ctx* c, int32_t n, const double* vel0, const double* vel,
                           const double* ft, const double* mass, const double* inertia,
                           const double* gravity, double dt, double* res, double* norms,
                           cudaStream_t s) {
  cudaMemsetAsync(norms, 0, 2 * sizeof(double), s);
  if (n > 0) {
    ProfScope ps(c, K_STEP, s);
    Gravity g{{gravity[0], gravity[1], gravity[2]}};
    launch_after(k_residual, blocks_for(c, n), kThreads, 0, s, n, vel0, vel, ft, mass, inertia, g,
                 dt, res, reinterpret_cast<unsigned long long*>(norms));
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_vel_axpy(mrdem_ctx* c, int64_t m, double a, const double* x, const double* y,
                    double* out, cudaStream_t s) {
  if (m > 0) {
    ProfScope ps(c, K_STEP, s);
    launch_after(k_vel_axpy, blocks_for(c, m), kThreads, 0, s, m, a, x, y, out);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

// Conjugate-gradient scratch: five vectors of 6n doubles, 3 (max_iter + 1)
// scalars and the state record.
static int ensure_cg(mrdem_ctx* c, int32_t n, int32_t max_iter, CgView* v) {
  const size_t m = (size_t)6 * n, ns = 3 * ((size_t)max_iter + 1);
  const size_t bytes = sizeof(double) * (5 * m + ns) + 64;
  if (bytes > c->cap_cg) {
    cudaFree(c->cg_mem);
    c->cg_mem = nullptr;
    c->cap_cg = 0;
    if (cudaMalloc(&c->cg_mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->cg_mem = nullptr;
      return MRDEM_ERR_OOM;
    }
    c->cap_cg = bytes;
  }
  unsigned char* p = static_cast<unsigned char*>(c->cg_mem);
  v->st = reinterpret_cast<CgState*>(p);
  double* d = reinterpret_cast<double*>(p + 64);
  v->rz = d;
  v->pap = d + (max_iter + 1);
  v->rr = d + 2 * ((size_t)max_iter + 1);
  d += ns;
  v->r = d;
  v->z = d + m;
  v->p = d + 2 * m;
  v->ap = d + 3 * m;
  v->diag = d + 4 * m;
  return MRDEM_OK;
}

int launch_newton_solve(mrdem_ctx* c, int32_t n, int64_t n_pairs, const int32_t* ab,
                        const double* blocks, const double* mass, const double* inertia,
                        double dt, const double* rhs, double* x, int32_t max_iter, double rel_tol,
                        int32_t check_every, double* info, cudaStream_t s) {
  (void)check_every;  // the solve stops on the device
  CgView v;
  int st = ensure_cg(c, n, max_iter, &v);
  if (st) return st;
  v.x = x;
  v.mass = mass;
  v.inertia = inertia;
  v.dt = dt;
  v.n = n;
  const size_t ns = 3 * ((size_t)max_iter + 1);
  ProfScope ps(c, K_CG, s);
  cudaMemsetAsync(c->cg_mem, 0, 64 + sizeof(double) * ns, s);
  // every block resident at once (a cooperative launch)
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_coop, kThreads, 0) != cudaSuccess ||
      occ <= 0) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  const int64_t m = (int64_t)6 * n, work = m > n_pairs ? m : n_pairs;
  const int64_t need = (work + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)occ * c->n_sms;
  const int grid = (int)(need < 1 ? 1 : (need < cap ? need : cap));
  const double tol2 = rel_tol * rel_tol;
  // a cooperative launch through the launch attribute (also valid as a node
  // of a captured CUDA graph)
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = s;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_cg_coop, v, rhs, n_pairs, ab, blocks, (int)max_iter, tol2,
                         info) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  return MRDEM_OK;
}

int launch_refine_contacts(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                           const double* eps, const double* poses, const mrdem_contacts* cand,
                           const mrdem_contacts* out, cudaStream_t s) {
  const int64_t cap = cand->capacity > 0 ? cand->capacity : 1;
  const size_t bytes = (sizeof(RefineRec) + sizeof(int32_t)) * (size_t)cap;
  if (bytes > c->cap_refine) {
    cudaFree(c->refine_mem);
    c->refine_mem = nullptr;
    c->cap_refine = 0;
    if (cudaMalloc(&c->refine_mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->refine_mem = nullptr;
      return MRDEM_ERR_OOM;
    }
    c->cap_refine = bytes;
  }
  RefineRec* rec = static_cast<RefineRec*>(c->refine_mem);
  int32_t* keep = reinterpret_cast<int32_t*>(rec + cap);
  ProfScope ps(c, K_STEP, s);
  cudaMemsetAsync(out->count, 0, sizeof(int64_t), s);
  const int nb = blocks_for(c, cap);
  launch_after(k_refine, nb, kThreads, 0, s, h->dev, ab, eps, poses, *cand, n_pairs, rec, keep);
  launch_after(k_refine_scan, 1, 1024, 0, s, keep, *cand, out->count);
  launch_after(k_refine_write, nb, kThreads, 0, s, *cand, (const RefineRec*)rec,
               (const int32_t*)keep, *out, c->status);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_motion_bound(mrdem_ctx* c, int32_t n, const double* ref, const double* poses,
                        const double* bound, double* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(double), s);
  if (n > 0) {
    ProfScope ps(c, K_STEP, s);
    launch_after(k_motion, blocks_for(c, n), kThreads, 0, s, n, ref, poses, bound,
                 reinterpret_cast<unsigned long long*>(out));
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
