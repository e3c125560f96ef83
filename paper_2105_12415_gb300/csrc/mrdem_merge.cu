// mrdem_merge.cu -- redundant-contact merge of Sec. 2 (Noble & Weinzierl,
// arXiv 2105.12415, the implementation note on the contact set).
//
// A contact spanned by two vertices (or a vertex and an edge) is found by
// every pair of triangles adjacent to them, with slightly different rounding;
// the paper merges contact points of a particle pair that lie closer than eps
// into one average point before the set is used.  Reading taken here: within
// a pair, contacts i and j are linked when their contact points
// x = (pa + pb)/2 satisfy ((dx*dx + dy*dy) + dz*dz) < eps*eps in FP64
// (explicitly rounded operations, no fused multiply-add); every connected
// component of two or more contacts becomes one contact with the members'
// mean pa and pb (so the mean contact point and the mean normal),
// dist = |pa - pb|, and the triangle indices of the member with the smallest
// (tri_a, tri_b); a lone contact is kept as detected.
//
// Pipeline (one stream, programmatic launches):
//   k_merge_count    contacts per pair;
//   k_merge_scan     exclusive scan -> segment begins;
//   k_merge_scatter  contact indices grouped by pair (the cursors end as the
//                    segment ends);
//   k_merge_small    one warp per pair with at most kSmallCap contacts,
//   k_merge_large    one block per larger pair (shared memory up to
//                    kLargeCap contacts, the context's scratch beyond):
//                    bitonic sort by (tri_a, tri_b), a second one along x,
//                    links by a sweep along x (a float test with an error
//                    bound decides all but the pairs near eps, which take
//                    the FP64 test), lock-free union-find with links to the
//                    smaller index and path halving (the root of a component
//                    is its smallest key), component means (a thread per
//                    small component, a warp per large one); each pair
//                    writes its merged contacts at the start of its segment
//                    of a scratch list;
//   k_merge_scan     exclusive scan of the merged counts -> output offsets
//                    and the total (the output count);
//   k_merge_copy     compaction into the caller's buffers.
// Every step is deterministic: the output order is (pair, representative
// key) and every sum runs in a fixed order.
#include <cuda_runtime.h>

#include "mrdem_device.cuh"

namespace mrdem {

namespace {

constexpr int kSmallCap = 64;     // contacts of a pair handled by one warp
constexpr int kLaneSum = 16;      // components up to this size are summed by one thread
constexpr int kSmallWarps = 4;
constexpr int kLargeThreads = 512;
constexpr int kLargeCap = 1024;   // contacts of a pair held in shared memory by one block
// pa, pb, key, xf, sx, src, px, parent
constexpr int kEntryBytes = 24 + 24 + 8 + 12 + 4 + 4 + 4 + 4;
constexpr size_t kLargeSmem = (size_t)kEntryBytes * kLargeCap;

// Per-contact working arrays of one pair's segment (shared or global
// memory), room for P entries (n rounded up to a power of two).
struct SegView {
  double* pa;       // [3][ld] point_a, key order
  double* pb;       // [3][ld] point_b, key order
  long long* key;   // [ld] (tri_a, tri_b) packed; later the list of roots (int)
  float* xf;        // [3][ld] contact point - the first one, float; later component sizes (int)
  float* sx;        // [ld] x of xf in x order
  int* src;         // [ld] contact index, sorted with the keys
  int* px;          // [ld] key-order index in x order; later output ranks of the roots
  int* parent;      // [ld] union-find forest over key order
  int ld;
};

__device__ __forceinline__ SegView carve(unsigned char* p, int cap) {
  SegView v;
  v.ld = cap;
  v.pa = reinterpret_cast<double*>(p);
  p += sizeof(double) * 3 * cap;
  v.pb = reinterpret_cast<double*>(p);
  p += sizeof(double) * 3 * cap;
  v.key = reinterpret_cast<long long*>(p);
  p += sizeof(long long) * cap;
  v.xf = reinterpret_cast<float*>(p);
  p += sizeof(float) * 3 * cap;
  v.sx = reinterpret_cast<float*>(p);
  p += sizeof(float) * cap;
  v.src = reinterpret_cast<int*>(p);
  p += sizeof(int) * cap;
  v.px = reinterpret_cast<int*>(p);
  p += sizeof(int) * cap;
  v.parent = reinterpret_cast<int*>(p);
  return v;
}

// Context scratch: the SegView arrays for pairs beyond kLargeCap contacts
// (2 cap entries: a segment [b, b + n) works in [2b, 2b + P), P < 2n, so the
// segments' regions do not overlap), the grouped indices and the per-segment
// merged contacts.
struct MergeScratch {
  double* wa;       // [3][2 cap]
  double* wb;       // [3][2 cap]
  long long* key;   // [2 cap]
  float* xf;        // [3][2 cap]
  float* sx;        // [2 cap]
  int* src;         // [2 cap]
  int* px;          // [2 cap]
  int* parent;      // [2 cap]
  int32_t* idx;     // [cap] contact indices grouped by pair
  // merged contacts, written at the start of each pair's segment
  double* dist;     // [cap]
  double* pa;       // [cap*3]
  double* pb;       // [cap*3]
  int32_t* pair;    // [cap], -1 past a segment's merged contacts
  int32_t* tri_a;
  int32_t* tri_b;
  int32_t* members;
  int64_t cap;
};

__device__ __forceinline__ SegView global_view(const MergeScratch& g, int b) {
  const int64_t o = 2 * (int64_t)b;
  SegView v;
  v.ld = (int)(2 * g.cap);
  v.pa = g.wa + o;
  v.pb = g.wb + o;
  v.key = g.key + o;
  v.xf = g.xf + o;
  v.sx = g.sx + o;
  v.src = g.src + o;
  v.px = g.px + o;
  v.parent = g.parent + o;
  return v;
}

template <int G>
__device__ __forceinline__ int grp_rank() { return G == 32 ? (int)lane_id() : (int)threadIdx.x; }
template <int G>
__device__ __forceinline__ void grp_sync() {
  if (G == 32) __syncwarp();
  else __syncthreads();
}

// Maximum over the group (NaN ignored); red: G/32 floats of shared memory.
template <int G>
__device__ __forceinline__ float grp_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (G == 32) return v;
  if (lane_id() == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = red[0];
  for (int k = 1; k < G / 32; ++k) r = fmaxf(r, red[k]);
  __syncthreads();
  return r;
}

// Exclusive prefix count of a flag over the group and the group's total;
// red: G/32 ints of shared memory.
template <int G>
__device__ __forceinline__ void grp_scan(bool f, int* red, int& excl, int& tot) {
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  const int lane = (int)lane_id();
  const int in_warp = __popc(bal & ((1u << lane) - 1u));
  if (G == 32) {
    excl = in_warp;
    tot = __popc(bal);
    return;
  }
  const int w = threadIdx.x >> 5;
  if (lane == 0) red[w] = __popc(bal);
  __syncthreads();
  int before = 0, all = 0;
  for (int k = 0; k < G / 32; ++k) {
    const int v = red[k];
    before += k < w ? v : 0;
    all += v;
  }
  __syncthreads();
  excl = before + in_warp;
  tot = all;
}

// Bitonic sort of entries [0, P) (P a power of two) by a strict order:
// less(i, j) compares entries i and j, swap(i, j) exchanges them.  A fixed
// network of log2(P) (log2(P) + 1) / 2 stages.
template <int G, class Less, class Swap>
__device__ __forceinline__ void grp_bitonic(int P, Less less, Swap swap) {
  const int t = grp_rank<G>();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = t; i < P; i += G) {
        const int l = i ^ j;
        if (l > i && less(l, i) == ((i & k) == 0)) swap(i, l);
      }
      grp_sync<G>();
    }
  }
}

// Union-find whose parent pointers always go to a smaller index: a find ends
// within i steps, and the root of a component is its smallest member.  Finds
// halve the path as they go (a node is pointed at its grandparent): dense
// clusters link almost every pair, and without it the trees grew deep enough
// for the finds to dominate.  Concurrent finds and hooks stay correct: a
// halving write goes to a node that is no longer a root and stores one of its
// ancestors, and roots change only by compare-and-swap.
__device__ __forceinline__ int uf_find(int* parent_, int i) {
  volatile int* parent = parent_;
  int p = parent[i];
  while (p != i) {
    const int g = parent[p];
    if (g == p) return p;
    parent[i] = g;
    i = g;
    p = parent[i];
  }
  return i;
}
// Hook the larger of the two roots under the smaller.  A failed compare-and-
// swap means another thread hooked that root first, to a smaller index, so
// every retry starts from smaller roots: at most about 2n rounds.
__device__ __forceinline__ void uf_unite(int* parent, int a, int b, int n) {
  for (int it = 0; it < 2 * n + 8; ++it) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(parent + b, b, a) == b) return;
  }
}

// Component q of the contact point (pa + pb)/2 of entry i.
__device__ __forceinline__ double xmid(const SegView& S, int q, int i) {
  return __dmul_rn(0.5, __dadd_rn(S.pa[q * S.ld + i], S.pb[q * S.ld + i]));
}

// The FP64 link test, operation for operation the reading's predicate.
__device__ __forceinline__ bool link64(const SegView& S, int i, int j, double lim) {
  const double dx = __dsub_rn(xmid(S, 0, i), xmid(S, 0, j));
  const double dy = __dsub_rn(xmid(S, 1, i), xmid(S, 1, j));
  const double dz = __dsub_rn(xmid(S, 2, i), xmid(S, 2, j));
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return d2 < lim;
}

// Merged output of one segment.
struct MergeOut {
  double* dist;
  double* pa;
  double* pb;
  int32_t* pair;
  int32_t* tri_a;
  int32_t* tri_b;
  int32_t* members;
  int32_t* mcnt;  // [n_pairs] merged contacts per pair
};

// Means of k summed contacts (one reciprocal, six products) and their
// distance.
__device__ __forceinline__ double finish_mean(double (&a)[3], double (&bb)[3], int k) {
  const double inv = __drcp_rn((double)k);
  for (int q = 0; q < 3; ++q) {
    a[q] = __dmul_rn(a[q], inv);
    bb[q] = __dmul_rn(bb[q], inv);
  }
  const double dx = __dsub_rn(a[0], bb[0]), dy = __dsub_rn(a[1], bb[1]), dz = __dsub_rn(a[2], bb[2]);
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__device__ __forceinline__ void write_merged(const MergeOut& o, int64_t w, int p, int ta, int tb,
                                             int k, const double (&a)[3], const double (&bb)[3],
                                             double d) {
  o.pair[w] = p;
  o.tri_a[w] = ta;
  o.tri_b[w] = tb;
  o.members[w] = k;
  o.dist[w] = d;
  for (int q = 0; q < 3; ++q) {
    o.pa[3 * w + q] = a[q];
    o.pb[3 * w + q] = bb[q];
  }
}

// Merge the n contacts idx[b .. b+n) of pair p with a group of G threads.
template <int G>
__device__ __forceinline__ void merge_segment(const mrdem_contacts& in,
                                              const int32_t* __restrict__ idx, int b, int n,
                                              int p, double ep, const SegView& S,
                                              const MergeOut& o, void* red) {
  const int t = grp_rank<G>();
  const int ld = S.ld;
  int P = 2;
  while (P < n) P <<= 1;
  // keys (tri_a, tri_b) with the contact index, padded to P with the largest
  // key, sorted: ties (repeated triangle pairs) go by contact index
  for (int i = t; i < P; i += G) {
    long long k = 0x7fffffffffffffffll;
    int c = 0x7fffffff;
    if (i < n) {
      c = idx[b + i];
      k = ((long long)in.tri_a[c] << 32) + ((long long)in.tri_b[c] + 0x80000000ll);
    }
    S.key[i] = k;
    S.src[i] = c;
  }
  grp_sync<G>();
  grp_bitonic<G>(
      P,
      [&](int i, int j) { return S.key[i] < S.key[j] || (S.key[i] == S.key[j] && S.src[i] < S.src[j]); },
      [&](int i, int j) {
        const long long k = S.key[i];
        S.key[i] = S.key[j];
        S.key[j] = k;
        const int c = S.src[i];
        S.src[i] = S.src[j];
        S.src[j] = c;
      });
  // closest points in key order
  for (int i = t; i < n; i += G) {
    const int64_t c = S.src[i];
    for (int q = 0; q < 3; ++q) {
      S.pa[q * ld + i] = in.point_a[3 * c + q];
      S.pb[q * ld + i] = in.point_b[3 * c + q];
    }
    S.parent[i] = i;
  }
  grp_sync<G>();
  // float copies relative to the first point and their extent
  float ext = 0.f;
  for (int i = t; i < n; i += G) {
    for (int q = 0; q < 3; ++q) {
      const float v = (float)__dsub_rn(xmid(S, q, i), xmid(S, q, 0));
      S.xf[q * ld + i] = v;
      ext = fmaxf(ext, fabsf(v));
    }
  }
  ext = grp_max<G>(ext, static_cast<float*>(red));
  // Float decision bands.  With u = 2^-24 and R the extent, each float
  // difference is within 4.01 u R of the double one per component and the
  // float squared norm within 3.01 u relative, so a float value below lo2
  // (above hi2) puts the point pair certainly inside (outside) eps with
  // room for the FP64 test's own rounding; the band between goes to FP64.
  // A float x gap above hi rules a pair out the same way.
  const float u = 5.9604645e-8f;
  const float ef = (float)ep;
  const float eta = 8.f * u * (ext + ef);
  const float lo = ef - eta, hi = ef + eta;
  const float lo2 = lo > 0.f ? lo * lo * (1.f - 8.f * u) : -1.f;
  const float hi2 = hi * hi * (1.f + 8.f * u);
  const double lim = __dmul_rn(ep, ep);
  // x order (ties by index), padded with +inf; a NaN x (it links to
  // nothing) sorts as +inf so the order stays total
  for (int i = t; i < P; i += G) {
    S.px[i] = i;
    S.sx[i] = i < n && !isnan(S.xf[i]) ? S.xf[i] : __int_as_float(0x7f800000);
  }
  grp_sync<G>();
  grp_bitonic<G>(
      P, [&](int i, int j) { return S.sx[i] < S.sx[j] || (S.sx[i] == S.sx[j] && S.px[i] < S.px[j]); },
      [&](int i, int j) {
        const float x = S.sx[i];
        S.sx[i] = S.sx[j];
        S.sx[j] = x;
        const int k = S.px[i];
        S.px[i] = S.px[j];
        S.px[j] = k;
      });
  // links: a thread per point in x order against the points after it until
  // the x gap exceeds hi
  for (int k1 = t; k1 < n; k1 += G) {
    const int i = S.px[k1];
    const float x1 = S.sx[k1];
    const float yi = S.xf[ld + i], zi = S.xf[2 * ld + i];
    for (int k2 = k1 + 1; k2 < n; ++k2) {
      const float dx = S.sx[k2] - x1;
      if (dx > hi) break;
      const int j = S.px[k2];
      const float dy = yi - S.xf[ld + j], dz = zi - S.xf[2 * ld + j];
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      bool link = d2 < lo2;
      if (!link && !(d2 > hi2)) link = link64(S, i, j, lim);
      if (link) uf_unite(S.parent, i, j, n);
    }
  }
  grp_sync<G>();
  // every parent pointer to its root (a concurrent reader sees either the
  // old parent or the root, both ancestors)
  for (int i = t; i < n; i += G) {
    const int r = uf_find(S.parent, i);
    static_cast<volatile int*>(S.parent)[i] = r;
  }
  grp_sync<G>();
  // the roots in key order: their output ranks (kept in px) and the list of
  // them (kept in the key array), and the component sizes (kept in xf); those
  // arrays are no longer needed
  int* roots = reinterpret_cast<int*>(S.key);
  int* size = reinterpret_cast<int*>(S.xf);
  for (int i = t; i < n; i += G) size[i] = 0;
  grp_sync<G>();
  for (int i = t; i < n; i += G) atomicAdd(size + S.parent[i], 1);
  int m = 0;
  for (int c0 = 0; c0 < n; c0 += G) {
    const int i = c0 + t;
    const bool root = i < n && S.parent[i] == i;
    int excl, tot;
    grp_scan<G>(root, static_cast<int*>(red), excl, tot);
    if (root) {
      S.px[i] = m + excl;
      roots[m + excl] = i;
    }
    m += tot;
  }
  grp_sync<G>();
  // One merged contact per root.  FP64 runs at a small fraction of the FP32
  // rate, so the sums are arranged to keep the FP64 instructions per group
  // nearly constant: a lone contact is copied as it is; a component of at
  // most kLaneSum members is summed by one thread (all such components in
  // parallel); a larger one by a warp (lane l takes the members r + l,
  // r + l + 32, ..., then a butterfly over the lanes).  Every order is fixed.
  for (int r = t; r < n; r += G) {
    if (S.parent[r] != r) continue;
    const int k = size[r];
    if (k > kLaneSum) continue;
    const int64_t c0 = S.src[r];
    double a[3], bb[3], d;
    if (k == 1) {
      for (int q = 0; q < 3; ++q) {
        a[q] = S.pa[q * ld + r];
        bb[q] = S.pb[q * ld + r];
      }
      d = in.dist[c0];
    } else {
      for (int q = 0; q < 3; ++q) a[q] = bb[q] = 0.0;
      int cnt = 0;
      for (int j = r; j < n && cnt < k; ++j) {
        if (S.parent[j] != r) continue;
        for (int q = 0; q < 3; ++q) {
          a[q] = __dadd_rn(a[q], S.pa[q * ld + j]);
          bb[q] = __dadd_rn(bb[q], S.pb[q * ld + j]);
        }
        ++cnt;
      }
      d = finish_mean(a, bb, k);
    }
    write_merged(o, (int64_t)b + S.px[r], p, in.tri_a[c0], in.tri_b[c0], k, a, bb, d);
  }
  {
    const int lane = t & 31, w = t >> 5;
    int big = 0;
    for (int q = 0; q < m; ++q) {
      const int r = roots[q];
      const int k = size[r];
      if (k <= kLaneSum) continue;
      if (big++ % (G / 32) != w) continue;
      double a[3] = {0.0, 0.0, 0.0}, bb[3] = {0.0, 0.0, 0.0};
      for (int j = r + lane; j < n; j += 32) {
        if (S.parent[j] != r) continue;
        for (int c = 0; c < 3; ++c) {
          a[c] = __dadd_rn(a[c], S.pa[c * ld + j]);
          bb[c] = __dadd_rn(bb[c], S.pb[c * ld + j]);
        }
      }
      for (int o2 = 16; o2 > 0; o2 >>= 1) {
        for (int c = 0; c < 3; ++c) {
          a[c] = __dadd_rn(a[c], __shfl_xor_sync(0xffffffffu, a[c], o2));
          bb[c] = __dadd_rn(bb[c], __shfl_xor_sync(0xffffffffu, bb[c], o2));
        }
      }
      if (lane == 0) {
        const double d = finish_mean(a, bb, k);
        const int64_t c0 = S.src[r];
        write_merged(o, (int64_t)b + q, p, in.tri_a[c0], in.tri_b[c0], k, a, bb, d);
      }
    }
  }
  for (int i = m + t; i < n; i += G) o.pair[b + i] = -1;
  if (t == 0) o.mcnt[p] = m;
  grp_sync<G>();  // the next segment reuses the working arrays
}

__device__ __forceinline__ int64_t input_count(const mrdem_contacts& in) {
  const int64_t n = *in.count;
  return n < in.capacity ? n : in.capacity;
}

// Contacts per pair; invalid pair indices and eps are latched (the entries
// are dropped).
__global__ void __launch_bounds__(256) k_merge_count(mrdem_contacts in, int64_t n_pairs,
                                                     const double* __restrict__ eps, int32_t* seg,
                                                     unsigned long long* status) {
  wait_prior_grid();
  const int64_t n = input_count(in);
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += step) {
    const int p = in.pair[k];
    if (p < 0 || p >= n_pairs) {
      bad = true;
      continue;
    }
    atomicAdd(seg + p, 1);
  }
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs; p += step) {
    const double e = eps[p];
    if (!(e > 0.0) || !isfinite(e)) bad = true;
  }
  if (bad) atomicExch(status + ST_NONFINITE, 1ull);
}

__global__ void __launch_bounds__(1024) k_merge_scan(int32_t* cnt, int64_t n, int64_t* total) {
  wait_prior_grid();
  block_exclusive_scan(cnt, n, total);
}

__global__ void __launch_bounds__(256) k_merge_scatter(mrdem_contacts in, int64_t n_pairs,
                                                       int32_t* seg, int32_t* idx) {
  wait_prior_grid();
  const int64_t n = input_count(in);
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += step) {
    const int p = in.pair[k];
    if (p < 0 || p >= n_pairs) continue;
    idx[atomicAdd(seg + p, 1)] = (int32_t)k;
  }
}

__device__ __forceinline__ MergeOut merge_out(const MergeScratch& g, int32_t* mcnt) {
  return MergeOut{g.dist, g.pa, g.pb, g.pair, g.tri_a, g.tri_b, g.members, mcnt};
}

// One warp per pair with 1..kSmallCap contacts (and the merged count of the
// empty pairs).
__global__ void __launch_bounds__(kSmallWarps * 32) k_merge_small(
    mrdem_contacts in, int64_t n_pairs, const double* __restrict__ eps,
    const int32_t* __restrict__ seg, MergeScratch g, int32_t* mcnt) {
  wait_prior_grid();
  __shared__ __align__(16) unsigned char sm[kSmallWarps][kEntryBytes * kSmallCap];
  __shared__ float red[kSmallWarps];
  const int w = threadIdx.x >> 5, lane = lane_id();
  const SegView S = carve(sm[w], kSmallCap);
  const MergeOut o = merge_out(g, mcnt);
  const int64_t warps = (int64_t)gridDim.x * kSmallWarps;
  for (int64_t p = (int64_t)blockIdx.x * kSmallWarps + w; p < n_pairs; p += warps) {
    const int b = p > 0 ? seg[p - 1] : 0, n = seg[p] - b;
    if (n > kSmallCap) continue;
    if (n == 0) {
      if (lane == 0) mcnt[p] = 0;
      continue;
    }
    merge_segment<32>(in, g.idx, b, n, (int)p, eps[p], S, o, &red[w]);
  }
}

// One block per pair with more than kSmallCap contacts: shared memory up to
// kLargeCap contacts, the context's scratch beyond.
__global__ void __launch_bounds__(kLargeThreads) k_merge_large(
    mrdem_contacts in, int64_t n_pairs, const double* __restrict__ eps,
    const int32_t* __restrict__ seg, MergeScratch g, int32_t* mcnt) {
  wait_prior_grid();
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ int red[kLargeThreads / 32];
  const MergeOut o = merge_out(g, mcnt);
  for (int64_t p = blockIdx.x; p < n_pairs; p += gridDim.x) {
    const int b = p > 0 ? seg[p - 1] : 0, n = seg[p] - b;
    if (n <= kSmallCap) continue;
    const SegView S = n <= kLargeCap ? carve(dyn, kLargeCap) : global_view(g, b);
    merge_segment<kLargeThreads>(in, g.idx, b, n, (int)p, eps[p], S, o, red);
  }
}

// Compaction of the merged contacts into the caller's buffers; *out.count
// already holds the total (the scan wrote it).
__global__ void __launch_bounds__(256) k_merge_copy(MergeScratch g, int64_t n_pairs,
                                                    const int32_t* __restrict__ seg,
                                                    const int32_t* __restrict__ moff,
                                                    mrdem_contacts out, int32_t* members,
                                                    unsigned long long* status) {
  wait_prior_grid();
  const int64_t total = *out.count;
  if (blockIdx.x == 0 && threadIdx.x == 0 && total > out.capacity)
    atomicMax(status + ST_REQ_CONTACTS, (unsigned long long)total);
  const int64_t n = n_pairs > 0 ? seg[n_pairs - 1] : 0;  // grouped entries
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += step) {
    const int p = g.pair[j];
    if (p < 0) continue;
    const int64_t r = j - (p > 0 ? seg[p - 1] : 0);
    const int64_t w = moff[p] + r;
    if (w >= out.capacity) continue;
    out.pair[w] = p;
    out.tri_a[w] = g.tri_a[j];
    out.tri_b[w] = g.tri_b[j];
    out.dist[w] = g.dist[j];
    for (int q = 0; q < 3; ++q) {
      out.point_a[3 * w + q] = g.pa[3 * j + q];
      out.point_b[3 * w + q] = g.pb[3 * j + q];
    }
    if (members) members[w] = g.members[j];
  }
}

// Bytes per input entry of the context scratch: twice the SegView arrays,
// the grouped index and a merged contact (dist, pa, pb, pair, tri_a, tri_b,
// members).
constexpr size_t kScratchBytes = 2 * kEntryBytes + 4 + 8 + 48 + 16;

int ensure_merge(mrdem_ctx* c, int64_t n_pairs, int64_t cap, MergeScratch* g) {
  if (n_pairs > c->cap_merge_pairs) {
    cudaFree(c->merge_seg);
    c->merge_seg = nullptr;
    c->cap_merge_pairs = 0;
    if (cudaMalloc(&c->merge_seg, sizeof(int32_t) * 2 * n_pairs) != cudaSuccess) {
      cudaGetLastError();
      c->merge_seg = nullptr;
      return MRDEM_ERR_OOM;
    }
    c->cap_merge_pairs = n_pairs;
  }
  const int64_t need = cap > 0 ? cap : 1;
  if (need > c->cap_merge) {
    cudaFree(c->merge_mem);
    c->merge_mem = nullptr;
    c->cap_merge = 0;
    if (cudaMalloc(&c->merge_mem, kScratchBytes * need) != cudaSuccess) {
      cudaGetLastError();
      c->merge_mem = nullptr;
      return MRDEM_ERR_OOM;
    }
    c->cap_merge = need;
  }
  // 8-byte arrays first, then 4-byte arrays (all aligned)
  const int64_t n = c->cap_merge, n2 = 2 * n;
  unsigned char* p = static_cast<unsigned char*>(c->merge_mem);
  auto take = [&p](size_t bytes) {
    unsigned char* r = p;
    p += bytes;
    return r;
  };
  g->cap = n;
  g->wa = reinterpret_cast<double*>(take(sizeof(double) * 3 * n2));
  g->wb = reinterpret_cast<double*>(take(sizeof(double) * 3 * n2));
  g->key = reinterpret_cast<long long*>(take(sizeof(long long) * n2));
  g->dist = reinterpret_cast<double*>(take(sizeof(double) * n));
  g->pa = reinterpret_cast<double*>(take(sizeof(double) * 3 * n));
  g->pb = reinterpret_cast<double*>(take(sizeof(double) * 3 * n));
  g->xf = reinterpret_cast<float*>(take(sizeof(float) * 3 * n2));
  g->sx = reinterpret_cast<float*>(take(sizeof(float) * n2));
  g->src = reinterpret_cast<int*>(take(sizeof(int) * n2));
  g->px = reinterpret_cast<int*>(take(sizeof(int) * n2));
  g->parent = reinterpret_cast<int*>(take(sizeof(int) * n2));
  g->idx = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  g->pair = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  g->tri_a = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  g->tri_b = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  g->members = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n));
  return MRDEM_OK;
}

}  // namespace

int launch_merge(mrdem_ctx* c, int64_t n_pairs, const double* eps, const mrdem_contacts* in,
                 const mrdem_contacts* out, int32_t* members, cudaStream_t s) {
  if (n_pairs == 0) {
    cudaMemsetAsync(out->count, 0, sizeof(int64_t), s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
  }
  MergeScratch g;
  int st = ensure_merge(c, n_pairs, in->capacity, &g);
  if (st) return st;
  if (!c->merge_smem_set) {  // the context's device
    if (cudaFuncSetAttribute(k_merge_large, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kLargeSmem) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->merge_side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->merge_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->merge_ev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return MRDEM_ERR_CUDA;
    }
    c->merge_smem_set = true;
  }
  int32_t* seg = c->merge_seg;
  int32_t* mcnt = c->merge_seg + c->cap_merge_pairs;
  ProfScope ps(c, K_MERGE, s);
  cudaMemsetAsync(seg, 0, sizeof(int32_t) * n_pairs, s);
  const int flat = c->n_sms * 8;
  const int64_t small_blocks = (n_pairs + kSmallWarps - 1) / kSmallWarps;
  const int gs = (int)(small_blocks < c->n_sms * 8 ? small_blocks : c->n_sms * 8);
  const int gl = (int)(n_pairs < c->n_sms * 2 ? n_pairs : c->n_sms * 2);
  launch_after(k_merge_count, flat, 256, 0, s, *in, n_pairs, eps, seg, c->status);
  launch_after(k_merge_scan, 1, 1024, 0, s, seg, n_pairs, (int64_t*)nullptr);
  launch_after(k_merge_scatter, flat, 256, 0, s, *in, n_pairs, seg, g.idx);
  // the pairs of more than kSmallCap contacts (few, a block each) run on the
  // second stream beside the small pairs (a warp each): they write disjoint
  // segments; both streams join before the scan of the merged counts
  cudaEventRecord(c->merge_ev[0], s);
  cudaStreamWaitEvent(c->merge_side, c->merge_ev[0], 0);
  k_merge_large<<<gl, kLargeThreads, kLargeSmem, c->merge_side>>>(
      *in, n_pairs, eps, (const int32_t*)seg, g, mcnt);
  cudaEventRecord(c->merge_ev[1], c->merge_side);
  launch_after(k_merge_small, gs, kSmallWarps * 32, 0, s, *in, n_pairs, eps, (const int32_t*)seg,
               g, mcnt);
  cudaStreamWaitEvent(s, c->merge_ev[1], 0);
  k_merge_scan<<<1, 1024, 0, s>>>(mcnt, n_pairs, out->count);
  launch_after(k_merge_copy, flat, 256, 0, s, g, n_pairs, (const int32_t*)seg,
               (const int32_t*)mcnt, *out, members, c->status);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
