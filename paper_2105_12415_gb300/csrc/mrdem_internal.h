// mrdem_internal.h -- data structures shared by the host code and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "mrdem.h"
#include "mrdem_dd.cuh"
#include "mrdem_geometry.cuh"

namespace mrdem {

constexpr int kMaxLevels = 16;  // unfold steps of the level loop (tree depth <= 16)

// Host-side surrogate trees of all particles (built by mrdem_build_hierarchy_host).
struct HierHost {
  int32_t n_particles = 0, max_depth = 0;
  int64_t n_nodes = 0, n_tri = 0, n_tri_pad = 0, n_verts = 0;
  std::vector<float> node_tri;      // [n_nodes * 9]
  std::vector<float> node_delta;    // [n_nodes]
  std::vector<float> node_box;      // [n_nodes * 16] oriented box: c, u0, u1, u2, h, 0
  std::vector<int32_t> node_child;  // [n_nodes * 2] (begin, count); count < 0: leaf slots
  std::vector<int32_t> node_level;  // [n_nodes]
  std::vector<int32_t> root;        // [n_particles]
  std::vector<float> slot_xyz;      // [n_tri_pad * 9] fine triangle per slot (body frame)
  std::vector<int32_t> slot_vid;    // [n_tri_pad * 3] global vertex index (-1 pad)
  std::vector<int32_t> slot_tri;    // [n_tri_pad] local input triangle index (-1 pad)
  std::vector<int32_t> slot_particle;  // [n_tri_pad]
  std::vector<int32_t> tri_slot;    // [n_tri] global input triangle -> slot
  std::vector<int64_t> tri_off;     // [n+1] input triangle offsets
  std::vector<int64_t> vert_off;    // [n+1]
  std::vector<float> bound_r;       // [n] max |v| over the particle's vertices
};

// Device view of a hierarchy, passed by value to kernels.
struct HierDev {
  const float4* node_geo;  // [n_nodes*3]: (v0.xyz, delta) (v1.xyz, 0) (v2.xyz, 0)
  const float4* node_sph;  // [n_nodes]: body-frame sphere (centre, radius + delta) holding
                           // the node's surrogate eps-free environment
  const float4* node_nrm;  // [n_nodes]: body-frame unit normal of the surrogate triangle and
                           // its plane offset n.v0 (FP64 on the host; zero if degenerate)
  const int2* node_child;  // [n_nodes]
  const float4* tri;       // [stride*3]: slot s's vertices as one 48-B record,
                           // (v0.xyz v1.x) (v1.yz v2.xy) (v2.z 0 0 0)
  const float4* tri_sph;   // [stride]: body-frame bounding sphere of each fine triangle
  const float4* node_box;  // [n_nodes*4]: oriented box around the node's fine vertices,
                           // (c.xyz, h0) (u0.xyz, h1) (u1.xyz, h2) (u2.xyz, 0)
  const float4* node_boxw; // [n_nodes]: the box's half widths along its own three axes,
                           // sum_k h_k |u_s . u_k| (FP64 of the float axes, rounded up), 0
  const int2* node_up;     // [n_nodes]: (parent node, -1 for a root; level, roots 1)
  const int32_t* vid;      // 3 planes: global vertex index of corner k of slot s
  const int32_t* slot_tri; // [stride] local input triangle index (-1 pad)
  const int32_t* tri_slot; // [n_tri] global input triangle -> slot
  const int64_t* tri_off;  // [n+1]
  const int32_t* root;     // [n]
  const float* bound_r;    // [n]
  int64_t stride;          // plane stride (n_tri_pad rounded up)
  int64_t n_tri;
  int64_t n_nodes;
  int32_t n_particles;
};

// Per particle pair transform, written by the setup kernel.
struct alignas(16) PairXf {
  float R[9];   // B body -> A body rotation (float)
  float t[3];   // B body -> A body translation (float)
  float tau;    // 2 eps
  float margin; // float rounding margin of the certificate
  int32_t A, B;
};
struct alignas(16) PairXf64 {
  double R[9], t[3];    // B body -> A body
  double RA[9], tA[3];  // A body -> world
  double eps;
  int32_t A, B, valid, pad;
};

// Work items.  A level item holds the node pairs still to be tested: the
// child sets Ca = [a_begin, a_begin + na) and Cb (a leaf side is its own
// one-element set): int4 (pair, a_begin, b_begin, na | nb << 8).
// A tile item is a pair of leaves with their fine-triangle slot ranges.
struct alignas(16) TileItem {
  int pair, node_a, node_b, slot_a;
  int slot_b, counts, pad0, pad1;  // counts = na | nb << 8
};

// A pair accepted by the float stage of the closest-point computation: its
// double geometry and the ranges of its work items.
// The pair's transforms in double-float (FP32 form of the final values).
struct alignas(16) PairXfDD {
  dd R[9], t[3];    // B body -> A body
  dd RA[9], tA[3];  // A body -> world
};
// FP32 form: a candidate's two triangles in double-float, relative to A's
// first vertex o (a float) and scaled by 2^-k (k from the largest
// coordinate), so that every intermediate stays well inside the float range.
struct CandDD {
  V3<dd> P[3], Q[3];
  float o[3];
  int k;
  double tau;  // 2 eps
};
// 192 B, moved as twelve 16-B words.
struct alignas(16) AccRec {
  CandDD g;
  int entry, pair;
  int pt_begin, ee_begin, cx_begin;
  int counts;  // point-triangle items | edge-edge items << 8 | crossing items << 16
};
static_assert(sizeof(AccRec) == 192, "AccRec layout");
// Result of one work item in double-float: squared distance (0 for a
// crossing, +inf for an edge that does not cross) and closest points (A's
// frame, relative to o, scaled like the candidate).  64 B, written as four
// 16-B stores.
struct alignas(16) ItemRes {
  dd d2;
  V3<dd> pa, pb;
  float pad[2];
};

// Device counters (one int64 array, zeroed at the start of every detect).
enum Counter : int {
  CNT_LEVEL = 0,                          // [0..kMaxLevels] items in level list l
  CNT_FETCH = CNT_LEVEL + kMaxLevels + 1, // [kMaxLevels+1] dynamic work fetch per kernel
  CNT_TILES = CNT_FETCH + kMaxLevels + 2,
  CNT_CANDS,
  CNT_FALLBACK,                           // one-kernel FP32 form: candidates for the full test
  CNT_SWEEP,                              // [kMaxLevels] entries in level l's sweep list
  CNT_FINE = CNT_SWEEP + kMaxLevels,      // entries in the fine list (all zeroed with the
                                          // rest, so no reset between the kernels)
  CNT_ACC,                                // pairs accepted by the float stage
  CNT_PT,                                 // point-triangle work items
  CNT_EE,                                 // edge-edge work items
  CNT_CX,                                 // edge-against-triangle crossing work items
  CNT_STATS,                              // [MRDEM_STAT_COUNT] statistics
  CNT_TOTAL = CNT_STATS + MRDEM_STAT_COUNT
};

// Latched device status (not cleared by detect; cleared by mrdem_check).
enum Status : int {
  ST_NONFINITE = 0,
  ST_REQ_LEVEL,
  ST_REQ_TILES,
  ST_REQ_CANDS,
  ST_REQ_CONTACTS,
  ST_REQ_SWEEP,
  ST_REQ_ACTIVE,   // active-set items beyond the output's capacity
  ST_TOTAL = 8
};

}  // namespace mrdem

struct mrdem_hier {
  mrdem::HierHost h;
  mrdem_ctx* ctx = nullptr;  // context it was uploaded to
  void* d_mem = nullptr;
  mrdem::HierDev dev{};
};

namespace mrdem {
// Launch shapes of the detection kernels (the tunable part of the params).
struct Shape {
  int level_warps;    // k_expand: warps per block (2, 4, 8)
  int expand_items;   // k_expand: level items per warp and pass, at most (8, 16, 32)
  int node_threads;   // k_sweep_nodes: threads per block (128, 256)
  int tile_warps;     // k_tile: warps per block (2, 4, 8)
  int sweep_warps;    // k_sweep_fine: warps per block (2, 4, 8)
  int exact_threads;  // exact pass: threads per block (64, 128, 256)
  int level_kernel;   // surrogate levels: 0 per-level launches, 1 one cooperative launch
};
constexpr int kSizeClasses = 4;  // particle pairs per call: < 256, < 4096, < 65536, more
inline int size_class(int64_t n_pairs) {
  return n_pairs < 256 ? 0 : n_pairs < 4096 ? 1 : n_pairs < 65536 ? 2 : 3;
}
enum KernelId : int { K_SETUP = 0, K_LEVEL, K_SWEEP_NODES, K_TILE, K_SWEEP_FINE, K_EXACT, K_EXACT64, K_FORCES, K_GRAD, K_PLAIN, K_TRIDIST, K_SORT, K_MERGE, K_BROAD, K_STEP, K_HESSIAN, K_CG, K_COUNT };
struct ProfRec {
  int kernel;
  cudaEvent_t a, b;
};
}  // namespace mrdem

struct mrdem_ctx {
  int device = 0;
  int n_sms = 0;
  mrdem_params params{};
  int4* level_list[2] = {nullptr, nullptr};
  mrdem::TileItem* tiles = nullptr;
  int3* cands = nullptr;
  int4* sweep = nullptr;  // pairs waiting for the penalty sweep (node pairs, then fine pairs)
  mrdem::AccRec* acc = nullptr;     // [cap_cands] pairs accepted by the float stage
  int* items_pt = nullptr;          // [cap_items] point-triangle work items
  int* items_ee = nullptr;          // [cap_items] edge-edge work items
  mrdem::ItemRes* res_pt = nullptr;  // [cap_items]
  mrdem::ItemRes* res_ee = nullptr;  // [cap_items]
  int* items_cx = nullptr;          // [cap_items] crossing work items
  mrdem::ItemRes* res_cx = nullptr;  // [cap_items]
  // each item's squared distance again, packed (the selection reads these)
  mrdem::dd* d2_pt = nullptr;
  mrdem::dd* d2_ee = nullptr;
  mrdem::dd* d2_cx = nullptr;
  int64_t cap_items = 0;
  int64_t cap_level = 0, cap_tiles = 0, cap_cands = 0, cap_sweep = 0;
  mrdem::PairXf* xf = nullptr;
  mrdem::PairXf64* xf64 = nullptr;
  mrdem::PairXfDD* xfdd = nullptr;
  int32_t* pair_cnt = nullptr;  // [cap_pairs]: contacts per pair, then write cursors
  int64_t cap_pairs = 0;
  // detection's contacts before they are ordered by pair (same layout as the
  // caller's buffers, capacity cap_tmp)
  int32_t* tmp_i = nullptr;   // pair, tri_a, tri_b: three arrays of cap_tmp
  double* tmp_d = nullptr;    // dist [cap_tmp], point_a [cap_tmp*3], point_b [cap_tmp*3]
  int64_t* tmp_count = nullptr;
  int64_t cap_tmp = 0;
  // redundant-contact merge: per pair, segment cursors and merged counts
  // (2 * cap_merge_pairs int32); per input entry, working arrays and the
  // merged contacts (cap_merge entries)
  int32_t* merge_seg = nullptr;
  int64_t cap_merge_pairs = 0;
  void* merge_mem = nullptr;
  int64_t cap_merge = 0;
  bool merge_smem_set = false;
  // the large pairs' merge runs beside the small pairs' on a second stream
  cudaStream_t merge_side = nullptr;
  cudaEvent_t merge_ev[2] = {nullptr, nullptr};
  // broad phase of the implicit step: grid record, per-particle cells, order
  // and counts, bucket ends (cap_broad bytes)
  void* broad_mem = nullptr;
  size_t cap_broad = 0;
  // conjugate-gradient solve of the Newton step: state, scalars, vectors
  void* cg_mem = nullptr;
  size_t cap_cg = 0;
  // refinement of a cached candidate list: per candidate its FP64 result
  // and a keep flag
  void* refine_mem = nullptr;
  size_t cap_refine = 0;
  // active sets (Algorithm 6): per input item its outcome and its output
  // count, then output offset (cap_active entries each)
  int8_t* as_status = nullptr;
  int32_t* as_off = nullptr;
  int64_t cap_active = 0;
  double* frames = nullptr;  // [cap_frames * 16]: per particle R (9), t (3), world com (3)
  int64_t cap_frames = 0;
  double* frames_grad = nullptr;  // the adjoint's own tables (it may run beside the forces)
  int64_t cap_frames_grad = 0;
  unsigned long long* counters = nullptr;  // [CNT_TOTAL]
  unsigned long long* status = nullptr;    // [ST_TOTAL]
  // resident blocks per SM of each kernel instance and block shape, filled
  // on first use (a fixed table: a launch never allocates host memory)
  struct Occ {
    const void* kernel;
    int threads;
    size_t smem;
    int blocks;
  };
  Occ occ[64] = {};
  int n_occ = 0;
  // launch shapes chosen by mrdem_autotune per size class (else the params')
  mrdem::Shape tuned[mrdem::kSizeClasses] = {};
  bool tuned_ok[mrdem::kSizeClasses] = {false, false, false, false};
  const mrdem::Shape* force_shape = nullptr;  // set while the autotuner times a shape
  bool prof = false;
  std::vector<mrdem::ProfRec> prof_recs;
  std::vector<cudaEvent_t> ev_pool;
};

namespace mrdem {
// Records an event pair around one kernel launch when profiling is enabled.
struct ProfScope {
  mrdem_ctx* c;
  int id;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(mrdem_ctx* ctx, int kernel, cudaStream_t st) : c(ctx), id(kernel), s(st) {
    if (c->prof) {
      a = take();
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (c->prof && a) {
      cudaEvent_t b = take();
      cudaEventRecord(b, s);
      c->prof_recs.push_back({id, a, b});
    }
  }
  cudaEvent_t take() {
    if (!c->ev_pool.empty()) {
      cudaEvent_t e = c->ev_pool.back();
      c->ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
}  // namespace mrdem

namespace mrdem {
// kernels / launchers (mrdem_detect.cu, mrdem_forces.cu)
int launch_detect(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs, const int32_t* pair_ab,
                  const double* pair_eps, const double* poses, int precision,
                  const mrdem_contacts* out, int64_t* stats, cudaStream_t s);
int launch_plain(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs, const int32_t* pair_ab,
                 const double* pair_eps, const double* poses, const mrdem_contacts* out,
                 cudaStream_t s);
// the finest-level stage of a detection whose leaf-pair tiles are listed:
// tile, fine sweep, exact distance, contacts ordered by pair into out
int launch_fine_tail(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const double* eps,
                     int precision, const mrdem_contacts* tmp, const mrdem_contacts* out,
                     const Shape& sh, cudaStream_t s);
int ensure_pairs(mrdem_ctx* c, int64_t n);
int launch_setup_transforms(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs,
                            const int32_t* ab, const double* eps, const double* poses,
                            cudaStream_t s);
int ensure_tmp(mrdem_ctx* c, int64_t cap, mrdem_contacts* tmp);
SweepConst sweep_const(const mrdem_params& p);
// active sets of the multiresolution implicit step (mrdem_frontier.cu)
int launch_active_init(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs,
                       const int32_t* pair_ab, const mrdem_active_set* out, cudaStream_t s);
int launch_active_step(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs,
                       const int32_t* pair_ab, const double* pair_eps, const double* poses,
                       int precision, const mrdem_active_set* in, const mrdem_active_set* out,
                       const mrdem_contacts* contacts, const mrdem_contacts* surrogate,
                       int64_t* counts, cudaStream_t s);
int launch_surrogate_forces(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs,
                            const int32_t* pair_ab, const double* pair_eps, const double* poses,
                            const mrdem_contacts* sur, const double* mass, const double* com,
                            double k_s, double weight, double* ft, double* energy,
                            cudaStream_t s);
// closest-point pipeline (mrdem_closest.cu)
int launch_exact_fp32(mrdem_ctx* c, const mrdem_hier* hier, const mrdem_contacts* out,
                      int threads, cudaStream_t s);
// launch shapes (mrdem_detect.cu)
Shape shape_for(const mrdem_ctx* c, int64_t n_pairs);
int autotune(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
             const double* eps, const double* poses, int precision, const mrdem_contacts* out,
             int reps, int32_t* chosen, double* ms);
int launch_forces(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs, const int32_t* pair_ab,
                  const double* pair_eps, const double* poses, const mrdem_contacts* c,
                  const double* mass, const double* com, double k_s, double* ft, double* energy,
                  cudaStream_t s);
int launch_grad(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs, const int32_t* pair_ab,
                const double* pair_eps, const double* poses, const mrdem_contacts* c,
                const double* mass, double k_s, double scale, float* dverts, double* dpose,
                double* jac, cudaStream_t s);
// redundant-contact merge (mrdem_merge.cu)
int launch_merge(mrdem_ctx* ctx, int64_t n_pairs, const double* pair_eps, const mrdem_contacts* in,
                 const mrdem_contacts* out, int32_t* members, cudaStream_t s);
// implicit time step (mrdem_step.cu)
int launch_broad_phase(mrdem_ctx* ctx, int32_t n, const double* poses, const double* bound,
                       const double* radius, double eps_rel, int32_t* pairs, double* pair_eps,
                       int64_t cap, int64_t* count, cudaStream_t s);
int launch_move_poses(mrdem_ctx* ctx, int32_t n, const double* poses0, const double* vel,
                      double dt, double* poses, cudaStream_t s);
int launch_twist_grad(mrdem_ctx* ctx, int32_t n, const double* twist, const double* g,
                      double* out, cudaStream_t s);
int launch_picard_update(mrdem_ctx* ctx, int32_t n, const double* vel0, const double* ft,
                         const double* mass, const double* inertia, const double* gravity,
                         double dt, double* vel, double* norms, cudaStream_t s);
int launch_contact_hessian(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                           const int32_t* pair_ab, const double* pair_eps, const double* poses,
                           const mrdem_contacts* c, const double* mass, double k_s,
                           double* blocks, int64_t* skipped, cudaStream_t s);
int launch_newton_residual(mrdem_ctx* ctx, int32_t n, const double* vel0, const double* vel,
                           const double* ft, const double* mass, const double* inertia,
                           const double* gravity, double dt, double* res, double* norms,
                           cudaStream_t s);
int launch_vel_axpy(mrdem_ctx* ctx, int64_t m, double a, const double* x, const double* y,
                    double* out, cudaStream_t s);
int launch_newton_solve(mrdem_ctx* ctx, int32_t n, int64_t n_pairs, const int32_t* pair_ab,
                        const double* blocks, const double* mass, const double* inertia,
                        double dt, const double* rhs, double* x, int32_t max_iter, double rel_tol,
                        int32_t check_every, double* info, cudaStream_t s);
int launch_refine_contacts(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                           const int32_t* pair_ab, const double* pair_eps, const double* poses,
                           const mrdem_contacts* cand, const mrdem_contacts* out, cudaStream_t s);
int launch_motion_bound(mrdem_ctx* ctx, int32_t n, const double* ref, const double* poses,
                        const double* bound, double* out, cudaStream_t s);
int launch_triangle_distance(mrdem_ctx* ctx, int64_t n, const double* P, const double* Q,
                             const double* eps, int precision, double* dist, double* pa,
                             double* pb, int32_t* feature, float* sx, float* sgap, int32_t* sconv,
                             cudaStream_t s);
// device hierarchy builder (mrdem_build.cu): fills *out like the host builder
int build_hierarchy_device(const mrdem_params& p, int32_t n, const int64_t* vert_off,
                           const float* d_verts, const int64_t* tri_off, const int32_t* d_tris,
                           HierHost* out, double* ms);
// host hierarchy builder (mrdem_hierarchy.cpp)
int build_hierarchy_host(const mrdem_params& p, int32_t n, const int64_t* vert_off,
                         const float* verts, const int64_t* tri_off, const int32_t* tris,
                         HierHost* out);
}  // namespace mrdem
