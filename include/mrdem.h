/*
 * mrdem.h -- C ABI of the GB300 multiresolution triangle-mesh contact library.
 *
 * Method: Noble & Weinzierl, "A multiresolution Discrete Element Method for
 * triangulated objects with implicit time stepping" (arXiv 2105.12415).
 * Rigid particles are closed triangle meshes.  Each particle carries a tree of
 * surrogate triangles (Sec. 4, Definition "surrogate tree"; Algorithm 7); each
 * surrogate has a slack delta such that every fine vertex below it lies within
 * delta of it, which makes it conservative (Definition "conservative").  The
 * detection (Algorithm 5) walks the two trees of a particle pair top-down:
 * surrogate pairs whose eps-environments cannot overlap are pruned, the rest
 * are unfolded, and at the finest level every remaining fine triangle pair is
 * compared (Algorithm 4: the penalty sweep of Eq. 3/4 with the comparison-based
 * distance of Sec. 3 as the exact fallback).  A fine triangle pair is a
 * contact iff its distance d satisfies d <= 2 eps (Definition "contact point":
 * |n| <= eps with n half the closest segment).  Penalty forces follow Sec. 2.
 *
 * Conventions for every call:
 *   - return value: MRDEM_OK (0) or a negative MRDEM_ERR_* code; nothing
 *     throws or aborts across this boundary; mrdem_status_string() names it;
 *   - "device" pointers are CUDA device memory owned by the caller (the
 *     Python binding allocates them with torch); "host" pointers are ordinary
 *     host memory owned by the caller;
 *   - arrays are dense, row-major, little-endian, without padding;
 *   - a pose is 7 doubles (tx, ty, tz, qw, qx, qy, qz); the quaternion is
 *     normalised before use; world = R(q) * body + t;
 *   - stream-ordered calls (detect, merge, forces, grad, triangle_distance) enqueue
 *     work on the given cudaStream_t (NULL = legacy default stream), never
 *     synchronise the host and can be captured into a CUDA graph, unless the
 *     call's comment says otherwise.  They keep per-pair and per-particle
 *     scratch in the context, which a call with more pairs or particles than
 *     any earlier one on that context grows (cudaMalloc): make such a call
 *     once before capturing.  Their device-side failures (work-list
 *     overflow, non-finite input) are latched in the context and reported by
 *     mrdem_check().
 */
#ifndef MRDEM_H_
#define MRDEM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrdem_ctx mrdem_ctx;
typedef struct mrdem_hier mrdem_hier;
typedef struct CUstream_st* mrdem_stream; /* same type as cudaStream_t */

/* status codes */
#define MRDEM_OK 0
#define MRDEM_ERR_INVALID (-1)   /* bad argument: size, index, null pointer, degenerate triangle */
#define MRDEM_ERR_OOM (-2)       /* host or device allocation failed */
#define MRDEM_ERR_CUDA (-3)      /* a CUDA runtime call failed (no device, launch error, ...) */
#define MRDEM_ERR_CAPACITY (-4)  /* a device work list or the contact buffer overflowed */
#define MRDEM_ERR_NONFINITE (-5) /* a pose or eps was NaN/Inf, or eps <= 0 */

/* arithmetic of the final distance of candidate triangle pairs */
#define MRDEM_PREC_FP32 0 /* FP32 comparison-based sub-tests with an error bound; the
                             sub-tests within that bound of the float minimum (all of
                             them, and the crossing tests, for crossing or nearly
                             touching pairs) finished in double-float arithmetic (pairs
                             of floats, about 48 significant bits) */
#define MRDEM_PREC_FP64 1 /* FP64 comparison-based distance for every candidate */

/* indices into the int64 statistics array filled by mrdem_detect */
#define MRDEM_STAT_LEVELS 8
#define MRDEM_STAT_TESTS 0       /* [0..7]  surrogate pairs examined at unfold step l (0 = roots) */
#define MRDEM_STAT_SURVIVORS 8   /* [8..15] of which not pruned (sphere test, then sweep) */
#define MRDEM_STAT_TILES 16      /* leaf-pair tiles reaching the finest level */
#define MRDEM_STAT_FINE_TESTS 17 /* fine triangle pairs tested after the cull (face-normal
                                    axes, then the iterative sweep) */
#define MRDEM_STAT_CANDIDATES 18 /* fine pairs not pruned by the sweep's certificate */
#define MRDEM_STAT_UNCONVERGED 19 /* candidates whose sweep had not converged (the paper's odot) */
#define MRDEM_STAT_CONTACTS 20   /* contacts written (or that would have been written) */
#define MRDEM_STAT_FP64 21       /* candidates given the full comparison-based test in extended
                                    precision (FP32 form: crossing or nearly touching pairs) */
#define MRDEM_STAT_SPHERE_TESTS 22 /* fine pairs given the bounding-sphere test */
#define MRDEM_STAT_FINE_SURROGATE 23 /* fine triangles tested against the other leaf's surrogate */
#define MRDEM_STAT_LEVEL_SWEEPS 24 /* surrogate pairs given the penalty sweep (all levels) */
#define MRDEM_STAT_NOALLOC_OVERFLOW 25 /* mrdem_detect_noalloc only: largest size a fixed list or
                                          the contact buffer needed beyond its limit, 0 if none */
#define MRDEM_STAT_NOALLOC_INVALID 26  /* mrdem_detect_noalloc only: non-zero if a pose, eps or
                                          particle index was invalid */
#define MRDEM_STAT_FINE_SWEEPS 27 /* of the fine tests, those the face normals did not
                                     separate, given the iterative sweep */
#define MRDEM_STAT_ITEMS_PT 28   /* FP32 form: point-triangle sub-tests finished in double-float */
#define MRDEM_STAT_ITEMS_EE 29   /* FP32 form: edge-edge sub-tests finished in double-float */
#define MRDEM_STAT_BOX_PRUNED 30 /* child node pairs that passed the sphere test and were pruned
                                    by the oriented boxes around their fine vertices */
#define MRDEM_STAT_COUNT 32

typedef struct mrdem_params {
  int32_t n_iter;   /* penalty-sweep iterations N_iterative (paper: 4) */
  float rho_reg;    /* alpha_regulariser = rho_reg * s, s = mean squared edge length of the pair */
  float rho_iter;   /* alpha_iterative   = rho_iter * s */
  float conv_c;     /* C: converged iff the contact point moved <= C eps in the last iteration */
  int32_t fanout;   /* N_surrogate: clusters per split (paper: 8) */
  int32_t leaf_max; /* a node with more fine triangles than this is split (<= 32) */
  int32_t leaf_min; /* split into fewer than fanout clusters if they would hold fewer */
  int32_t kmeans_iters;
  int64_t cap_level;      /* capacity (items) of each per-level work list */
  int64_t cap_tiles;      /* capacity of the leaf-pair tile list */
  int64_t cap_candidates; /* capacity of the fine candidate list (< 2^27) */
  /* Launch shapes of the detection kernels (mrdem_autotune picks them per
   * device and workload size; these are the shapes used where it has not
   * run).  Each must be one of the listed values. */
  int32_t tile_warps;     /* k_tile, one warp per leaf-pair tile: warps per block (2, 4, 8) */
  int32_t sweep_warps;    /* k_sweep_fine: warps per block (2, 4, 8) */
  int32_t level_warps;    /* k_expand: warps per block (2, 4, 8) */
  int32_t exact_threads;  /* exact-distance kernels: threads per block (64, 128, 256) */
  int64_t cap_sweep;      /* capacity of the list of pairs waiting for the penalty sweep */
  int32_t expand_items;   /* k_expand: level items a warp takes per pass, at most (8, 16, 32) */
  int32_t node_threads;   /* k_sweep_nodes: threads per block (128, 256) */
  int32_t level_kernel;   /* surrogate levels: 0 = two launches per level (k_expand,
                             k_sweep_nodes); 1 = one cooperative launch over all levels,
                             grid-wide barriers between the phases; 2 = one launch per
                             level (k_level: the expand phase's survivors swept by the
                             same warp; level_warps and expand_items set its shape) */
} mrdem_params;

/* Contact output.  All arrays are caller-owned device memory of `capacity`
 * entries; `count` is one device int64 written by mrdem_detect (it may exceed
 * capacity, in which case entries beyond capacity were dropped and
 * mrdem_check reports MRDEM_ERR_CAPACITY).  Entry k is a fine triangle pair
 * (tri_a of particle A, tri_b of particle B, input numbering) of pair[k] with
 * distance dist[k] <= 2 eps and closest points point_a/point_b (world frame;
 * equal when the triangles cross, dist = 0).  Order is unspecified. */
typedef struct mrdem_contacts {
  int64_t capacity;
  int64_t* count;
  int32_t* pair;
  int32_t* tri_a;
  int32_t* tri_b;
  double* dist;
  double* point_a; /* [capacity * 3] */
  double* point_b; /* [capacity * 3] */
} mrdem_contacts;

/* Active sets of the multiresolution implicit Euler step (Algorithm 6, the
 * active set A(p_i, p_j) kept per particle pair across Picard iterations).
 * Per pair, the set is a cut through the product of the two surrogate trees:
 * node pairs (node_a of particle A, node_b of particle B; hierarchy node
 * indices) such that every pair of fine triangles lies below exactly one
 * item, stored in depth-first order of the product tree (a pair's children
 * (a_i, b_j) follow each other, A's child index major; a leaf side stays as
 * it is while the other side unfolds, as in Algorithm 5), the pairs one
 * after another in pair order.  Caller-owned device memory: item
 * [capacity * 4] int32 (pair, node_a, node_b, flags), count one device
 * int64 (may exceed capacity; see mrdem_active_set_step).  flags bit 0:
 * removal vetoed (the memory set U: the item was re-added after its group
 * had been narrowed); bit 1: made by narrowing. */
typedef struct mrdem_active_set {
  int64_t capacity;
  int64_t* count;
  int32_t* item;
} mrdem_active_set;

/* Host-side description of a built hierarchy (see mrdem_hier_export). */
typedef struct mrdem_hier_info {
  int32_t n_particles;
  int32_t max_depth; /* largest number of surrogate levels of any particle */
  int64_t n_nodes;
  int64_t n_tri;     /* fine triangles (input count) */
  int64_t n_tri_pad; /* stored slots: leaves are padded to a multiple of 4 */
  int64_t n_verts;
} mrdem_hier_info;

/* Fill *p with the defaults (paper constants where it gives them:
 * N_iterative = 4, C = 1, N_surrogate = 8). */
void mrdem_default_params(mrdem_params* p);

/* Text for a status code (static storage). */
const char* mrdem_status_string(int status);

/* Create a context on CUDA device `device` with parameters *p (NULL =
 * defaults).  Allocates the device work lists (capacities from *p).
 * Errors: INVALID (bad parameter), CUDA (no such device), OOM. */
int mrdem_create(mrdem_ctx** out, int device, const mrdem_params* p);
int mrdem_destroy(mrdem_ctx* ctx);
int mrdem_get_params(const mrdem_ctx* ctx, mrdem_params* out);
/* Change the sweep constants / launch shapes (not the capacities) of a context. */
int mrdem_set_params(mrdem_ctx* ctx, const mrdem_params* p);
/* Reallocate the work lists (0 keeps a capacity).  Synchronises the device. */
int mrdem_reserve(mrdem_ctx* ctx, int64_t cap_level, int64_t cap_tiles, int64_t cap_candidates,
                  int64_t cap_sweep);

/* Build the surrogate trees of n_particles meshes (Sec. 4, Algorithm 7,
 * Appendix A) on the host.  Host inputs: vert_off [n+1] and tri_off [n+1]
 * (int64 prefix offsets), verts [vert_off[n] * 3] float32 body-frame
 * coordinates, tris [tri_off[n] * 3] int32 vertex indices local to each
 * particle, counter-clockwise seen from outside.  Each node of a tree holds one
 * surrogate triangle; a node with more than leaf_max fine triangles is split by
 * balanced k-means of the triangle centroids into fanout clusters (fewer if
 * clusters would be smaller than leaf_min); leaves hold their fine triangles.
 * Each surrogate's slack delta is the largest FP64 distance from any fine
 * vertex below it to the (float32-rounded) surrogate triangle, rounded up to
 * float32 (the smallest eps that keeps it conservative, Algorithm 7).
 * Deterministic.  `params` supplies fanout/leaf_max/leaf_min/kmeans_iters
 * (NULL = defaults).  *out owns host arrays only (no device memory).
 * Errors: INVALID (index out of range, degenerate triangle, empty particle),
 * OOM. */
int mrdem_build_hierarchy_host(const mrdem_params* params, int32_t n_particles,
                               const int64_t* vert_off, const float* verts,
                               const int64_t* tri_off, const int32_t* tris, mrdem_hier** out);
/* Copy a host-built hierarchy to ctx's device (synchronous). */
int mrdem_hier_upload(mrdem_ctx* ctx, mrdem_hier* hier);
/* mrdem_build_hierarchy_host followed by mrdem_hier_upload. */
int mrdem_build_hierarchy(mrdem_ctx* ctx, int32_t n_particles, const int64_t* vert_off,
                          const float* verts, const int64_t* tri_off, const int32_t* tris,
                          mrdem_hier** out);

/* Build the surrogate trees on the GPU (Sec. 4, Algorithm 7, Appendix A) and
 * keep them on ctx's device: the same tree shape as the host builder (node
 * sizes follow from the counts), clusters from the recursive median split
 * along the principal axis of the triangle centroids (the host builder's
 * k-means seeding; its Lloyd refinement, kmeans_iters, is not run), one
 * surrogate per node fitted on the device, its slack delta the largest FP64
 * distance from a fine vertex below the node to the stored float triangle,
 * rounded up (so every node is conservative), and the oriented boxes.
 * Inputs: vert_off [n+1] and tri_off [n+1] host int64 offsets; verts
 * (device float32 [vert_off[n]*3], body frame) and tris (device int32
 * [tri_off[n]*3], local vertex indices) stay owned by the caller.
 * Synchronous.  build_ms: NULL or host double, the device part's time.
 * *out also holds the host copy (mrdem_hier_export works).  Errors: INVALID
 * (offsets, index out of range, non-finite or degenerate input, degenerate
 * fitted surrogate), OOM, CUDA. */
int mrdem_build_hierarchy_device(mrdem_ctx* ctx, int32_t n_particles, const int64_t* vert_off,
                                 const float* verts, const int64_t* tri_off, const int32_t* tris,
                                 mrdem_hier** out, double* build_ms);
int mrdem_hier_destroy(mrdem_hier* hier);
int mrdem_hier_get_info(const mrdem_hier* hier, mrdem_hier_info* out);
/* Copy the host arrays of a hierarchy into caller host buffers (any may be
 * NULL), sized from mrdem_hier_info:
 *   node_tri    float [n_nodes*9]  surrogate triangle (body frame)
 *   node_delta  float [n_nodes]    slack delta
 *   node_child  int32 [n_nodes*2]  (begin, count): count > 0: child nodes
 *                                  [begin, begin+count); count < 0: leaf with
 *                                  -count fine slots [begin, begin-count)
 *   node_level  int32 [n_nodes]    1 = root
 *   root        int32 [n_particles]
 *   slot_tri    int32 [n_tri_pad]  input triangle index (local) of each fine
 *                                  slot, -1 for padding
 *   slot_particle int32 [n_tri_pad] particle of each slot, -1 for padding */
int mrdem_hier_export(const mrdem_hier* hier, float* node_tri, float* node_delta,
                      int32_t* node_child, int32_t* node_level, int32_t* root,
                      int32_t* slot_tri, int32_t* slot_particle);

/* Copy the oriented box of every node into node_box (host float
 * [n_nodes*16]): centre xyz, three axes (rows, unit length up to float
 * rounding), half extents along them, 0.  The box holds every fine vertex
 * below the node: for each vertex v, |u_k . (v - c)| <= half_k in FP64 with
 * the stored values.  Principal axes of the vertices' covariance.  A further
 * conservative bound of a node's fine geometry beside surrogate + delta: the
 * detection prunes child node pairs whose boxes a face axis separates by more
 * than 2 eps (plus the pair's rounding margin).  Errors: INVALID (null
 * pointers). */
int mrdem_hier_export_boxes(const mrdem_hier* hier, float* node_box);

/* Multiresolution contact detection (Algorithm 5 with the hybrid test of
 * Algorithm 4) for n_pairs particle pairs.  Device inputs: pair_ab [n_pairs*2]
 * int32 particle indices of hier (A, B; A != B not required), pair_eps
 * [n_pairs] eps of each pair (both particles), poses [n_particles*7].
 * `precision` is MRDEM_PREC_FP32 or MRDEM_PREC_FP64.  Writes the contact set
 * of every pair into *out (count overwritten), grouped by pair with the pairs
 * in increasing order (the order within a pair is not fixed); the context
 * keeps a scratch contact list of out's capacity, grown on a call with a
 * larger capacity than before.  stats: NULL or device int64
 * [MRDEM_STAT_COUNT], overwritten.  The result equals the brute-force contact
 * set over all fine triangle pairs (Lemma 1).  Errors returned directly:
 * INVALID (sizes, null pointers, hier not uploaded to ctx), CUDA. */
int mrdem_detect(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs, const int32_t* pair_ab,
                 const double* pair_eps, const double* poses, int32_t precision,
                 const mrdem_contacts* out, int64_t* stats, mrdem_stream stream);

/* Launch-shape autotuner for mrdem_detect (no counterpart in the paper: it
 * picks block sizes and items per warp for this GPU).  Runs the detection of
 * the given batch (same arguments as mrdem_detect; n_pairs >= 1) under nine
 * candidate shapes, reps + 1 times each, times every kernel with CUDA
 * events, and stores for the batch's size class (n_pairs < 256, < 4096,
 * < 65536, larger) the fastest value of each shape parameter: k_expand warps
 * per block and items per warp, k_sweep_nodes threads, k_tile warps,
 * k_sweep_fine warps, exact-pass threads; then the chosen shape once more
 * with the surrogate levels in one cooperative launch (level_kernel 1) and
 * three times with one launch per level (level_kernel 2, at 2, 4 and 8
 * warps per block), the fastest of these kept.  Later mrdem_detect and
 * mrdem_detect_noalloc calls of that size class use them; mrdem_set_params
 * clears the table.  Synchronises the device (do not call during stream
 * capture).  The results of every shape are the same contact set; *out holds
 * the last run's.  chosen: NULL or host int32 [7] (the six values in that
 * order, then level_kernel); ms: NULL or host double [2], the time of one detection with the
 * params' shapes and with the chosen ones.  Errors: INVALID, CUDA, CAPACITY
 * or NONFINITE when a run overflowed a list or met a bad input (status left
 * latched for mrdem_check; grow the lists and call again). */
int mrdem_autotune(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                   const int32_t* pair_ab, const double* pair_eps, const double* poses,
                   int32_t precision, const mrdem_contacts* out, int32_t reps, int32_t* chosen,
                   double* ms);

/* Synchronise `stream` and report the latched device-side status of ctx since
 * the last check: CAPACITY (a work list or a contact buffer overflowed; the
 * required sizes go to required[0..4] = level list, tiles, candidates,
 * contacts, sweep list when required != NULL), NONFINITE, or OK.  Clears the
 * latch. */
int mrdem_check(mrdem_ctx* ctx, mrdem_stream stream, int64_t* required);

/* The same check without a synchronisation of its own, for callers that
 * synchronise anyway (a step whose results go back to the host): enqueues
 * on `stream` a copy of the latched status words into host_words and then
 * clears the latch.  host_words: MRDEM_STATUS_WORDS uint64 of page-locked
 * (pinned) host memory, owned by the caller, valid once the stream has
 * reached that point (after a synchronisation of the caller's own); then
 * mrdem_status_decode reads them.  Stream-ordered, no allocation, no host
 * synchronisation (capturable).  Errors: INVALID (null pointers), CUDA. */
#define MRDEM_STATUS_WORDS 8
int mrdem_status_async(mrdem_ctx* ctx, uint64_t* host_words, mrdem_stream stream);
/* Decode status words copied by mrdem_status_async, as mrdem_check reports
 * them: CAPACITY (required[0..4] as in mrdem_check when required != NULL),
 * NONFINITE or OK.  Host only. */
int mrdem_status_decode(const uint64_t* host_words, int64_t* required);

/* Penalty forces of a contact set (Sec. 2, F(c)):
 *   F = K_s sqrt(mu) (1 - d/(2 eps)) u on A and -F on B,
 *   mu = 1/(1/M_A + 1/M_B), u = (point_a - point_b)/d (at d = 0: minus the
 *   outward unit normal of A's triangle), applied at the contact point
 *   (point_a + point_b)/2; torques about each world centre of mass.
 * Device inputs: the detect inputs, mass [n_particles], com [n_particles*3]
 * (body frame).  Device outputs (accumulated, caller zeroes):
 * force_torque [n_particles*6] (force xyz, torque xyz, world frame) and
 * energy [1] += sum K_s sqrt(mu) eps (1 - d/(2 eps))^2 (whose negative
 * d-derivative is |F|).  Either output may be NULL. */
int mrdem_contact_forces(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                         const int32_t* pair_ab, const double* pair_eps, const double* poses,
                         const mrdem_contacts* contacts, const double* mass, const double* com,
                         double k_s, double* force_torque, double* energy, mrdem_stream stream);

/* Adjoint of the contact energy E = sum_c e(d_c) (the energy of
 * mrdem_contact_forces), scaled by dE_scale (the upstream gradient).  Like
 * mrdem_contact_forces it takes each contact's dist, point_a and point_b as
 * mrdem_detect wrote them, so `contacts` must come from a detection at these
 * poses; the barycentric weights of the closest points (for the float
 * output dE_dverts) are recomputed in float from the body-frame triangles and
 * the world offsets (taken in FP64).  Outputs
 * (accumulated, caller zeroes; each may be NULL):
 *   dE_dverts float [n_verts*3]  gradient w.r.t. body-frame vertex positions
 *                                (vertex numbering of the hierarchy's input)
 *   dE_dpose  double [n_particles*6] gradient w.r.t. a world translation and
 *                                a world rotation increment theta about the
 *                                particle origin (R <- exp([theta]x) R)
 *   jac       double [n_pairs*144] per pair, the Gauss-Newton block
 *                                sum_c e''(d) J J^T of the 12 pose unknowns
 *                                (t_A, theta_A, t_B, theta_B), barycentrics
 *                                frozen, e'' = K_s sqrt(mu)/(2 eps).
 * The paper's implicit step uses Picard iterations (Algorithm 3); these
 * derivatives are what a Newton step needs instead. */
int mrdem_contact_grad(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                       const int32_t* pair_ab, const double* pair_eps, const double* poses,
                       const mrdem_contacts* contacts, const double* mass, double k_s,
                       double dE_scale, float* dE_dverts, double* dE_dpose, double* jac,
                       mrdem_stream stream);

/* Redundant-contact merge (Sec. 2, the implementation note on the contact
 * set: contact points closer than eps are merged into one average point
 * before the set is used).  Within each pair p, contacts i and j are linked
 * when their contact points x = (point_a + point_b)/2 lie closer than
 * pair_eps[p], evaluated in FP64 as ((dx*dx + dy*dy) + dz*dz) < eps*eps with
 * every operation rounded on its own (no fused multiply-add); each connected
 * component of the links becomes one contact whose point_a and point_b are
 * the means of its members' (so its contact point is their mean contact point
 * and its normal their mean normal), dist = |point_a - point_b|, and tri_a,
 * tri_b those of the member with the smallest (tri_a, tri_b).
 * Device inputs: pair_eps [n_pairs]; `in`, any contact list (for example
 * mrdem_detect's output, in any order; entries past min(*in->count,
 * in->capacity) are ignored).  Device outputs: `out` (buffers distinct from
 * in's; count overwritten with the number of merged contacts, which may
 * exceed out->capacity), grouped by pair in increasing order and within a
 * pair by increasing (tri_a, tri_b); members: NULL or int32
 * [out->capacity], the number of contacts merged into each entry.  The result
 * does not depend on the order of `in` (sums run in (tri_a, tri_b) order).
 * The merged list serves mrdem_contact_forces; the adjoint
 * (mrdem_contact_grad) is defined on the unmerged list.  Work per pair grows
 * with the number of its contacts within eps of each other along x
 * (quadratic at worst, for a dense patch).  The context keeps 244 bytes of
 * scratch per entry of in's capacity and 8 per pair, grown on a larger call.
 * Device-side failures latched for mrdem_check: a pair index outside
 * [0, n_pairs) (the entry is dropped) or an eps that is not finite and
 * positive: NONFINITE; more merged contacts than out->capacity: CAPACITY with
 * required[3].  Errors returned directly: INVALID (null pointers,
 * overlapping in/out buffers, n_pairs or a capacity >= 2^31), OOM, CUDA. */
int mrdem_merge_contacts(mrdem_ctx* ctx, int64_t n_pairs, const double* pair_eps,
                         const mrdem_contacts* in, const mrdem_contacts* out, int32_t* members,
                         mrdem_stream stream);

/* ---- implicit time step (Algorithm 3, Sec. 6 many-particle setup)
 *
 * Broad phase: every particle pair i < j whose bounding spheres, widened by
 * the pair's eps, overlap: |c_i - c_j| <= R_i + R_j + 2 eps_ij with
 * eps_ij = eps_rel * 2 * min(r_i, r_j) (eps relative to the smaller
 * particle diameter, Sec. 6).
 *   poses   device double [n*7] (centre xyz, quaternion wxyz); only the
 *           centres are read;
 *   bound   device double [n]: bounding radius R_i of particle i about its
 *           centre (the largest distance of a vertex from the body origin);
 *   radius  device double [n]: the radius r_i that scales eps;
 *   pairs   device int32 [cap*2] and pair_eps device double [cap]: the
 *           candidates ordered by (i, j) and their eps_ij (the inputs
 *           mrdem_detect takes);
 *   count   device int64: the number of candidates.  When it exceeds cap
 *           nothing is written to pairs / pair_eps: grow to count and call
 *           again.
 * The decision |c_i - c_j| <= ... is taken in FP64 without fused
 * multiply-adds ((dx^2 + dy^2) + dz^2, sqrt; (R_i + R_j) + 2 eps_ij), so the
 * list is a deterministic function of the inputs.  Particles are sorted into
 * up to 8 size classes by R (class k: R in (R_max/2^(k+1), R_max/2^k]), each
 * with a uniform grid of cells of side 2 R_max/2^k, all hashed into 2^k >= 2n
 * buckets; a particle searches each class's cells within R_i + R_max/2^k +
 * 4 eps_rel r_i of its centre (or that class's particles, when fewer), so
 * big particles among small ones do not coarsen the small ones' cells.  The
 * context keeps about 36 n + 4 * 2^k bytes of scratch, grown on a larger
 * call.  Device-side failure latched for mrdem_check: a centre,
 * bound or radius that is not finite, or a negative bound or radius:
 * NONFINITE (count is then 0).  Errors returned directly: INVALID (null
 * pointers, n > 2^26, cap >= 2^31, eps_rel negative or not finite), OOM,
 * CUDA.  Stream-ordered, no host synchronisation. */
int mrdem_broad_phase(mrdem_ctx* ctx, int32_t n, const double* poses, const double* bound,
                      const double* radius, double eps_rel, int32_t* pairs, double* pair_eps,
                      int64_t cap, int64_t* count, mrdem_stream stream);

/* Rigid-body pose update of the implicit Euler step: for each particle,
 * centre' = centre + dt v and orientation' = quat(dt omega) * orientation
 * (the rotation vector dt omega applied in the world frame), renormalised.
 *   poses0  device double [n*7] (centre xyz, quaternion wxyz, any norm > 0);
 *   vel     device double [n*6]: (v xyz, omega xyz) in the world frame;
 *   poses   device double [n*7] output; may be poses0 itself, not vel.
 * Errors: INVALID (null pointers, dt not finite, vel == poses), CUDA. */
int mrdem_move_poses(mrdem_ctx* ctx, int32_t n, const double* poses0, const double* vel,
                     double dt, double* poses, mrdem_stream stream);

/* The chain rule of a pose twist (extension of the adjoint, no counterpart
 * in the paper): for poses moved by twist [n*6] (device FP64: a world
 * translation v and a rotation vector w per particle, the orientation turned
 * on the left, as mrdem_move_poses with dt = 1), out [n*6] = the gradient of
 * the energy in the twist, from grad_pose [n*6] = its gradient in a
 * translation and a left rotation increment at the moved poses (what
 * mrdem_contact_grad returns there): out = (g_t, J_l(w)^T g_r), J_l the left
 * Jacobian of the rotation exponential.  out may alias grad_pose.  Errors:
 * INVALID, CUDA. */
int mrdem_twist_grad(mrdem_ctx* ctx, int32_t n, const double* twist, const double* grad_pose,
                     double* out, mrdem_stream stream);

/* One Picard update of the implicit Euler step (Algorithm 3): from the
 * contact forces and torques at the geometry moved by the guessed
 * velocities, new velocities
 *   v' = v0 + dt (F / m + g),   omega' = omega0 + dt tau / I
 * (isotropic inertia I per particle; torques about the centre of mass).
 *   vel0          device double [n*6]: velocities at the start of the step;
 *   force_torque  device double [n*6]: (F, tau) at the guessed geometry
 *                 (mrdem_contact_forces' output);
 *   mass, inertia device double [n];
 *   gravity       HOST double [3];
 *   vel           device double [n*6]: in, the guess; out, the update;
 *   norms         device double [2]: out, (max |v' - guess|, max |v'|) over
 *                 all components, the iteration's convergence measure (NaN
 *                 if any update is NaN).
 * Errors: INVALID (null pointers, dt or gravity not finite, vel aliasing
 * vel0 or force_torque), CUDA. */
int mrdem_picard_update(mrdem_ctx* ctx, int32_t n, const double* vel0,
                        const double* force_torque, const double* mass, const double* inertia,
                        const double* gravity, double dt, double* vel, double* norms,
                        mrdem_stream stream);

/* Contact Hessian for Newton's method on the implicit Euler equations: for
 * every contact of the list with 0 < d <= 2 eps, the second derivatives of
 * its energy e(d) = K_s sqrt(mu) eps (1 - d/(2 eps))^2 (Sec. 2 force law) in
 * the pair's two pose twists, with the closest points free to move, added to
 * blocks[p] of its pair p (device double [n_pairs*144], row-major 12x12, rows
 * and columns (t_A, theta_A, t_B, theta_B); t a world translation, theta a
 * world rotation increment about the particle origin applied on the left of
 * R; accumulated, the caller zeroes).  The closest points and their features
 * are recomputed in FP64 from the world triangles (the contact list only
 * names the triangle pairs), so the blocks do not depend on the precision
 * form of the detection.  Skipped: crossing triangles (d = 0, where d is not
 * differentiable) and contacts between parallel features (an edge on a face,
 * two faces), counted in *skipped (device int64, accumulated, nullable).
 * Errors: INVALID (null pointers, k_s negative or not finite), CUDA. */
int mrdem_contact_hessian(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                          const int32_t* pair_ab, const double* pair_eps, const double* poses,
                          const mrdem_contacts* contacts, const double* mass, double k_s,
                          double* blocks, int64_t* skipped, mrdem_stream stream);

/* Residual of the implicit Euler equations at velocities vel (Newton's
 * method on Algorithm 3's fixed point):
 *   res = M (vel - vel0) / dt - force_torque - (m g, 0),
 * M = diag(m, m, m, I, I, I), force_torque the contact forces and torques at
 * the geometry moved by dt vel (mrdem_move_poses, mrdem_detect,
 * mrdem_contact_forces).  Device double [n*6] each; mass, inertia [n];
 * gravity HOST double [3].  norms (device double [2]) receives
 * (max |res|, max |M vel| / dt), the convergence test's two sides.  Rounded
 * operation by operation in the order written.  Errors: INVALID (null
 * pointers, dt not positive and finite, gravity not finite), CUDA. */
int mrdem_newton_residual(mrdem_ctx* ctx, int32_t n, const double* vel0, const double* vel,
                          const double* force_torque, const double* mass, const double* inertia,
                          const double* gravity, double dt, double* res, double* norms,
                          mrdem_stream stream);

/* Newton step of the implicit Euler equations: solves
 *   (M/dt + dt K) x = rhs,   K = sum over pairs of the pair's 12x12 block
 * (mrdem_contact_hessian's layout) placed at its two particles' twists,
 * by conjugate gradients with the diagonal as preconditioner (an entry that
 * is not positive uses M/dt instead), from x = 0, stopping when
 * |r| <= rel_tol |rhs| or after max_iter iterations.  The whole solve is
 * one cooperative kernel launch that loops and stops on the device (no host
 * synchronisation); check_every is accepted and ignored.  pair_ab int32
 * [n_pairs*2], blocks double [n_pairs*144], mass and
 * inertia [n], rhs and x [n*6]: device.  info (device double [4]) receives
 * (iterations, |r|/|rhs|, 1 if p.Ap <= 0 stopped it (K not positive
 * definite enough; x is then the last iterate, or, when the first
 * direction p already has p.Ap < 0, the step (r.z / |p.Ap|) p), |rhs|).  The context keeps 240 n + 24 max_iter bytes of
 * scratch.  Errors: INVALID (null pointers, rhs == x, n > 2^26,
 * max_iter outside [0, 100000], rel_tol or check_every negative), OOM,
 * CUDA. */
int mrdem_newton_solve(mrdem_ctx* ctx, int32_t n, int64_t n_pairs, const int32_t* pair_ab,
                       const double* blocks, const double* mass, const double* inertia,
                       double dt, const double* rhs, double* x, int32_t max_iter, double rel_tol,
                       int32_t check_every, double* info, mrdem_stream stream);

/* out = y + a x over m doubles (device; out may be y or x): the trial
 * velocities of a line search along a Newton step.  Errors: INVALID, CUDA. */
int mrdem_vel_axpy(mrdem_ctx* ctx, int64_t m, double a, const double* x, const double* y,
                   double* out, mrdem_stream stream);

/* Contacts of a cached candidate list (the active set kept across the
 * iterations of one implicit step): for every listed triangle pair of
 * `candidates` (pair, tri_a, tri_b; its other fields are not read), the
 * exact FP64 comparison-based distance of the two world triangles at
 * `poses`; pairs with d <= 2 eps (pair_eps) are written to `out` in the
 * list's order (pair, triangles, d, closest points in the world frame, as
 * mrdem_detect writes them), out->count = their number.  With candidates
 * from mrdem_detect at eps + w at reference poses, the result equals
 * mrdem_detect at eps at any poses whose points moved by at most w from
 * the reference ones (triangle distances change by at most the sum of the
 * two particles' displacements; see mrdem_motion_bound).  The context keeps
 * 60 bytes per entry of the candidates' capacity.  Device-side failure
 * latched for mrdem_check: more contacts than out->capacity: CAPACITY with
 * required[3].  Errors: INVALID (null pointers, overlapping buffers,
 * capacities >= 2^31), OOM, CUDA. */
int mrdem_refine_contacts(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                          const int32_t* pair_ab, const double* pair_eps, const double* poses,
                          const mrdem_contacts* candidates, const mrdem_contacts* out,
                          mrdem_stream stream);

/* Initial active sets of Algorithm 6: one item (pair, root of A, root of B,
 * 0) per pair, out->count = n_pairs (an invalid particle index gives nodes
 * -1, which later steps keep as they are).  Errors: INVALID (null pointers,
 * out->capacity < n_pairs), CUDA. */
int mrdem_active_set_init(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                          const int32_t* pair_ab, const mrdem_active_set* out,
                          mrdem_stream stream);

/* One detection of Algorithm 6 on the active sets `in` at `poses`, and the
 * next active sets in `out` (a distinct buffer).  Each item's two surrogates
 * get the certified tests of a surrogate level (node spheres, oriented
 * boxes, the float penalty sweep with its certificate and the face normals,
 * threshold delta_a + delta_b + 2 eps):
 *   - certified apart (bottom): kept, unless all items of its sibling group
 *     (the children of one pair, listed side by side) are bottom and none is
 *     vetoed: the group is then replaced by that pair, with flag bit 1
 *     (narrowing);
 *   - not apart, both nodes leaves: kept; its fine triangle pairs go through
 *     the finest-level stage and exact distance of mrdem_detect, and the
 *     contacts (d <= 2 eps) are written to `contacts` grouped by pair;
 *   - not apart otherwise: replaced by its children (widening; they carry
 *     flag bit 0 when the item carried bit 0 or 1); when the sweep converged
 *     and its iterate's distance d is <= delta_a + delta_b + 2 eps, a
 *     surrogate contact is appended to `surrogate`: pair, tri_a = node_a,
 *     tri_b = node_b (node indices), dist = d, point_a/point_b the iterate's
 *     points in the world frame (not ordered).
 * counts: NULL or device int64[4]: items widened, groups narrowed, pairs of
 * leaves compared, surrogate contacts.  Stream-ordered, no host
 * synchronisation (capturable after a first call with the same sizes).  The
 * context keeps 5 bytes per item of in->capacity.  Device-side failures
 * latched for mrdem_check: out->count > out->capacity (items beyond
 * dropped) or more contacts than a buffer holds: CAPACITY; non-finite
 * input: NONFINITE.  Errors: INVALID (null pointers, in == out, capacities
 * >= 2^31), OOM, CUDA. */
int mrdem_active_set_step(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                          const int32_t* pair_ab, const double* pair_eps, const double* poses,
                          int precision, const mrdem_active_set* in,
                          const mrdem_active_set* out, const mrdem_contacts* contacts,
                          const mrdem_contacts* surrogate, int64_t* counts,
                          mrdem_stream stream);

/* Forces of surrogate contacts (Algorithm 6's implicit guess, weighted down
 * on coarse levels): for each entry of `surrogate` (as mrdem_active_set_step
 * writes it), with tau = delta_a + delta_b + 2 eps of its two nodes, adds
 * weight * k_s * sqrt(mu) * max(0, 1 - d / tau) * u to A's force and its
 * negative to B's (u = (point_a - point_b) / d, or minus A's surrogate normal
 * in the world frame when d = 0; mu = 1 / (1/m_A + 1/m_B)), applied at
 * (point_a + point_b) / 2, torques about each particle's centre of mass (com:
 * device double [n*3], body frame), into force_torque (device double
 * [n*6], accumulated, not cleared), and weight * k_s * sqrt(mu) * tau / 2 *
 * (1 - d / tau)^2 per entry into *energy (NULL: not computed).  Errors:
 * INVALID (weight outside [0, 1], k_s < 0, null pointers), CUDA. */
int mrdem_surrogate_forces(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                           const int32_t* pair_ab, const double* pair_eps, const double* poses,
                           const mrdem_contacts* surrogate, const double* mass,
                           const double* com, double k_s, double weight, double* force_torque,
                           double* energy, mrdem_stream stream);

/* Largest displacement of any point of any particle between poses_ref and
 * poses (device double [n*7] each): |t - t_ref| + theta * bound, theta the
 * angle of the rotation taking the reference orientation to the current
 * one, bound (device double [n]) the particle's largest vertex distance
 * from its origin; written to *out (device double).  Errors: INVALID,
 * CUDA. */
int mrdem_motion_bound(mrdem_ctx* ctx, int32_t n, const double* poses_ref, const double* poses,
                       const double* bound, double* out, mrdem_stream stream);

/* Plain GPU form (reported baseline): the contact set by FP64 comparison-based
 * distance over ALL fine triangle pairs of each pair (Algorithm 2), no
 * hierarchy, one kernel launch per particle pair.  Same inputs and outputs as
 * mrdem_detect.  Copies pair_ab to the host and synchronises `stream` (not
 * capturable). */
int mrdem_detect_plain_fp64(mrdem_ctx* ctx, const mrdem_hier* hier, int64_t n_pairs,
                            const int32_t* pair_ab, const double* pair_eps, const double* poses,
                            const mrdem_contacts* out, mrdem_stream stream);

/* Triangle-pair kernel entry (Sec. 3): for n explicit pairs of triangles
 * P[k], Q[k] (device double [n*9] each, vertices v0 v1 v2, any common frame)
 * and eps[k]:
 *   dist/point_a/point_b/feature: exact distance by the comparison-based
 *     method in the requested precision (FP32: the float-rounded triangles
 *     relative to P's first vertex; FP64: as given).  feature codes: k (0..2)
 *     vertex k of P vs Q; 3+k vertex k of Q vs P; 6+3i+j edge i of P vs edge j
 *     of Q (edge i joins vertex i and i+1 mod 3); 100+i edge i of P crosses Q;
 *     103+j edge j of Q crosses P.  The FP32 form is the detection's: float
 *     sub-tests, then double-float finishing; its feature code is -2 for a
 *     pair it decides to be beyond 2 eps (the reported distance is then the
 *     full double result).
 *   sweep_x [n*4], sweep_gap [n], sweep_conv [n]: the FP32 penalty sweep of
 *     Eq. 3/4 (ctx's constants) on the float-rounded triangles: final
 *     barycentric unknowns (a1, b1, a2, b2), the certified lower bound of the
 *     distance along the final iterate's direction (-inf if undefined), and
 *     whether the contact point moved <= C eps in the last iteration.
 * Any output may be NULL. */
int mrdem_triangle_distance(mrdem_ctx* ctx, int64_t n, const double* P, const double* Q,
                            const double* eps, int32_t precision, double* dist, double* point_a,
                            double* point_b, int32_t* feature, float* sweep_x, float* sweep_gap,
                            int32_t* sweep_conv, mrdem_stream stream);

/* Detection for callers that may not allocate device memory.  Some callers
 * own every byte of device memory themselves: a simulation host that hands
 * this library a fixed memory budget at start-up, or a real-time loop that
 * must not call cudaMalloc/cudaFree after initialisation because those calls
 * synchronise the device and can stall the loop.  They cannot use
 * mrdem_detect, whose context allocates its work lists (and grows them on
 * demand).  This call does the same work as mrdem_detect with the same
 * kernels, but every work list lives in one fixed array in device memory that
 * is part of the library image (about 7.2 MB; every GPU that loads the library
 * holds it until the process exits).  It allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.  The method has no counterpart of
 * this call in the paper; it is a deployment variant of mrdem_detect.
 *
 * Arguments: as mrdem_detect, without a context: hier must have been
 * uploaded (its context supplies the device, the sweep constants and the
 * launch shapes; the surrogate levels always take two launches each, as
 * level_kernel 0); stats is required (device int64 [MRDEM_STAT_COUNT]).
 * Limits: n_pairs <= 1024 (larger: MRDEM_ERR_INVALID, nothing enqueued); per
 * call at most 65536 node-pair items per level, 65536 leaf-pair tiles, 131072
 * pairs waiting for a sweep and 65536 fine candidates.  Work beyond a limit
 * is dropped: after the stream completes, stats[MRDEM_STAT_NOALLOC_OVERFLOW]
 * holds the size that would have been needed (0 when nothing overflowed; the
 * contact buffer's overflow is reported there too) and the contact set is
 * then incomplete; stats[MRDEM_STAT_NOALLOC_INVALID] is non-zero when an
 * input was invalid.  These flags are not latched in the context.
 * The first call on a device looks up the device address of the fixed array;
 * make that first call before any stream capture.  Every call on a device
 * shares the one array and clears its counters on entry, so calls that
 * overlap on the GPU (concurrent streams, or host threads on one device)
 * race and corrupt each other's results: serialise them.  Returns
 * MRDEM_ERR_INVALID for bad arguments, MRDEM_ERR_CUDA if a launch failed. */
int mrdem_detect_noalloc(const mrdem_hier* hier, int64_t n_pairs, const int32_t* pair_ab,
                         const double* pair_eps, const double* poses, int32_t precision,
                         const mrdem_contacts* out, int64_t* stats, mrdem_stream stream);

/* Kernel timing for benchmarks (not part of the method).  While enabled, the
 * context records a CUDA event pair on the launch stream around every kernel
 * it launches (do not enable it during stream capture).  mrdem_profile_read
 * synchronises the device, writes up to n_max entries (kernel name in static
 * storage, total milliseconds, launch count) accumulated since the previous
 * read, sets *n_out and clears the totals. */
int mrdem_profile(mrdem_ctx* ctx, int32_t enable);
int mrdem_profile_read(mrdem_ctx* ctx, int32_t n_max, const char** names, double* ms,
                       int64_t* launches, int32_t* n_out);

#ifdef __cplusplus
}
#endif
#endif /* MRDEM_H_ */
