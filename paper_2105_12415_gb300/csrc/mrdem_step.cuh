// mrdem_step.cuh -- per-particle arithmetic of the implicit time step
// (Algorithm 3): the broad phase that lists the candidate particle pairs, the
// rigid-body pose update and the Picard update of the velocities.  Host and
// device functions, so the kernels in mrdem_step.cu are thin loops around them.
//
// Broad phase.  Particle i has centre c_i (the translation of its pose),
// bounding radius R_i about it and radius r_i; pair eps_ij = eps_rel 2 min(r_i, r_j)
// (eps relative to the smaller particle diameter, Sec. 6).  A pair i < j is a
// candidate when the bounding spheres widened by eps_ij overlap:
//   |c_i - c_j| <= R_i + R_j + 2 eps_ij.
// Particles are sorted into size classes by R, each class with a grid of its
// own (cells hashed into one power-of-two table with the spatial hash of
// Teschner et al. 2003, "Optimized spatial hashing for collision detection of
// deformable objects", the class mixed into the hash); a bucket can hold
// several cells, so a particle found in a bucket counts only if its own cell
// and class are the ones being visited, which also keeps a particle from
// being seen twice when two visited cells share a bucket.  The distance test
// runs in FP64 without fused multiply-adds, term by term
// ((dx^2 + dy^2) + dz^2, then sqrt), so its decisions do not depend on the
// compiler.
#pragma once

#include <math.h>
#include <stdint.h>

#include "mrdem_geometry.cuh"

namespace mrdem {

// Size classes: class k holds the bounding radii R in (R_max/2^(k+1),
// R_max/2^k], the last class everything smaller; each class has its own grid
// of cells of side 2 R_max/2^k, hashed into one shared table.  Particle i
// finds its candidates of class b in the cells of b's grid that meet the box
// of half-width R_i + R_max/2^b + 4 eps_rel r_i around c_i (every candidate
// j of class b lies in it: R_j <= R_max/2^b and 2 eps_ij <= 4 eps_rel r_i),
// or, when that box holds more cells than class b has particles, by running
// through class b's particles.  So a few big particles among many small
// ones cost the small ones nothing: cells are sized per class, not by the
// largest particle.
constexpr int kMaxClasses = 8;

// Grid of the broad phase, written by the bounds kernel.
struct BroadGrid {
  double lo[3];                 // smallest centre coordinate per axis
  double r_max;                 // largest bounding radius
  double h[kMaxClasses];        // cell side of class k
  double inv_h[kMaxClasses];
  int32_t classes;              // number of classes K
  int32_t bad;                  // a centre, bound or radius was not finite (or negative)
};

// Cell sides and search radii are widened by this relative slack, and the
// search box by a few ulps of the coordinates, so that rounding in
// (x - lo) * inv_h cannot leave a candidate outside the cells visited.
constexpr double kCellSlack = 1.0 + 1.0 / 65536.0;
constexpr double kCellMax = 1073741824.0;  // cell coordinates are clamped to [0, 2^30]

MRDEM_HD double bp_mul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}

MRDEM_HD double bp_add(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}

// Upper end R_max / 2^k of class k (exact: a power-of-two scaling).
MRDEM_HD double bp_class_top(double r_max, int k) { return ldexp(r_max, -k); }

// Number of classes for radii in [r_min, r_max]: enough that the smallest
// radius falls in the last one, at most kMaxClasses.
MRDEM_HD int bp_classes(double r_max, double r_min) {
  int K = 1;
  while (K < kMaxClasses && r_min <= bp_class_top(r_max, K)) ++K;
  return K;
}

// Class of bounding radius R.
MRDEM_HD int bp_class(double R, double r_max, int K) {
  int k = 0;
  while (k < K - 1 && R <= bp_class_top(r_max, k + 1)) ++k;
  return k;
}

// Cell side of class k.
MRDEM_HD double bp_cell_side(double r_max, int k) {
  const double h = 2.0 * bp_class_top(r_max, k) * kCellSlack;
  return h > 0.0 ? h : 1.0;  // all zero: candidates coincide, any side will do
}

// Cell coordinate along one axis; monotone in x, clamped to [0, 2^30].
MRDEM_HD int32_t bp_cell(double x, double lo, double inv_h) {
  const double q = (x - lo) * inv_h;
  if (!(q > 0.0)) return 0;
  if (q >= kCellMax) return (int32_t)kCellMax;
  return (int32_t)q;  // truncation = floor for q > 0
}

// Bucket of cell (x, y, z) of class k in a table of 2^log2_t buckets.
MRDEM_HD uint32_t bp_bucket(int32_t x, int32_t y, int32_t z, int32_t k, int log2_t) {
  const uint32_t hsh = ((uint32_t)x * 73856093u) ^ ((uint32_t)y * 19349663u) ^
                       ((uint32_t)z * 83492791u) ^ ((uint32_t)k * 1566083941u);
  return hsh & ((1u << log2_t) - 1u);
}

// eps of pair (i, j): eps_rel * 2 * min(r_i, r_j), in that order of operations.
MRDEM_HD double bp_pair_eps(double r_i, double r_j, double eps_rel) {
  return bp_mul(eps_rel * 2.0, r_i < r_j ? r_i : r_j);
}

// The candidate test |c_i - c_j| <= R_i + R_j + 2 eps_ij.
MRDEM_HD bool bp_candidate(const double* ci, const double* cj, double Ri, double Rj, double eij) {
  const double dx = ci[0] - cj[0], dy = ci[1] - cj[1], dz = ci[2] - cj[2];
  double s = bp_mul(dx, dx);
  s = bp_add(s, bp_mul(dy, dy));
  s = bp_add(s, bp_mul(dz, dz));
  const double lim = bp_add(bp_add(Ri, Rj), bp_mul(2.0, eij));
  return sqrt(s) <= lim;
}

// Input arrays of the broad phase (device pointers in the kernels).
struct BroadIn {
  const double* poses;   // [n*7]: centre xyz, quaternion wxyz
  const double* bound;   // [n] bounding radius about the centre
  const double* radius;  // [n]
  double eps_rel;
  int32_t n;
};

// Cell of a particle: coordinates in its class's grid, class, bucket.
struct alignas(8) BroadCell {
  int32_t x, y, z, k;
  uint32_t b;
  int32_t pad;
};

// Working arrays: cell[i] of particle i; order = the particles grouped by
// bucket, bucket_end[b] = one past the last entry of bucket b in order
// (bucket b starts at bucket_end[b - 1], or 0); class_order = the particles
// grouped by class, class_end[k] likewise.
struct BroadWork {
  BroadCell* cell;
  int32_t* order;
  int32_t* bucket_end;
  int32_t* class_order;
  int32_t* class_end;
  int log2_t;
};

// Cell of particle i from its centre and bounding radius.
MRDEM_HD BroadCell bp_cell_of(const BroadIn& in, const BroadGrid& g, int32_t i, int log2_t) {
  const double* c = in.poses + (int64_t)7 * i;
  BroadCell cl;
  cl.k = bp_class(in.bound[i], g.r_max, g.classes);
  cl.x = bp_cell(c[0], g.lo[0], g.inv_h[cl.k]);
  cl.y = bp_cell(c[1], g.lo[1], g.inv_h[cl.k]);
  cl.z = bp_cell(c[2], g.lo[2], g.inv_h[cl.k]);
  cl.b = bp_bucket(cl.x, cl.y, cl.z, cl.k, log2_t);
  cl.pad = 0;
  return cl;
}

// Visits the candidates j > i of particle i, class by class; calls f(j, eps_ij)
// for each and returns how many there were.
template <typename F>
MRDEM_HD int32_t bp_visit(const BroadIn& in, const BroadGrid& g, const BroadWork& w, int32_t i,
                          F f) {
  const double* ci = in.poses + (int64_t)7 * i;
  const double Ri = in.bound[i], ri = in.radius[i];
  int32_t found = 0;
  auto test = [&](int32_t j) {
    if (j <= i) return;
    const double eij = bp_pair_eps(ri, in.radius[j], in.eps_rel);
    if (!bp_candidate(ci, in.poses + (int64_t)7 * j, Ri, in.bound[j], eij)) return;
    f(j, eij);
    ++found;
  };
  for (int b = 0; b < g.classes; ++b) {
    const int32_t beg = b ? w.class_end[b - 1] : 0, end = w.class_end[b];
    if (end <= beg) continue;
    const double rho = (Ri + bp_class_top(g.r_max, b) + 4.0 * in.eps_rel * ri) * kCellSlack;
    int32_t lo[3], hi[3];
    double ncells = 1.0;
    for (int a = 0; a < 3; ++a) {
      const double pad = (fabs(ci[a]) + fabs(g.lo[a]) + rho) * 0x1p-48;
      lo[a] = bp_cell(ci[a] - rho - pad, g.lo[a], g.inv_h[b]);
      hi[a] = bp_cell(ci[a] + rho + pad, g.lo[a], g.inv_h[b]);
      ncells *= (double)(hi[a] - lo[a] + 1);
    }
    if (ncells > (double)(end - beg)) {
      for (int32_t q = beg; q < end; ++q) test(w.class_order[q]);
      continue;
    }
    for (int32_t z = lo[2]; z <= hi[2]; ++z)
      for (int32_t y = lo[1]; y <= hi[1]; ++y)
        for (int32_t x = lo[0]; x <= hi[0]; ++x) {
          const uint32_t bk = bp_bucket(x, y, z, b, w.log2_t);
          const int32_t kb = bk ? w.bucket_end[bk - 1] : 0, ke = w.bucket_end[bk];
          for (int32_t q = kb; q < ke; ++q) {
            const int32_t j = w.order[q];
            const BroadCell cj = w.cell[j];
            if (cj.k == b && cj.x == x && cj.y == y && cj.z == z) test(j);
          }
        }
  }
  return found;
}

// The same visit split over `nl` lanes: lane `l` takes every nl-th unit of
// work (a cell of a class's search box, or a particle of a class run
// through directly), so the lanes together visit every candidate of i
// exactly once.  Returns the candidates this lane found.
template <typename F>
MRDEM_HD int32_t bp_visit_lane(const BroadIn& in, const BroadGrid& g, const BroadWork& w, int32_t i,
                               int l, int nl, F f) {
  const double* ci = in.poses + (int64_t)7 * i;
  const double Ri = in.bound[i], ri = in.radius[i];
  int32_t found = 0;
  auto test = [&](int32_t j) {
    if (j <= i) return;
    const double eij = bp_pair_eps(ri, in.radius[j], in.eps_rel);
    if (!bp_candidate(ci, in.poses + (int64_t)7 * j, Ri, in.bound[j], eij)) return;
    f(j, eij);
    ++found;
  };
  for (int b = 0; b < g.classes; ++b) {
    const int32_t beg = b ? w.class_end[b - 1] : 0, end = w.class_end[b];
    if (end <= beg) continue;
    const double rho = (Ri + bp_class_top(g.r_max, b) + 4.0 * in.eps_rel * ri) * kCellSlack;
    int32_t lo[3], hi[3];
    double ncells = 1.0;
    for (int a = 0; a < 3; ++a) {
      const double pad = (fabs(ci[a]) + fabs(g.lo[a]) + rho) * 0x1p-48;
      lo[a] = bp_cell(ci[a] - rho - pad, g.lo[a], g.inv_h[b]);
      hi[a] = bp_cell(ci[a] + rho + pad, g.lo[a], g.inv_h[b]);
      ncells *= (double)(hi[a] - lo[a] + 1);
    }
    if (ncells > (double)(end - beg)) {
      for (int32_t q = beg + l; q < end; q += nl) test(w.class_order[q]);
      continue;
    }
    const int64_t nx = hi[0] - lo[0] + 1, ny = hi[1] - lo[1] + 1;
    const int64_t nc = (int64_t)ncells;
    for (int64_t u = l; u < nc; u += nl) {
      const int32_t x = lo[0] + (int32_t)(u % nx), y = lo[1] + (int32_t)((u / nx) % ny);
      const int32_t z = lo[2] + (int32_t)(u / (nx * ny));
      const uint32_t bk = bp_bucket(x, y, z, b, w.log2_t);
      const int32_t kb = bk ? w.bucket_end[bk - 1] : 0, ke = w.bucket_end[bk];
      for (int32_t q = kb; q < ke; ++q) {
        const int32_t j = w.order[q];
        const BroadCell cj = w.cell[j];
        if (cj.k == b && cj.x == x && cj.y == y && cj.z == z) test(j);
      }
    }
  }
  return found;
}

// ---- rigid-body update and Picard iteration (Algorithm 3)

// Unit quaternion (w, x, y, z) of the rotation by rotation vector r.
MRDEM_HD void rotvec_to_quat(const double r[3], double q[4]) {
  const double th = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (th == 0.0) {
    q[0] = 1.0;
    q[1] = q[2] = q[3] = 0.0;
    return;
  }
  const double s = sin(0.5 * th) / th;
  q[0] = cos(0.5 * th);
  q[1] = s * r[0];
  q[2] = s * r[1];
  q[3] = s * r[2];
}

// Hamilton product a * b.
MRDEM_HD void quat_mul(const double a[4], const double b[4], double out[4]) {
  out[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  out[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  out[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  out[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Rotation matrix (row-major) of quaternion q = (w, x, y, z) of any norm.
MRDEM_HD void quat_matrix(const double* q, double R[9]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  const double s = 2.0 / (w * w + x * x + y * y + z * z);
  R[0] = 1.0 - s * (y * y + z * z); R[1] = s * (x * y - w * z);       R[2] = s * (x * z + w * y);
  R[3] = s * (x * y + w * z);       R[4] = 1.0 - s * (x * x + z * z); R[5] = s * (y * z - w * x);
  R[6] = s * (x * z - w * y);       R[7] = s * (y * z + w * x);       R[8] = 1.0 - s * (x * x + y * y);
}

// World position R v + t of body-frame point v under pose (t, q).
MRDEM_HD V3<double> pose_point(const double R[9], const double* t, const V3<double>& v) {
  return {R[0] * v.x + R[1] * v.y + R[2] * v.z + t[0], R[3] * v.x + R[4] * v.y + R[5] * v.z + t[1],
          R[6] * v.x + R[7] * v.y + R[8] * v.z + t[2]};
}

// Pose after a step dt with velocity (v, omega): centre c + dt v, orientation
// turned by the rotation vector dt omega in the world frame (left
// multiplication), renormalised.
MRDEM_HD void move_pose(const double* pose0, const double* vel, double dt, double* out) {
  for (int k = 0; k < 3; ++k) out[k] = pose0[k] + dt * vel[k];
  const double r[3] = {dt * vel[3], dt * vel[4], dt * vel[5]};
  double dq[4], q0[4], q[4];
  rotvec_to_quat(r, dq);
  const double n0 = sqrt(pose0[3] * pose0[3] + pose0[4] * pose0[4] + pose0[5] * pose0[5] +
                         pose0[6] * pose0[6]);
  for (int k = 0; k < 4; ++k) q0[k] = pose0[3 + k] / n0;
  quat_mul(dq, q0, q);
  const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) out[3 + k] = q[k] / n;
}

// Gradient of E(exp(w) R, t + v) in the twist (v, w) from the gradient g in
// a left rotation increment at the moved pose: the translation part is g's,
// the rotation part J_l(w)^T g_rot, with J_l(w) = I + (1 - cos th)/th^2 [w]x
// + (th - sin th)/th^3 [w]x^2 (th = |w|) the left Jacobian of the rotation
// group's exponential map: exp(w + e) = exp(J_l(w) e) exp(w) to first order.
MRDEM_HD void twist_gradient(const double* tw, const double* g, double* out) {
  for (int k = 0; k < 3; ++k) out[k] = g[k];
  const double w[3] = {tw[3], tw[4], tw[5]};
  const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;  // (1 - cos th)/th^2 and (th - sin th)/th^3
  if (th2 < 1e-8) {
    a = 0.5 - th2 / 24.0;
    b = 1.0 / 6.0 - th2 / 120.0;
  } else {
    const double th = sqrt(th2);
    a = (1.0 - cos(th)) / th2;
    b = (th - sin(th)) / (th2 * th);
  }
  // J^T g = g - a (w x g) + b (w x (w x g))   ([w]x^T = -[w]x, ([w]x^2)^T = [w]x^2)
  const double* gr = g + 3;
  const double c1[3] = {w[1] * gr[2] - w[2] * gr[1], w[2] * gr[0] - w[0] * gr[2],
                        w[0] * gr[1] - w[1] * gr[0]};
  const double c2[3] = {w[1] * c1[2] - w[2] * c1[1], w[2] * c1[0] - w[0] * c1[2],
                        w[0] * c1[1] - w[1] * c1[0]};
  for (int k = 0; k < 3; ++k) out[3 + k] = gr[k] - a * c1[k] + b * c2[k];
}

// One Picard update of particle i's velocities: new = (v0 + dt (F / m + g),
// omega0 + dt tau / I) from the forces at the guessed geometry.  Returns
// max_k |new_k - guess_k| and max_k |new_k| through *change and *scale.
MRDEM_HD void picard_velocity(const double* vel0, const double* ft, double m, double inertia,
                              const double g[3], double dt, const double* guess, double* out,
                              double* change, double* scale) {
  double c = 0.0, s = 0.0;
  for (int k = 0; k < 6; ++k) {
    // no contraction into fused multiply-adds: the rounding is that of the
    // plain formula, operation by operation
    const double v = k < 3 ? bp_add(vel0[k], bp_mul(dt, bp_add(ft[k] / m, g[k])))
                           : bp_add(vel0[k], bp_mul(dt, ft[k]) / inertia);
    const double d = fabs(v - guess[k]), a = fabs(v);
    c = d > c ? d : c;
    s = a > s ? a : s;
    if (d != d) c = d;  // NaN propagates
    if (a != a) s = a;
    out[k] = v;
  }
  *change = c;
  *scale = s;
}

}  // namespace mrdem

namespace mrdem {

// ---- contact Hessian for Newton's method on the implicit Euler equations
//
// Second derivatives of one contact's energy e(d) (Sec. 2 force law,
// e = K_s sqrt(mu) eps (1 - d/(2 eps))^2) in the two particles' pose twists
// (world translation; world rotation increment about the particle origin t,
// on the left of R), with the closest points free to move.  Let the closest
// points be pa = sum_v s_v X_v on A's active feature and pb on B's (active =
// barycentric weight above kActiveTol: a vertex, an edge or the face), r =
// pa - pb = d u, rho_A = pa - t_A, rho_B = -(pb - t_B), and
//   Z = [I; [rho_A]x; -I; [rho_B]x]   (12 x 3),
// the twist Jacobian of a point moving rigidly with A minus one moving with
// B.  The free barycentric parameters q of the active features (at most two
// for a contact between non-parallel features) have directions G_q (an edge
// of A's feature, or minus an edge of B's), and
//   N_q = Z G_q + (G_q x r in the rotation rows of the particle owning q).
// Eliminating q by the implicit function theorem (the closest points are
// optimal) gives
//   H = Z [(e'' - e'/d) u u^T + (e'/d) I] Z^T - (e'/d) N (G G^T)^-1 N^T + R,
// R the second-order term of the exponential map in each rotation block,
// sym(g rho^T) - (g . rho) I with g = e' u.  For a vertex against a vertex
// (no q) the translation block is e'' u u^T + e' (I - u u^T)/d.
constexpr double kActiveTol = 1e-9;

// A contact's Hessian block in compact form: the block's entries follow from
// these (hessian_entry).  Rows of Z: z_i with (Z x)_i = z_i . x.
struct HessRep {
  double u[3], r[3];   // unit separation direction and r = pa - pb = d u
  double rA[3], rB[3]; // rho_A = pa - t_A, rho_B = -(pb - t_B)
  double G[2][3];      // directions of the free barycentric parameters
  double K[3];         // (G G^T)^-1: K00, K01, K11
  double a, b;         // e'' - e'/d and e'/d
  double g[3];         // e' u
  double zu[9];        // Z u in the reduced rows (see hess_map)
  double N[2][9];      // N_q in the reduced rows (zero beyond nq)
  int nq;              // free parameters (0..2)
  int own[2];          // particle of each (0: A, 1: B)
};

// The twelve pose rows (A's translation, A's rotation, B's translation, B's
// rotation) and the nine reduced rows (translation, A's rotation, B's
// rotation): B's translation row c is minus A's translation row c in every
// term of the block (Z, Z u, N_q), and the rotation correction sits in the
// rotation blocks only, so block(i, j) = s_i s_j H9(m_i, m_j).
MRDEM_HD void hess_map(int i, int* m, double* s) {
  const int blk = i / 3, c = i % 3;
  *m = (blk == 2 ? 0 : (blk == 3 ? 2 : blk)) * 3 + c;
  *s = blk == 2 ? -1.0 : 1.0;
}

// Reduced row z_p of Z: e_c for the translation, the rows of the
// cross-product matrices [rho_A]x and [rho_B]x for the rotations.
MRDEM_HD void hess_zrow9(const HessRep& h, int p, double z[3]) {
  const int blk = p / 3, c = p % 3;
  if (blk == 0) {
    z[0] = c == 0 ? 1.0 : 0.0;
    z[1] = c == 1 ? 1.0 : 0.0;
    z[2] = c == 2 ? 1.0 : 0.0;
    return;
  }
  const double* q = blk == 1 ? h.rA : h.rB;
  // row c of the cross-product matrix [q]x: (q x v)_c = z . v
  if (c == 0) { z[0] = 0.0; z[1] = -q[2]; z[2] = q[1]; }
  else if (c == 1) { z[0] = q[2]; z[1] = 0.0; z[2] = -q[0]; }
  else { z[0] = -q[1]; z[1] = q[0]; z[2] = 0.0; }
}

// Entry (p, q) of the reduced block H9:
//   a (Zu)_p (Zu)_q + b (Z Z^T)_pq - b sum_kl N_k,p K_kl N_l,q
//   + in the rotation blocks sym(g rho^T) - (g . rho) I.
MRDEM_HD double hessian_entry9(const HessRep& h, int p, int q) {
  double zp[3], zq[3];
  hess_zrow9(h, p, zp);
  hess_zrow9(h, q, zq);
  double v = h.a * h.zu[p] * h.zu[q] + h.b * (zp[0] * zq[0] + zp[1] * zq[1] + zp[2] * zq[2]);
  if (h.nq > 0) {
    const double np0 = h.N[0][p], nq0 = h.N[0][q];
    if (h.nq == 1) {
      v -= h.b * np0 * h.K[0] * nq0;
    } else {
      const double np1 = h.N[1][p], nq1 = h.N[1][q];
      v -= h.b * (np0 * h.K[0] * nq0 + np0 * h.K[1] * nq1 + np1 * h.K[1] * nq0 +
                  np1 * h.K[2] * nq1);
    }
  }
  const int bp = p / 3, bq = q / 3;
  if (bp == bq && bp > 0) {
    const double* rho = bp == 1 ? h.rA : h.rB;
    const int ii = p % 3, jj = q % 3;
    v += 0.5 * (h.g[ii] * rho[jj] + h.g[jj] * rho[ii]);
    if (ii == jj) v -= h.g[0] * rho[0] + h.g[1] * rho[1] + h.g[2] * rho[2];
  }
  return v;
}

// Entry (i, j) of the 12x12 block, from the reduced one.
MRDEM_HD double hessian_entry(const HessRep& h, int i, int j) {
  int p, q;
  double si, sj;
  hess_map(i, &p, &si);
  hess_map(j, &q, &sj);
  return si * sj * hessian_entry9(h, p, q);
}

// Closest points of two world triangles for the contact Hessian, screened
// as the exact pass screens its candidates: the fifteen sub-tests in float
// on coordinates relative to A's first vertex with their error bound, then
// FP64 only for the sub-tests that may hold the minimum (the first smallest
// in the fixed sub-test order wins, as in tri_tri_distance); crossing or
// nearly touching triangles take the full FP64 test, and pairs certainly
// beyond tau come back with d > tau.
MRDEM_HD TriTriResult<double> tri_tri_screened(const V3<double> TA[3], const V3<double> TB[3],
                                               double tau) {
  const V3<double> o = TA[0];
  CandGeom g;
  V3<float> Pf[3], Qf[3];
  for (int k = 0; k < 3; ++k) {
    g.P[k] = TA[k] - o;
    g.Q[k] = TB[k] - o;
    Pf[k] = {(float)g.P[k].x, (float)g.P[k].y, (float)g.P[k].z};
    Qf[k] = {(float)g.Q[k].x, (float)g.Q[k].y, (float)g.Q[k].z};
  }
  g.o = o;
  g.tau = tau;
  unsigned mask = 0;
  const int st = cand_float_stage(Pf, Qf, tau, 0.f, &mask);
  if (st < 0) return tri_tri_distance<double>(TA, TB);
  TriTriResult<double> r;
  r.feature = -1;
  r.near_parallel = false;
  for (int k = 0; k < 3; ++k) r.wa[k] = r.wb[k] = 0.0;
  if (st == 0) {
    r.d = 2.0 * tau + 1.0;
    r.pa = r.pb = o;
    return r;
  }
  V3<double> pa = o, pb = o;
  r.d = cand_double_stage(g, mask, pa, pb, r.wa, r.wb);
  r.pa = pa + o;
  r.pb = pb + o;
  return r;
}

// The compact block of the contact between world triangles TA (on A) and TB
// (on B).  Returns 0 when the contact has a block, 1 when the triangles are
// more than 2 eps apart or cross (d = 0: not differentiable), 2 when the
// active features are parallel (more than two free parameters or a
// singular G G^T).
MRDEM_HD int contact_hessian_rep(const V3<double> TA[3], const V3<double> TB[3],
                                 const V3<double>& tA, const V3<double>& tB, double ks,
                                 double eps, HessRep* out) {
  typedef V3<double> D;
  const TriTriResult<double> t = tri_tri_screened(TA, TB, 2.0 * eps);
  if (!(t.d > 0.0) || t.d > 2.0 * eps) return 1;
  // active vertices of the two features (no array indexed by a variable, so
  // that everything stays in registers)
  const bool a0 = t.wa[0] > kActiveTol, a1 = t.wa[1] > kActiveTol, a2 = t.wa[2] > kActiveTol;
  const bool b0 = t.wb[0] > kActiveTol, b1 = t.wb[1] > kActiveTol, b2 = t.wb[2] > kActiveTol;
  const int na = (int)a0 + (int)a1 + (int)a2, nb = (int)b0 + (int)b1 + (int)b2;
  if (na == 0 || nb == 0) return 2;
  const int nq = (na - 1) + (nb - 1);
  if (nq > 2) return 2;
  const double sa = (a0 ? t.wa[0] : 0.0) + (a1 ? t.wa[1] : 0.0) + (a2 ? t.wa[2] : 0.0);
  const double sb = (b0 ? t.wb[0] : 0.0) + (b1 ? t.wb[1] : 0.0) + (b2 ? t.wb[2] : 0.0);
  D pa = {0.0, 0.0, 0.0}, pb = {0.0, 0.0, 0.0};
  if (a0) pa = pa + (t.wa[0] / sa) * TA[0];
  if (a1) pa = pa + (t.wa[1] / sa) * TA[1];
  if (a2) pa = pa + (t.wa[2] / sa) * TA[2];
  if (b0) pb = pb + (t.wb[0] / sb) * TB[0];
  if (b1) pb = pb + (t.wb[1] / sb) * TB[1];
  if (b2) pb = pb + (t.wb[2] / sb) * TB[2];
  const D r = pa - pb;
  const double d = sqrt(dot(r, r));
  if (!(d > 0.0)) return 1;
  const D u = (1.0 / d) * r;
  const double e1 = -ks * (1.0 - d / (2.0 * eps)), e2 = ks / (2.0 * eps);
  const D rA = pa - tA, rB = -1.0 * (pb - tB);
  // directions of the free parameters: edges from each feature's first
  // active vertex to its other active vertices (minus for B's), in order
  D G[2] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  int own[2] = {0, 0};
  int q = 0;
  auto push = [&](const D& g, int o) {
    if (q == 0) { G[0] = g; own[0] = o; }
    else { G[1] = g; own[1] = o; }
    ++q;
  };
  const D A0 = a0 ? TA[0] : (a1 ? TA[1] : TA[2]);
  if (a1 && a0) push(TA[1] - A0, 0);
  if (a2 && (a0 || a1)) push(TA[2] - A0, 0);
  const D B0 = b0 ? TB[0] : (b1 ? TB[1] : TB[2]);
  if (b1 && b0) push(-1.0 * (TB[1] - B0), 1);
  if (b2 && (b0 || b1)) push(-1.0 * (TB[2] - B0), 1);
  double K[3] = {0.0, 0.0, 0.0};
  if (nq == 1) {
    const double g11 = dot(G[0], G[0]);
    if (!(g11 > 0.0)) return 2;
    K[0] = 1.0 / g11;
  } else if (nq == 2) {
    const double g11 = dot(G[0], G[0]), g12 = dot(G[0], G[1]), g22 = dot(G[1], G[1]);
    const double det = g11 * g22 - g12 * g12;
    if (!(det > 1e-12 * g11 * g22)) return 2;
    K[0] = g22 / det;
    K[1] = -g12 / det;
    K[2] = g11 / det;
  }
  HessRep& h = *out;
  h.u[0] = u.x; h.u[1] = u.y; h.u[2] = u.z;
  h.r[0] = r.x; h.r[1] = r.y; h.r[2] = r.z;
  h.rA[0] = rA.x; h.rA[1] = rA.y; h.rA[2] = rA.z;
  h.rB[0] = rB.x; h.rB[1] = rB.y; h.rB[2] = rB.z;
  for (int k = 0; k < 2; ++k) {
    h.G[k][0] = G[k].x; h.G[k][1] = G[k].y; h.G[k][2] = G[k].z;
    h.own[k] = own[k];
  }
  for (int k = 0; k < 3; ++k) h.K[k] = K[k];
  h.a = e2 - e1 / d;
  h.b = e1 / d;
  h.g[0] = e1 * u.x; h.g[1] = e1 * u.y; h.g[2] = e1 * u.z;
  h.nq = nq;
  // Z u and N_q in the reduced rows, in closed form: Z x = (x, rho_A x x,
  // rho_B x x), and N_k = Z G_k plus G_k x r in the rotation rows of the
  // particle that owns parameter k
  const D zA = cross(rA, u), zB = cross(rB, u);
  h.zu[0] = u.x; h.zu[1] = u.y; h.zu[2] = u.z;
  h.zu[3] = zA.x; h.zu[4] = zA.y; h.zu[5] = zA.z;
  h.zu[6] = zB.x; h.zu[7] = zB.y; h.zu[8] = zB.z;
  for (int k = 0; k < 2; ++k) {
    const bool on = k < nq;
    const D gk = on ? G[k] : D{0.0, 0.0, 0.0};
    const D gr = cross(gk, r);
    const D nA = cross(rA, gk) + (own[k] == 0 ? gr : D{0.0, 0.0, 0.0});
    const D nB = cross(rB, gk) + (own[k] == 1 ? gr : D{0.0, 0.0, 0.0});
    double* N = h.N[k];
    N[0] = gk.x; N[1] = gk.y; N[2] = gk.z;
    N[3] = nA.x; N[4] = nA.y; N[5] = nA.z;
    N[6] = nB.x; N[7] = nB.y; N[8] = nB.z;
  }
  return 0;
}

// Adds the 12x12 block of the contact between world triangles TA (on A) and
// TB (on B) to out (row-major); the status of contact_hessian_rep.
MRDEM_HD int contact_hessian_block(const V3<double> TA[3], const V3<double> TB[3],
                                   const V3<double>& tA, const V3<double>& tB, double ks,
                                   double eps, double* out) {
  HessRep h;
  const int st = contact_hessian_rep(TA, TB, tA, tB, ks, eps, &h);
  if (st != 0) return st;
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) out[12 * i + j] += hessian_entry(h, i, j);
  return 0;
}

}  // namespace mrdem

namespace mrdem {

// Residual of the implicit Euler equations at velocities V (Newton's
// method): r = M (V - V0) / dt - (F, tau)(geometry moved by dt V) - (m g, 0),
// M = diag(m, m, m, I, I, I), rounded operation by operation in that order.
// Returns max_k |r_k| and max_k |M_k V_k| / dt (the scale of the
// convergence test) through *rmax and *smax.
MRDEM_HD void newton_residual(const double* vel0, const double* vel, const double* ft, double m,
                              double inertia, const double g[3], double dt, double* out,
                              double* rmax, double* smax) {
  double a = 0.0, s = 0.0;
  for (int k = 0; k < 6; ++k) {
    const double mk = k < 3 ? m : inertia;
    double r = bp_add(bp_mul(mk, vel[k] - vel0[k]) / dt, -ft[k]);
    if (k < 3) r = bp_add(r, -bp_mul(m, g[k]));
    const double sv = fabs(bp_mul(mk, vel[k])) / dt;
    out[k] = r;
    a = (fabs(r) > a || r != r) ? fabs(r) : a;
    s = (sv > s || sv != sv) ? sv : s;
  }
  *rmax = a;
  *smax = s;
}

// Largest displacement of a point of a particle between pose a and pose b
// (centre xyz, quaternion wxyz, any norm): |t_b - t_a| + theta R, theta the
// angle of the rotation q_b q_a^-1 and R the particle's bounding radius (a
// rotation by theta about the origin moves a point at distance r by
// 2 r sin(theta/2) <= theta r).
MRDEM_HD double particle_motion(const double* a, const double* b, double R) {
  const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
  const double na = sqrt(a[3] * a[3] + a[4] * a[4] + a[5] * a[5] + a[6] * a[6]);
  const double nb = sqrt(b[3] * b[3] + b[4] * b[4] + b[5] * b[5] + b[6] * b[6]);
  const double qa[4] = {a[3] / na, -a[4] / na, -a[5] / na, -a[6] / na};
  const double qb[4] = {b[3] / nb, b[4] / nb, b[5] / nb, b[6] / nb};
  double q[4];
  quat_mul(qb, qa, q);
  const double vn = sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double ang = 2.0 * atan2(vn, fabs(q[0]));
  return sqrt(dx * dx + dy * dy + dz * dz) + ang * R;
}

// 12x12 block times the 12-vector (x_A, x_B), row-major block.
MRDEM_HD void block_mul(const double* B, const double* xa, const double* xb, double* y) {
  for (int i = 0; i < 12; ++i) {
    double acc = 0.0;
    for (int j = 0; j < 6; ++j) acc += B[12 * i + j] * xa[j];
    for (int j = 0; j < 6; ++j) acc += B[12 * i + 6 + j] * xb[j];
    y[i] = acc;
  }
}

// A pair's share of (dt K) p: dt times its block applied to (p_A, p_B),
// split into A's six rows and B's six rows.
MRDEM_HD void cg_pair_apply(const double* B, const double* pa, const double* pb, double dt,
                            double ya[6], double yb[6]) {
  double y[12];
  block_mul(B, pa, pb, y);
  for (int k = 0; k < 6; ++k) {
    ya[k] = dt * y[k];
    yb[k] = dt * y[6 + k];
  }
}

// A pair's share of the diagonal of dt K: dt times the block's diagonal,
// A's six entries and B's six.
MRDEM_HD void cg_pair_diag(const double* B, double dt, double da[6], double db[6]) {
  for (int k = 0; k < 6; ++k) {
    da[k] = dt * B[13 * k];
    db[k] = dt * B[13 * (6 + k)];
  }
}

// Entry i (= 6 particle + component) of M / dt: mass for the three
// translations, the moment of inertia for the three rotations.
MRDEM_HD double cg_mdt(const double* mass, const double* inertia, double dt, int64_t i) {
  const int64_t part = i / 6;
  return (i % 6 < 3 ? mass[part] : inertia[part]) / dt;
}

// The preconditioner's entry: the matrix's diagonal, or M / dt where that
// is not positive.
MRDEM_HD double cg_precond(double diag, double mdt) { return diag > 0.0 ? diag : mdt; }

}  // namespace mrdem
