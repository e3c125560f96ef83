// mrdem_oracle.cpp -- plain FP64 CPU oracle for the multiresolution contact
// detection of Noble & Weinzierl, "A multiresolution Discrete Element Method
// for triangulated objects with implicit time stepping" (arXiv 2105.12415).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark may load this library.  The product (the CUDA
// library and its Python binding) never calls it and shares no code with it.
//
// What it computes is the plain definition of the result the method reaches
// faster (Lemma 1, Sec. 5.1: the hierarchical search yields exactly the
// result of the brute-force search over all fine triangle pairs):
//   * the distance between two triangles, by the comparison-based approach of
//     Sec. 3 ("Direct distance calculation"): six point-to-triangle distances,
//     nine edge-to-edge distances, plus the six edge-against-triangle
//     intersection tests that detect crossing triangles (distance 0);
//   * the contact set of a particle pair (Algorithm 2, findContacts): every
//     fine triangle pair whose eps-environments overlap, i.e. |n| <= eps with
//     n half the closest segment (Definition "Contact point", Eq. 2), which is
//     d <= 2 eps;
//   * the penalty force of each contact (Sec. 2, F(c)), summed per particle,
//     with torques about the centres of mass, and the contact energy
//     e(d) = K_s sqrt(mu) eps (1 - d/(2 eps))^2 whose negative derivative is
//     |F(c)|;
//   * the analytic gradient of that energy with respect to vertex positions
//     and 6-DoF poses, and the Gauss-Newton 12x12 blocks per particle pair;
//   * the paper's iterative penalty sweep (Eq. 3 functional, Eq. 4 modified
//     Newton, fixed iteration count of the hybrid scheme, Algorithm 4 top) in
//     FP64, for comparison with the FP32 sweep on the GPU (parity unpinned
//     beyond the properties the tests check: the sweep's constants are not
//     given by the paper);
//   * the conservativeness check of a surrogate (Definition "conservative",
//     Algorithm 7): the largest distance from any fine vertex under a node to
//     the node's surrogate triangle.
//
// Everything is double precision.  Particle vertices are passed as doubles
// (callers widen float32 body-frame coordinates exactly).  Poses are
// (tx, ty, tz, qw, qx, qy, qz); the quaternion is normalised before use and
// world = R(q) * body + t.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct V3 {
  double x, y, z;
};
inline V3 mk(const double* p) { return {p[0], p[1], p[2]}; }
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline void put(double* o, V3 a) { o[0] = a.x; o[1] = a.y; o[2] = a.z; }

// ---------------------------------------------------------------------------
// Closest point on a segment [a, b] to p (projection, clamped).
V3 closest_on_segment(V3 p, V3 a, V3 b) {
  V3 ab = b - a;
  double l2 = dot(ab, ab);
  if (l2 <= 0.0) return a;
  double t = dot(p - a, ab) / l2;
  t = std::min(1.0, std::max(0.0, t));
  return a + t * ab;
}

// Closest point on triangle (a, b, c) to p.  Project p onto the plane; if the
// projection lies inside (all three sub-area barycentrics >= 0) it is the
// answer, otherwise the answer is on the boundary: the nearest of the three
// edge projections.
V3 closest_on_triangle(V3 p, V3 a, V3 b, V3 c) {
  V3 n = cross(b - a, c - a);
  double nn = dot(n, n);
  if (nn > 0.0) {
    V3 pp = p - (dot(p - a, n) / nn) * n;
    double u = dot(cross(b - pp, c - pp), n) / nn;  // weight of a
    double v = dot(cross(c - pp, a - pp), n) / nn;  // weight of b
    double w = 1.0 - u - v;                         // weight of c
    if (u >= 0.0 && v >= 0.0 && w >= 0.0) return pp;
  }
  V3 best = closest_on_segment(p, a, b);
  double bd = dot(p - best, p - best);
  V3 q = closest_on_segment(p, b, c);
  double qd = dot(p - q, p - q);
  if (qd < bd) { best = q; bd = qd; }
  q = closest_on_segment(p, c, a);
  qd = dot(p - q, p - q);
  if (qd < bd) { best = q; bd = qd; }
  return best;
}

// Closest points between segments [p1, q1] and [p2, q2].  If the stationary
// point of the squared distance over (s, t) lies in [0,1]^2 it is the global
// minimum; otherwise the minimum of this convex function over the square is
// on its boundary, i.e. an endpoint of one segment against the other segment.
double segment_segment(V3 p1, V3 q1, V3 p2, V3 q2, V3* c1, V3* c2) {
  V3 d1 = q1 - p1, d2 = q2 - p2, r = p1 - p2;
  double a = dot(d1, d1), e = dot(d2, d2), b = dot(d1, d2);
  double c = dot(d1, r), f = dot(d2, r);
  double den = a * e - b * b;
  if (den > 1e-13 * a * e) {
    double s = (b * f - c * e) / den;
    double t = (a * f - b * c) / den;
    if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
      *c1 = p1 + s * d1;
      *c2 = p2 + t * d2;
      return norm(*c1 - *c2);
    }
  }
  double best = std::numeric_limits<double>::infinity();
  V3 cand[4][2] = {{p1, closest_on_segment(p1, p2, q2)},
                   {q1, closest_on_segment(q1, p2, q2)},
                   {closest_on_segment(p2, p1, q1), p2},
                   {closest_on_segment(q2, p1, q1), q2}};
  for (int k = 0; k < 4; ++k) {
    double d = norm(cand[k][0] - cand[k][1]);
    if (d < best) { best = d; *c1 = cand[k][0]; *c2 = cand[k][1]; }
  }
  return best;
}

// Does segment [p, q] cross triangle (a, b, c)?  Solve
// p + t (q - p) = a + u (b - a) + v (c - a) by Cramer's rule; a segment
// parallel to the plane is reported as not crossing (a coplanar overlap has
// distance 0 through the point/edge tests anyway).
bool segment_crosses_triangle(V3 p, V3 q, V3 a, V3 b, V3 c, V3* x) {
  V3 d = q - p, e1 = b - a, e2 = c - a, s = p - a;
  // columns: [-d, e1, e2] * (t, u, v) = s
  V3 m0 = -1.0 * d;
  double det = dot(m0, cross(e1, e2));
  if (det == 0.0) return false;
  double t = dot(s, cross(e1, e2)) / det;
  double u = dot(m0, cross(s, e2)) / det;
  double v = dot(m0, cross(e1, s)) / det;
  if (t < 0.0 || t > 1.0 || u < 0.0 || v < 0.0 || u + v > 1.0) return false;
  *x = p + t * d;
  return true;
}

// Triangle-triangle distance by comparisons (Sec. 3).  Feature codes:
//   100+i : edge i of P crosses Q (d = 0);  103+j : edge j of Q crosses P
//   k     : vertex k of P against triangle Q (k = 0..2)
//   3+k   : vertex k of Q against triangle P
//   6+3i+j: edge i of P against edge j of Q
// Edge i joins vertex i and vertex (i+1) mod 3.  Ties keep the first minimum.
double tri_tri(const V3 P[3], const V3 Q[3], V3* pa, V3* pb, int* feature) {
  V3 x;
  for (int i = 0; i < 3; ++i)
    if (segment_crosses_triangle(P[i], P[(i + 1) % 3], Q[0], Q[1], Q[2], &x)) {
      *pa = x; *pb = x; *feature = 100 + i; return 0.0;
    }
  for (int j = 0; j < 3; ++j)
    if (segment_crosses_triangle(Q[j], Q[(j + 1) % 3], P[0], P[1], P[2], &x)) {
      *pa = x; *pb = x; *feature = 103 + j; return 0.0;
    }
  double best = std::numeric_limits<double>::infinity();
  for (int k = 0; k < 3; ++k) {
    V3 q = closest_on_triangle(P[k], Q[0], Q[1], Q[2]);
    double d = norm(P[k] - q);
    if (d < best) { best = d; *pa = P[k]; *pb = q; *feature = k; }
  }
  for (int k = 0; k < 3; ++k) {
    V3 p = closest_on_triangle(Q[k], P[0], P[1], P[2]);
    double d = norm(p - Q[k]);
    if (d < best) { best = d; *pa = p; *pb = Q[k]; *feature = 3 + k; }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      V3 c1, c2;
      double d = segment_segment(P[i], P[(i + 1) % 3], Q[j], Q[(j + 1) % 3], &c1, &c2);
      if (d < best) { best = d; *pa = c1; *pb = c2; *feature = 6 + 3 * i + j; }
    }
  return best;
}

// Barycentric weights (w0, w1, w2) of a point x lying on triangle (a, b, c):
// least-squares solution of x - a = s (b - a) + t (c - a).
void barycentric(V3 x, V3 a, V3 b, V3 c, double w[3]) {
  V3 e1 = b - a, e2 = c - a, r = x - a;
  double g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
  double r1 = dot(r, e1), r2 = dot(r, e2);
  double det = g11 * g22 - g12 * g12;
  double s = (r1 * g22 - r2 * g12) / det;
  double t = (g11 * r2 - g12 * r1) / det;
  w[0] = 1.0 - s - t; w[1] = s; w[2] = t;
}

struct Pose {
  double R[3][3];
  V3 t;
};

Pose make_pose(const double* p) {
  double w = p[3], x = p[4], y = p[5], z = p[6];
  double n = std::sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  Pose o;
  o.R[0][0] = w * w + x * x - y * y - z * z;
  o.R[0][1] = 2.0 * (x * y - w * z);
  o.R[0][2] = 2.0 * (x * z + w * y);
  o.R[1][0] = 2.0 * (x * y + w * z);
  o.R[1][1] = w * w - x * x + y * y - z * z;
  o.R[1][2] = 2.0 * (y * z - w * x);
  o.R[2][0] = 2.0 * (x * z - w * y);
  o.R[2][1] = 2.0 * (y * z + w * x);
  o.R[2][2] = w * w - x * x - y * y + z * z;
  o.t = {p[0], p[1], p[2]};
  return o;
}
V3 apply(const Pose& P, V3 v) {
  return {P.R[0][0] * v.x + P.R[0][1] * v.y + P.R[0][2] * v.z + P.t.x,
          P.R[1][0] * v.x + P.R[1][1] * v.y + P.R[1][2] * v.z + P.t.y,
          P.R[2][0] * v.x + P.R[2][1] * v.y + P.R[2][2] * v.z + P.t.z};
}
V3 rotate_T(const Pose& P, V3 v) {  // R^T v
  return {P.R[0][0] * v.x + P.R[1][0] * v.y + P.R[2][0] * v.z,
          P.R[0][1] * v.x + P.R[1][1] * v.y + P.R[2][1] * v.z,
          P.R[0][2] * v.x + P.R[1][2] * v.y + P.R[2][2] * v.z};
}
V3 rotate(const Pose& P, V3 v) {
  return {P.R[0][0] * v.x + P.R[0][1] * v.y + P.R[0][2] * v.z,
          P.R[1][0] * v.x + P.R[1][1] * v.y + P.R[1][2] * v.z,
          P.R[2][0] * v.x + P.R[2][1] * v.y + P.R[2][2] * v.z};
}

struct Mesh {
  const int64_t* vert_off;
  const double* verts;
  const int64_t* tri_off;
  const int32_t* tris;
};

// World-frame vertices of triangle `t` (local index) of particle `i`.
void world_triangle(const Mesh& m, const Pose& P, int i, int64_t t, V3 out[3]) {
  const int32_t* tv = m.tris + 3 * (m.tri_off[i] + t);
  const double* vb = m.verts + 3 * m.vert_off[i];
  for (int k = 0; k < 3; ++k) out[k] = apply(P, mk(vb + 3 * tv[k]));
}

struct Contact {
  int32_t pair, ta, tb, feature;
  double d;
  V3 pa, pb;
};

int resolve_threads(int n) {
#ifdef _OPENMP
  return n > 0 ? n : omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// Brute force over all fine triangle pairs of one particle pair (Algorithm 2).
void detect_pair(const Mesh& m, const double* poses, int32_t pair_id, int32_t A, int32_t B,
                 double eps, std::vector<Contact>& out, int threads) {
  Pose PA = make_pose(poses + 7 * A), PB = make_pose(poses + 7 * B);
  int64_t na = m.tri_off[A + 1] - m.tri_off[A];
  int64_t nb = m.tri_off[B + 1] - m.tri_off[B];
  std::vector<V3> wb(3 * nb);
  for (int64_t j = 0; j < nb; ++j) world_triangle(m, PB, B, j, &wb[3 * j]);
  const double tau = 2.0 * eps;
  std::vector<std::vector<Contact>> local(threads);
#pragma omp parallel for num_threads(threads) schedule(dynamic, 4)
  for (int64_t i = 0; i < na; ++i) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    V3 P[3];
    world_triangle(m, PA, A, i, P);
    for (int64_t j = 0; j < nb; ++j) {
      V3 pa, pb;
      int f;
      double d = tri_tri(P, &wb[3 * j], &pa, &pb, &f);
      if (d <= tau) local[tid].push_back({pair_id, (int32_t)i, (int32_t)j, f, d, pa, pb});
    }
  }
  for (auto& v : local) out.insert(out.end(), v.begin(), v.end());
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Primitive entry points (arrays of n items, row-major).
void orc_point_triangle(int64_t n, const double* p, const double* T, double* q, double* d) {
  for (int64_t i = 0; i < n; ++i) {
    const double* t = T + 9 * i;
    V3 c = closest_on_triangle(mk(p + 3 * i), mk(t), mk(t + 3), mk(t + 6));
    if (q) put(q + 3 * i, c);
    d[i] = norm(mk(p + 3 * i) - c);
  }
}

void orc_segment_segment(int64_t n, const double* S1, const double* S2, double* c1, double* c2,
                         double* d) {
  for (int64_t i = 0; i < n; ++i) {
    const double* a = S1 + 6 * i;
    const double* b = S2 + 6 * i;
    V3 x, y;
    d[i] = segment_segment(mk(a), mk(a + 3), mk(b), mk(b + 3), &x, &y);
    if (c1) put(c1 + 3 * i, x);
    if (c2) put(c2 + 3 * i, y);
  }
}

void orc_tri_tri(int64_t n, const double* P, const double* Q, double* d, double* pa, double* pb,
                 int32_t* feature) {
  for (int64_t i = 0; i < n; ++i) {
    V3 p[3] = {mk(P + 9 * i), mk(P + 9 * i + 3), mk(P + 9 * i + 6)};
    V3 q[3] = {mk(Q + 9 * i), mk(Q + 9 * i + 3), mk(Q + 9 * i + 6)};
    V3 a, b;
    int f;
    d[i] = tri_tri(p, q, &a, &b, &f);
    if (pa) put(pa + 3 * i, a);
    if (pb) put(pb + 3 * i, b);
    if (feature) feature[i] = f;
  }
}

// World pose matrix (row-major 3x3) of a pose (t, q).
void orc_pose_matrix(const double* pose, double* R) {
  Pose P = make_pose(pose);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[3 * r + c] = P.R[r][c];
}

// ---------------------------------------------------------------------------
// Contact set of every listed particle pair (Algorithm 2 over all pairs).
// Output is sorted by (pair, ta, tb).  Triangle indices are local to their
// particle.  Points are in the world frame.  Returns the number of contacts;
// if it exceeds `cap`, nothing beyond `cap` is written (call again).
int64_t orc_detect(const int64_t* vert_off, const double* verts, const int64_t* tri_off,
                   const int32_t* tris, const double* poses, int64_t n_pairs,
                   const int32_t* pairs, const double* eps, int64_t cap, int32_t* o_pair,
                   int32_t* o_ta, int32_t* o_tb, double* o_d, double* o_pa, double* o_pb,
                   int32_t* o_feature, int n_threads) {
  Mesh m{vert_off, verts, tri_off, tris};
  int threads = resolve_threads(n_threads);
  std::vector<Contact> all;
  for (int64_t p = 0; p < n_pairs; ++p)
    detect_pair(m, poses, (int32_t)p, pairs[2 * p], pairs[2 * p + 1], eps[p], all, threads);
  std::sort(all.begin(), all.end(), [](const Contact& a, const Contact& b) {
    if (a.pair != b.pair) return a.pair < b.pair;
    if (a.ta != b.ta) return a.ta < b.ta;
    return a.tb < b.tb;
  });
  int64_t n = (int64_t)all.size();
  for (int64_t k = 0; k < n && k < cap; ++k) {
    const Contact& c = all[k];
    o_pair[k] = c.pair; o_ta[k] = c.ta; o_tb[k] = c.tb; o_d[k] = c.d;
    put(o_pa + 3 * k, c.pa); put(o_pb + 3 * k, c.pb);
    if (o_feature) o_feature[k] = c.feature;
  }
  return n;
}

// Distances of listed fine triangle pairs (particle A's triangle ta against
// particle B's triangle tb), with the world triangles and the exact distance
// of orc_detect: the same values orc_detect reports for a pair it lists.
void orc_tri_pairs(const int64_t* vert_off, const double* verts, const int64_t* tri_off,
                   const int32_t* tris, const double* poses, int64_t n, const int32_t* abt,
                   double* d, double* pa, double* pb, int32_t* feature, int n_threads) {
  Mesh m{vert_off, verts, tri_off, tris};
  int threads = resolve_threads(n_threads);
#pragma omp parallel for num_threads(threads) schedule(static)
  for (int64_t k = 0; k < n; ++k) {
    const int32_t* q = abt + 4 * k;  // A, ta, B, tb
    Pose PA = make_pose(poses + 7 * q[0]), PB = make_pose(poses + 7 * q[2]);
    V3 P[3], Q[3], a, b;
    world_triangle(m, PA, q[0], q[1], P);
    world_triangle(m, PB, q[2], q[3], Q);
    int f;
    d[k] = tri_tri(P, Q, &a, &b, &f);
    put(pa + 3 * k, a);
    put(pb + 3 * k, b);
    feature[k] = f;
  }
}

// ---------------------------------------------------------------------------
// Penalty forces (Sec. 2, F(c)) of a contact list (as returned by orc_detect).
// force_torque[6*i..]: world force (3) and torque about the world centre of
// mass (3) of particle i, accumulated (caller zeroes).  energy[0] accumulates
// sum_c K_s sqrt(mu) eps (1 - d/(2 eps))^2.  At d = 0 the direction is minus
// the outward unit normal of A's triangle.
void orc_forces(const int64_t* vert_off, const double* verts, const int64_t* tri_off,
                const int32_t* tris, const double* poses, const double* mass, const double* com,
                const int32_t* pairs, const double* eps, double k_s, int64_t n_contacts,
                const int32_t* c_pair, const int32_t* c_ta, const double* c_d,
                const double* c_pa, const double* c_pb, double* force_torque, double* energy) {
  Mesh m{vert_off, verts, tri_off, tris};
  for (int64_t k = 0; k < n_contacts; ++k) {
    int p = c_pair[k];
    int A = pairs[2 * p], B = pairs[2 * p + 1];
    double e = eps[p], d = c_d[k];
    double mu = 1.0 / (1.0 / mass[A] + 1.0 / mass[B]);
    double ks = k_s * std::sqrt(mu);
    V3 pa = mk(c_pa + 3 * k), pb = mk(c_pb + 3 * k);
    V3 u;
    if (d > 0.0) {
      u = (1.0 / d) * (pa - pb);
    } else {
      Pose PA = make_pose(poses + 7 * A);
      V3 T[3];
      world_triangle(m, PA, A, c_ta[k], T);
      V3 n = cross(T[1] - T[0], T[2] - T[0]);
      u = (-1.0 / norm(n)) * n;
    }
    double mag = ks * (1.0 - d / (2.0 * e));
    V3 F = mag * u;
    V3 xc = 0.5 * (pa + pb);
    Pose PA = make_pose(poses + 7 * A), PB = make_pose(poses + 7 * B);
    V3 cA = apply(PA, mk(com + 3 * A)), cB = apply(PB, mk(com + 3 * B));
    V3 tA = cross(xc - cA, F), tB = cross(xc - cB, -1.0 * F);
    double* fa = force_torque + 6 * A;
    double* fb = force_torque + 6 * B;
    fa[0] += F.x; fa[1] += F.y; fa[2] += F.z; fa[3] += tA.x; fa[4] += tA.y; fa[5] += tA.z;
    fb[0] -= F.x; fb[1] -= F.y; fb[2] -= F.z; fb[3] += tB.x; fb[4] += tB.y; fb[5] += tB.z;
    double s = 1.0 - d / (2.0 * e);
    energy[0] += ks * e * s * s;
  }
}

// Total contact energy of all pairs (brute-force contact set, then the sum of
// e(d)); the function whose finite differences pin the gradient.
double orc_energy(const int64_t* vert_off, const double* verts, const int64_t* tri_off,
                  const int32_t* tris, const double* poses, const double* mass, int64_t n_pairs,
                  const int32_t* pairs, const double* eps, double k_s, int n_threads) {
  Mesh m{vert_off, verts, tri_off, tris};
  int threads = resolve_threads(n_threads);
  double E = 0.0;
  for (int64_t p = 0; p < n_pairs; ++p) {
    std::vector<Contact> c;
    int A = pairs[2 * p], B = pairs[2 * p + 1];
    detect_pair(m, poses, (int32_t)p, A, B, eps[p], c, threads);
    double mu = 1.0 / (1.0 / mass[A] + 1.0 / mass[B]);
    double ks = k_s * std::sqrt(mu);
    // sum in a fixed order so the result does not depend on the thread count
    std::sort(c.begin(), c.end(), [](const Contact& a, const Contact& b) {
      return a.ta != b.ta ? a.ta < b.ta : a.tb < b.tb;
    });
    for (auto& x : c) {
      double s = 1.0 - x.d / (2.0 * eps[p]);
      E += ks * eps[p] * s * s;
    }
  }
  return E;
}

// Analytic gradient of the contact energy.  For a contact with d > 0 the
// closest points are optimal, so dd/d(vertex) is the barycentric weight of
// the closest point times +u (A's triangle) or -u (B's triangle), with
// u = (pa - pb)/d.  With g = e'(d) u, e'(d) = -K_s sqrt(mu) (1 - d/(2 eps)):
//   dE/dv (body frame) = R^T (w g) for A's vertices, R^T (-w g) for B's;
//   dE/dt_A = g, dE/dtheta_A = (pa - t_A) x g, and -g, (pb - t_B) x (-g)
//   for B, where theta is a world-frame rotation increment about t applied on
//   the left of R.
// jac[144 p + 12 r + c] accumulates e''(d) J J^T with
// J = [u, (pa - t_A) x u, -u, -(pb - t_B) x u], e'' = K_s sqrt(mu) / (2 eps):
// the Gauss-Newton block of the pair with frozen barycentrics.
// Every output is accumulated; any may be null.
void orc_grad(const int64_t* vert_off, const double* verts, const int64_t* tri_off,
              const int32_t* tris, const double* poses, const double* mass,
              const int32_t* pairs, const double* eps, double k_s, int64_t n_contacts,
              const int32_t* c_pair, const int32_t* c_ta, const int32_t* c_tb,
              double* dE_dverts, double* dE_dpose, double* jac) {
  Mesh m{vert_off, verts, tri_off, tris};
  for (int64_t k = 0; k < n_contacts; ++k) {
    int p = c_pair[k];
    int A = pairs[2 * p], B = pairs[2 * p + 1];
    Pose PA = make_pose(poses + 7 * A), PB = make_pose(poses + 7 * B);
    V3 TA[3], TB[3];
    world_triangle(m, PA, A, c_ta[k], TA);
    world_triangle(m, PB, B, c_tb[k], TB);
    V3 pa, pb;
    int f;
    double d = tri_tri(TA, TB, &pa, &pb, &f);
    double e = eps[p];
    if (d > 2.0 * e) continue;
    double mu = 1.0 / (1.0 / mass[A] + 1.0 / mass[B]);
    double ks = k_s * std::sqrt(mu);
    V3 u;
    if (d > 0.0) {
      u = (1.0 / d) * (pa - pb);
    } else {
      V3 n = cross(TA[1] - TA[0], TA[2] - TA[0]);
      u = (-1.0 / norm(n)) * n;
    }
    double de = -ks * (1.0 - d / (2.0 * e));
    V3 g = de * u;
    if (dE_dverts) {
      double wa[3], wb[3];
      barycentric(pa, TA[0], TA[1], TA[2], wa);
      barycentric(pb, TB[0], TB[1], TB[2], wb);
      const int32_t* va = tris + 3 * (tri_off[A] + c_ta[k]);
      const int32_t* vb = tris + 3 * (tri_off[B] + c_tb[k]);
      for (int i = 0; i < 3; ++i) {
        V3 ga = rotate_T(PA, wa[i] * g);
        V3 gb = rotate_T(PB, -wb[i] * g);
        double* oa = dE_dverts + 3 * (vert_off[A] + va[i]);
        double* ob = dE_dverts + 3 * (vert_off[B] + vb[i]);
        oa[0] += ga.x; oa[1] += ga.y; oa[2] += ga.z;
        ob[0] += gb.x; ob[1] += gb.y; ob[2] += gb.z;
      }
    }
    V3 ra = pa - PA.t, rb = pb - PB.t;
    if (dE_dpose) {
      V3 tq = cross(ra, g), tqb = cross(rb, -1.0 * g);
      double* oa = dE_dpose + 6 * A;
      double* ob = dE_dpose + 6 * B;
      oa[0] += g.x; oa[1] += g.y; oa[2] += g.z; oa[3] += tq.x; oa[4] += tq.y; oa[5] += tq.z;
      ob[0] -= g.x; ob[1] -= g.y; ob[2] -= g.z; ob[3] += tqb.x; ob[4] += tqb.y; ob[5] += tqb.z;
    }
    if (jac) {
      V3 c1 = cross(ra, u), c2 = cross(rb, u);
      double J[12] = {u.x, u.y, u.z, c1.x, c1.y, c1.z, -u.x, -u.y, -u.z, -c2.x, -c2.y, -c2.z};
      double h = ks / (2.0 * e);
      double* o = jac + 144 * (int64_t)p;
      for (int r = 0; r < 12; ++r)
        for (int c = 0; c < 12; ++c) o[12 * r + c] += h * J[r] * J[c];
    }
  }
}

// ---------------------------------------------------------------------------
// The iterative penalty sweep of Sec. 3 (Eq. 3 and Eq. 4), in FP64, for n
// triangle pairs.  Reading of the paper taken here:
//   * t1(a1, b1) = P0 + a1 (P1 - P0) + b1 (P2 - P0), likewise t2 on Q;
//     start at a1 = b1 = a2 = b2 = 0 (Algorithm 4);
//   * first half-step: x <- x - diag(H^ + a_reg I)^-1 grad J^,
//     J^ = 1/2 |t1 - t2|^2, all four unknowns from the same iterate;
//   * second half-step on the penalty J~ = a_iter sum over both triangles of
//     1/2 (max(0,-a)^2 + max(0,a-1)^2 + max(0,-b)^2 + max(0,b-1)^2
//     + max(0,a+b-1)^2), without the Dirac terms of its Hessian, so the
//     diagonal entry of a is a_iter times the number of violated constraints
//     that contain a;
//   * a_reg = rho_reg s and a_iter = rho_iter s with
//     s = (|P1-P0|^2 + |P2-P0|^2 + |Q1-Q0|^2 + |Q2-Q0|^2) / 4;
//   * exactly n_iter iterations; converged iff the contact point
//     x(c) = (t1 + t2)/2 moved by at most C eps in the last iteration (Sec. 6.3);
//   * the certificate of no contact: with u = (t1 - t2)/|t1 - t2| at the final
//     iterate, gap = min_k u.P_k - max_k u.Q_k is a lower bound of the distance.
// Outputs per pair: x[4], gap, converged flag, |t1 - t2| at the final iterate.
void orc_sweep(int64_t n, const double* P, const double* Q, int n_iter, double rho_reg,
               double rho_iter, double conv_c, const double* eps, double* x_out, double* gap,
               int32_t* converged, double* dist_iter) {
  for (int64_t i = 0; i < n; ++i) {
    V3 P0 = mk(P + 9 * i), P1 = mk(P + 9 * i + 3), P2 = mk(P + 9 * i + 6);
    V3 Q0 = mk(Q + 9 * i), Q1 = mk(Q + 9 * i + 3), Q2 = mk(Q + 9 * i + 6);
    V3 e1 = P1 - P0, e2 = P2 - P0, f1 = Q1 - Q0, f2 = Q2 - Q0;
    double h[4] = {dot(e1, e1), dot(e2, e2), dot(f1, f1), dot(f2, f2)};
    double s = 0.25 * (h[0] + h[1] + h[2] + h[3]);
    double a_reg = rho_reg * s, a_it = rho_iter * s;
    double x[4] = {0.0, 0.0, 0.0, 0.0};
    V3 xc_old{0, 0, 0}, xc{0, 0, 0};
    for (int it = 0; it < n_iter; ++it) {
      V3 t1 = P0 + x[0] * e1 + x[1] * e2;
      V3 t2 = Q0 + x[2] * f1 + x[3] * f2;
      xc_old = 0.5 * (t1 + t2);
      V3 r = t1 - t2;
      double g[4] = {dot(r, e1), dot(r, e2), -dot(r, f1), -dot(r, f2)};
      for (int k = 0; k < 4; ++k) x[k] -= g[k] / (h[k] + a_reg);
      for (int tri = 0; tri < 2; ++tri) {
        double a = x[2 * tri], b = x[2 * tri + 1];
        double lo_a = std::max(0.0, -a), hi_a = std::max(0.0, a - 1.0);
        double lo_b = std::max(0.0, -b), hi_b = std::max(0.0, b - 1.0);
        double sum = std::max(0.0, a + b - 1.0);
        double ga = a_it * (-lo_a + hi_a + sum);
        double gb = a_it * (-lo_b + hi_b + sum);
        double na = (a < 0.0) + (a > 1.0) + (a + b > 1.0);
        double nb = (b < 0.0) + (b > 1.0) + (a + b > 1.0);
        x[2 * tri] = a - ga / (a_it * na + a_reg);
        x[2 * tri + 1] = b - gb / (a_it * nb + a_reg);
      }
      t1 = P0 + x[0] * e1 + x[1] * e2;
      t2 = Q0 + x[2] * f1 + x[3] * f2;
      xc = 0.5 * (t1 + t2);
    }
    V3 t1 = P0 + x[0] * e1 + x[1] * e2;
    V3 t2 = Q0 + x[2] * f1 + x[3] * f2;
    V3 r = t1 - t2;
    double rn = norm(r);
    for (int k = 0; k < 4; ++k) x_out[4 * i + k] = x[k];
    dist_iter[i] = rn;
    converged[i] = norm(xc - xc_old) <= conv_c * eps[i];
    if (rn > 0.0) {
      V3 u = (1.0 / rn) * r;
      double mp = std::min(dot(u, P0), std::min(dot(u, P1), dot(u, P2)));
      double mq = std::max(dot(u, Q0), std::max(dot(u, Q1), dot(u, Q2)));
      gap[i] = mp - mq;
    } else {
      gap[i] = -std::numeric_limits<double>::infinity();
    }
  }
}

// ---------------------------------------------------------------------------
// Conservativeness of surrogates (Definition "conservative"; Algorithm 7
// assigns each surrogate the smallest eps that makes it conservative).  For
// each of n (vertex, surrogate triangle) entries returns the FP64 distance;
// the caller takes the maximum per node and compares with the node's stored
// slack.  Distance to a triangle is convex, so its maximum over a fine
// triangle is reached at a vertex: checking vertices suffices.
void orc_vertex_surrogate_distance(int64_t n, const double* v, const double* T, double* d) {
  orc_point_triangle(n, v, T, nullptr, d);
}

}  // extern "C"
