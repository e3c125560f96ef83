// mrdem_hierarchy.cpp -- host construction of the surrogate trees.
//
// Sec. 4 (Definitions "surrogate model", "conservative", "weakly connected",
// "surrogate tree"), Implementation remark 3, Algorithm 7 and Appendix A of
// Noble & Weinzierl (arXiv 2105.12415):
//   * top-down: a node holding more than leaf_max fine triangles is split into
//     clusters of roughly equal size by a balanced k-means of the triangle
//     centroids (fanout clusters, fewer when they would fall below leaf_min);
//     recursion until every leaf holds at most leaf_max triangles;
//   * every node holds one surrogate triangle fitted to the fine vertices below
//     it (a minimax fit: Appendix A minimises the largest distance between
//     surrogate and fine geometry, with a regulariser against degenerate
//     triangles; its constants are not given, so this builder minimises that
//     largest distance directly over a family of non-degenerate triangles);
//   * each surrogate gets the smallest slack delta that keeps it conservative:
//     the largest FP64 distance from a fine vertex below it to the stored
//     float32 triangle (distance to a triangle is convex, so its maximum over
//     a fine triangle is at a vertex), rounded up to float32;
//   * beyond the paper, every node also gets an oriented box around the fine
//     vertices below it (principal axes of their covariance; the box is
//     convex, so it holds the node's fine triangles too), a further
//     conservative bound that the detection tests after the node spheres.
// Layout: nodes of a particle in breadth-first order, children contiguous;
// fine triangles reordered so that each leaf owns a contiguous run of slots,
// padded to a multiple of 4 slots.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "mrdem_geometry.cuh"
#include "mrdem_internal.h"

namespace mrdem {
namespace {

using D3 = V3<double>;

inline double norm(D3 a) { return std::sqrt(dot(a, a)); }

// Eigen-decomposition of a symmetric 3x3 matrix (cyclic Jacobi rotations).
// Returns eigenvalues ascending in w and eigenvectors as columns of V.
void sym_eig3(double A[3][3], double w[3], double V[3][3]) {
  double a[3][3];
  std::memcpy(a, A, sizeof(a));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    if (off < 1e-30 * (a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2]) + 1e-300) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (std::fabs(a[p][q]) < 1e-300) continue;
        double theta = (a[q][q] - a[p][p]) / (2 * a[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        double c = 1 / std::sqrt(t * t + 1), s = t * c;
        for (int k = 0; k < 3; ++k) {
          double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  int idx[3] = {0, 1, 2};
  std::sort(idx, idx + 3, [&](int i, int j) { return a[i][i] < a[j][j]; });
  double Vs[3][3];
  for (int c = 0; c < 3; ++c) {
    w[c] = a[idx[c]][idx[c]];
    for (int r = 0; r < 3; ++r) Vs[r][c] = V[r][idx[c]];
  }
  std::memcpy(V, Vs, sizeof(Vs));
}

struct PCA {
  D3 mean, axis[3];  // axis[0] largest variance ... axis[2] smallest
};

PCA pca(const std::vector<D3>& pts) {
  PCA r;
  D3 m{0, 0, 0};
  for (auto& p : pts) m = m + p;
  m = (1.0 / pts.size()) * m;
  double C[3][3] = {{0}};
  for (auto& p : pts) {
    D3 d = p - m;
    double v[3] = {d.x, d.y, d.z};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) C[i][j] += v[i] * v[j];
  }
  double w[3], V[3][3];
  sym_eig3(C, w, V);
  r.mean = m;
  for (int k = 0; k < 3; ++k) r.axis[k] = {V[0][2 - k], V[1][2 - k], V[2][2 - k]};
  return r;
}

// ---------------------------------------------------------------------------
// Balanced k-means of triangle centroids (Algorithm 7 "split into sets of
// roughly the same size"; Appendix B: a tailored k-means keeps them compact).
// Seeds: recursive median splits along the principal axis; then Lloyd
// iterations whose assignment respects exact cluster sizes (points with the
// largest regret, second-best minus best distance, choose first).
void median_split(std::vector<int>& idx, int lo, int hi, int k0, int k1,
                  const std::vector<int>& sizes, const std::vector<D3>& c,
                  std::vector<int>& label) {
  if (k1 - k0 == 1) {
    for (int i = lo; i < hi; ++i) label[idx[i]] = k0;
    return;
  }
  int km = (k0 + k1) / 2;
  int nl = 0;
  for (int k = k0; k < km; ++k) nl += sizes[k];
  std::vector<D3> pts;
  pts.reserve(hi - lo);
  for (int i = lo; i < hi; ++i) pts.push_back(c[idx[i]]);
  PCA p = pca(pts);
  D3 ax = p.axis[0];
  std::nth_element(idx.begin() + lo, idx.begin() + lo + nl, idx.begin() + hi, [&](int a, int b) {
    double pa = dot(c[a], ax), pb = dot(c[b], ax);
    return pa != pb ? pa < pb : a < b;
  });
  median_split(idx, lo, lo + nl, k0, km, sizes, c, label);
  median_split(idx, lo + nl, hi, km, k1, sizes, c, label);
}

std::vector<std::vector<int32_t>> balanced_kmeans(const std::vector<int32_t>& tris,
                                                  const std::vector<D3>& cen_all, int k,
                                                  int iters) {
  int n = (int)tris.size();
  std::vector<D3> c(n);
  for (int i = 0; i < n; ++i) c[i] = cen_all[tris[i]];
  std::vector<int> sizes(k);
  for (int j = 0; j < k; ++j) sizes[j] = n / k + (j < n % k ? 1 : 0);
  std::vector<int> label(n), idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  median_split(idx, 0, n, 0, k, sizes, c, label);
  std::vector<D3> ctr(k);
  std::vector<double> dist((size_t)n * k);
  std::vector<double> regret(n);
  std::vector<int> order(n), cap(k);
  for (int it = 0; it <= iters; ++it) {
    std::vector<int> cnt(k, 0);
    for (int j = 0; j < k; ++j) ctr[j] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
      ctr[label[i]] = ctr[label[i]] + c[i];
      cnt[label[i]]++;
    }
    for (int j = 0; j < k; ++j) ctr[j] = (1.0 / std::max(1, cnt[j])) * ctr[j];
    if (it == iters) break;
    for (int i = 0; i < n; ++i) {
      double b1 = DBL_MAX, b2 = DBL_MAX;
      for (int j = 0; j < k; ++j) {
        D3 d = c[i] - ctr[j];
        double v = dot(d, d);
        dist[(size_t)i * k + j] = v;
        if (v < b1) { b2 = b1; b1 = v; } else if (v < b2) { b2 = v; }
      }
      regret[i] = b2 - b1;
    }
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      return regret[a] != regret[b] ? regret[a] > regret[b] : a < b;
    });
    cap = sizes;
    for (int i : order) {
      int best = -1;
      double bv = DBL_MAX;
      for (int j = 0; j < k; ++j)
        if (cap[j] > 0 && dist[(size_t)i * k + j] < bv) { bv = dist[(size_t)i * k + j]; best = j; }
      label[i] = best;
      cap[best]--;
    }
  }
  std::vector<std::vector<int32_t>> out(k);
  for (int i = 0; i < n; ++i) out[label[i]].push_back(tris[i]);
  return out;
}

// ---------------------------------------------------------------------------
// Surrogate triangle fit: minimise delta(t) = max_v dist(v, t) over the
// vertices v below the node (Appendix A's first term with a very high
// exponent is this maximum).  Candidates: in the principal plane, at the
// middle of the vertices' normal extent, the triangle with edge normals 120
// degrees apart that encloses the projected vertices (orientation with the
// smallest perimeter), scaled about its centroid by a set of factors (a tiny
// triangle is the best surrogate of a round cluster, a spanning one of a
// flat patch), then a coordinate descent on the nine coordinates.  Every
// candidate keeps a non-zero area (the role of Appendix A's area term).
double max_dist(const std::vector<D3>& V, const D3 T[3]) {
  double m = 0;
  double w[3];
  for (auto& v : V) {
    D3 q = closest_on_triangle(v, T[0], T[1], T[2], w);
    D3 d = v - q;
    m = std::max(m, dot(d, d));
  }
  return std::sqrt(m);
}

double tri_area(const D3 T[3]) { return 0.5 * norm(cross(T[1] - T[0], T[2] - T[0])); }

void fit_surrogate(const std::vector<D3>& Vall, D3 normal_hint, D3 out[3]) {
  // optimisation on a bounded subsample; the final delta uses all vertices
  std::vector<D3> V;
  const size_t kSample = 1536;
  if (Vall.size() > kSample) {
    V.reserve(kSample);
    double step = (double)Vall.size() / kSample;
    for (size_t i = 0; i < kSample; ++i) V.push_back(Vall[(size_t)(i * step)]);
  } else {
    V = Vall;
  }
  PCA p = pca(V);
  D3 e1 = p.axis[0], e2 = p.axis[1], n = p.axis[2];
  if (dot(n, normal_hint) < 0) { n = -1.0 * n; e2 = -1.0 * e2; }  // keep (e1, e2, n) right-handed
  double zmin = DBL_MAX, zmax = -DBL_MAX;
  std::vector<double> px(V.size()), py(V.size());
  for (size_t i = 0; i < V.size(); ++i) {
    D3 d = V[i] - p.mean;
    px[i] = dot(d, e1);
    py[i] = dot(d, e2);
    double z = dot(d, n);
    zmin = std::min(zmin, z);
    zmax = std::max(zmax, z);
  }
  double zmid = 0.5 * (zmin + zmax);
  const double kPi = 3.14159265358979323846;
  double best_cost = DBL_MAX, best_h[3] = {0, 0, 0}, best_th = 0;
  for (int s = 0; s < 24; ++s) {
    double th = (2 * kPi / 3) * s / 24.0;
    double h[3];
    for (int k = 0; k < 3; ++k) {
      double a = th + 2 * kPi * k / 3, cx = std::cos(a), cy = std::sin(a);
      double m = -DBL_MAX;
      for (size_t i = 0; i < V.size(); ++i) m = std::max(m, cx * px[i] + cy * py[i]);
      h[k] = m;
    }
    double cost = h[0] + h[1] + h[2];
    if (cost < best_cost) {
      best_cost = cost; best_th = th;
      std::memcpy(best_h, h, sizeof(h));
    }
  }
  // vertices: intersection of edge lines k and k+1 (n_k . x = h_k)
  D3 T0[3];
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    double a0 = best_th + 2 * kPi * k / 3, a1 = best_th + 2 * kPi * k1 / 3;
    double ax = std::cos(a0), ay = std::sin(a0), bx = std::cos(a1), by = std::sin(a1);
    double det = ax * by - ay * bx;
    double x = (best_h[k] * by - ay * best_h[k1]) / det;
    double y = (ax * best_h[k1] - best_h[k] * bx) / det;
    T0[k] = p.mean + x * e1 + y * e2 + zmid * n;
  }
  // orient counter-clockwise about n
  if (dot(cross(T0[1] - T0[0], T0[2] - T0[0]), n) < 0) std::swap(T0[1], T0[2]);
  D3 cen = (1.0 / 3.0) * (T0[0] + T0[1] + T0[2]);
  double area0 = tri_area(T0);
  const double scales[] = {1.0, 0.85, 0.7, 0.55, 0.4, 0.25, 0.12, 0.05, 0.02};
  D3 T[3];
  double best = DBL_MAX;
  for (double sc : scales) {
    D3 C[3];
    for (int k = 0; k < 3; ++k) C[k] = cen + sc * (T0[k] - cen);
    double m = max_dist(V, C);
    if (m < best) { best = m; std::memcpy(T, C, sizeof(C)); }
  }
  // coordinate descent
  double size = 0;
  for (int k = 0; k < 3; ++k) size = std::max(size, norm(T[k] - cen));
  double step = 0.1 * std::max(size, 1e-12);
  double min_area = 1e-4 * std::max(tri_area(T), 1e-6 * area0);
  int evals = 0;
  const int kMaxEvals = V.size() > 512 ? 36 : 90;
  for (int round = 0; round < 6 && evals < kMaxEvals; ++round) {
    bool improved = true;
    while (improved && evals < kMaxEvals) {
      improved = false;
      for (int c = 0; c < 9 && evals < kMaxEvals; ++c) {
        for (double sgn : {1.0, -1.0}) {
          D3 C[3];
          std::memcpy(C, T, sizeof(C));
          double* coord = &C[c / 3].x + (c % 3);
          *coord += sgn * step;
          if (tri_area(C) < min_area) continue;
          double m = max_dist(V, C);
          ++evals;
          if (m < best) {
            best = m;
            std::memcpy(T, C, sizeof(C));
            improved = true;
            break;
          }
        }
      }
    }
    step *= 0.5;
  }
  std::memcpy(out, T, sizeof(T));
}

float round_up_f32(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, FLT_MAX);
  return f;
}

// Eigenvectors of a symmetric 3x3 matrix by cyclic Jacobi rotations: each
// rotation zeroes one off-diagonal entry; the sweeps stop when the
// off-diagonal part is negligible.  Rows of U are the eigenvectors.
void sym3_eigenvectors(double A[3][3], double U[3][3]) {
  double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-30 * diag || off == 0.0) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        // the rotation angle that annihilates A[p][q]
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - sn * akq;
          A[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - sn * aqk;
          A[q][k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {  // V <- V J
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - sn * vkq;
          V[k][q] = sn * vkp + c * vkq;
        }
      }
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) U[r][k] = V[k][r];
}

// Oriented box around a node's fine vertices: the principal axes of their
// covariance, stored in float, the centre of their extents along those axes
// in float, and half extents that are the largest FP64 projections
// |u_k . (v - c)| of the vertices on the stored axes about the stored centre,
// rounded up: the stored box contains every vertex when evaluated in FP64.
// Layout: centre xyz, axes u0 u1 u2 (rows), half extents xyz, 0.
void fit_box(const std::vector<D3>& pts, float box[16]) {
  D3 m{0, 0, 0};
  for (const D3& p : pts) m = m + p;
  m = (1.0 / (double)pts.size()) * m;
  double C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (const D3& p : pts) {
    const double d[3] = {p.x - m.x, p.y - m.y, p.z - m.z};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) C[a][b] += d[a] * d[b];
  }
  double U[3][3];
  sym3_eigenvectors(C, U);
  // orthonormalise (Gram-Schmidt) and round the axes to float
  D3 u[3] = {{U[0][0], U[0][1], U[0][2]}, {U[1][0], U[1][1], U[1][2]}, {0, 0, 0}};
  u[0] = (1.0 / std::sqrt(dot(u[0], u[0]))) * u[0];
  u[1] = u[1] - dot(u[1], u[0]) * u[0];
  u[1] = (1.0 / std::sqrt(dot(u[1], u[1]))) * u[1];
  u[2] = cross(u[0], u[1]);
  D3 uf[3];
  for (int k = 0; k < 3; ++k) uf[k] = {(double)(float)u[k].x, (double)(float)u[k].y, (double)(float)u[k].z};
  double lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  for (const D3& p : pts)
    for (int k = 0; k < 3; ++k) {
      const double t = dot(uf[k], p - m);
      lo[k] = std::min(lo[k], t);
      hi[k] = std::max(hi[k], t);
    }
  D3 c = m;
  for (int k = 0; k < 3; ++k) c = c + (0.5 * (lo[k] + hi[k])) * uf[k];
  const D3 cf{(double)(float)c.x, (double)(float)c.y, (double)(float)c.z};
  double half[3] = {0, 0, 0};
  for (const D3& p : pts)
    for (int k = 0; k < 3; ++k) half[k] = std::max(half[k], std::fabs(dot(uf[k], p - cf)));
  box[0] = (float)cf.x; box[1] = (float)cf.y; box[2] = (float)cf.z;
  for (int k = 0; k < 3; ++k) {
    box[3 + 3 * k] = (float)uf[k].x;
    box[4 + 3 * k] = (float)uf[k].y;
    box[5 + 3 * k] = (float)uf[k].z;
    box[12 + k] = round_up_f32(half[k] * (1.0 + 1e-12));
  }
  box[15] = 0.f;
}

struct Node {
  std::vector<int32_t> tris;  // local triangle indices below the node
  int level = 1;
  std::vector<int> children;
  bool leaf = false;
  float tri[9];
  float delta = 0;
  float box[16];  // oriented box around the fine vertices below (fit_box)
};

// Build one particle's tree (nodes in breadth-first order).
int build_particle(const mrdem_params& prm, const float* V, int nv, const int32_t* T, int nt,
                   std::vector<Node>& nodes) {
  for (int i = 0; i < 3 * nt; ++i)
    if (T[i] < 0 || T[i] >= nv) return MRDEM_ERR_INVALID;
  std::vector<D3> vd(nv);
  for (int i = 0; i < nv; ++i) {
    vd[i] = {V[3 * i], V[3 * i + 1], V[3 * i + 2]};
    if (!std::isfinite(vd[i].x) || !std::isfinite(vd[i].y) || !std::isfinite(vd[i].z))
      return MRDEM_ERR_INVALID;
  }
  std::vector<D3> cen(nt), nrm(nt);
  for (int t = 0; t < nt; ++t) {
    D3 a = vd[T[3 * t]], b = vd[T[3 * t + 1]], c = vd[T[3 * t + 2]];
    cen[t] = (1.0 / 3.0) * (a + b + c);
    nrm[t] = cross(b - a, c - a);
    if (dot(nrm[t], nrm[t]) <= 0) return MRDEM_ERR_INVALID;  // degenerate triangle
  }
  nodes.clear();
  nodes.emplace_back();
  nodes[0].tris.resize(nt);
  std::iota(nodes[0].tris.begin(), nodes[0].tris.end(), 0);
  for (size_t q = 0; q < nodes.size(); ++q) {
    int n = (int)nodes[q].tris.size();
    if (n <= prm.leaf_max) {
      nodes[q].leaf = true;
      continue;
    }
    int k = prm.fanout;
    if (n / prm.fanout < prm.leaf_min)
      k = std::min(prm.fanout, std::max(2, (n + prm.leaf_max - 1) / prm.leaf_max));
    k = std::min(k, n);
    auto parts = balanced_kmeans(nodes[q].tris, cen, k, prm.kmeans_iters);
    int lvl = nodes[q].level;
    for (auto& part : parts) {
      if (part.empty()) continue;
      std::sort(part.begin(), part.end());
      Node c;
      c.tris = std::move(part);
      c.level = lvl + 1;
      nodes[q].children.push_back((int)nodes.size());
      nodes.push_back(std::move(c));
    }
  }
  std::vector<int> stamp(nv, -1);
  for (size_t q = 0; q < nodes.size(); ++q) {
    Node& nd = nodes[q];
    std::vector<D3> pts;
    D3 nh{0, 0, 0};
    for (int t : nd.tris) {
      nh = nh + nrm[t];
      for (int k = 0; k < 3; ++k) {
        int v = T[3 * t + k];
        if (stamp[v] != (int)q) { stamp[v] = (int)q; pts.push_back(vd[v]); }
      }
    }
    D3 S[3];
    fit_surrogate(pts, nh, S);
    D3 Sf[3];
    for (int k = 0; k < 3; ++k) {
      nd.tri[3 * k + 0] = (float)S[k].x;
      nd.tri[3 * k + 1] = (float)S[k].y;
      nd.tri[3 * k + 2] = (float)S[k].z;
      Sf[k] = {nd.tri[3 * k], nd.tri[3 * k + 1], nd.tri[3 * k + 2]};
    }
    if (dot(cross(Sf[1] - Sf[0], Sf[2] - Sf[0]), cross(Sf[1] - Sf[0], Sf[2] - Sf[0])) <= 0)
      return MRDEM_ERR_INVALID;
    // exact slack of the stored triangle over every vertex below the node
    nd.delta = round_up_f32(max_dist(pts, Sf) * (1.0 + 1e-12));
    fit_box(pts, nd.box);
  }
  return MRDEM_OK;
}

}  // namespace

int build_hierarchy_host(const mrdem_params& prm, int32_t n, const int64_t* vert_off,
                         const float* verts, const int64_t* tri_off, const int32_t* tris,
                         HierHost* out) {
  if (n <= 0 || !vert_off || !verts || !tri_off || !tris) return MRDEM_ERR_INVALID;
  if (prm.fanout < 2 || prm.fanout > 8 || prm.leaf_max < 1 || prm.leaf_max > 32 || prm.leaf_min < 1)
    return MRDEM_ERR_INVALID;
  if (vert_off[0] != 0 || tri_off[0] != 0) return MRDEM_ERR_INVALID;
  for (int i = 0; i < n; ++i)
    if (vert_off[i + 1] <= vert_off[i] || tri_off[i + 1] <= tri_off[i]) return MRDEM_ERR_INVALID;
  if (tri_off[n] >= (int64_t)1 << 31 || vert_off[n] >= (int64_t)1 << 31) return MRDEM_ERR_INVALID;
  std::vector<std::vector<Node>> trees(n);
  std::vector<int> err(n, 0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; ++i) {
    err[i] = build_particle(prm, verts + 3 * vert_off[i], (int)(vert_off[i + 1] - vert_off[i]),
                            tris + 3 * tri_off[i], (int)(tri_off[i + 1] - tri_off[i]), trees[i]);
  }
  for (int i = 0; i < n; ++i)
    if (err[i]) return err[i];
  HierHost& h = *out;
  h = HierHost();
  h.n_particles = n;
  h.n_tri = tri_off[n];
  h.n_verts = vert_off[n];
  h.tri_off.assign(tri_off, tri_off + n + 1);
  h.vert_off.assign(vert_off, vert_off + n + 1);
  // global node and slot offsets
  std::vector<int64_t> node_off(n + 1, 0), slot_off(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    node_off[i + 1] = node_off[i] + (int64_t)trees[i].size();
    int64_t slots = 0;
    for (auto& nd : trees[i])
      if (nd.leaf) slots += (nd.tris.size() + 3) / 4 * 4;
    slot_off[i + 1] = slot_off[i] + slots;
  }
  h.n_nodes = node_off[n];
  h.n_tri_pad = slot_off[n];
  if (h.n_nodes >= (int64_t)1 << 31 || h.n_tri_pad >= (int64_t)1 << 31) return MRDEM_ERR_INVALID;
  h.node_tri.resize(h.n_nodes * 9);
  h.node_delta.resize(h.n_nodes);
  h.node_box.resize(h.n_nodes * 16);
  h.node_child.resize(h.n_nodes * 2);
  h.node_level.resize(h.n_nodes);
  h.root.resize(n);
  h.slot_xyz.assign(h.n_tri_pad * 9, 0.f);
  h.slot_vid.assign(h.n_tri_pad * 3, -1);
  h.slot_tri.assign(h.n_tri_pad, -1);
  h.slot_particle.assign(h.n_tri_pad, -1);
  h.tri_slot.assign(h.n_tri, -1);
  h.bound_r.resize(n);
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    const float* V = verts + 3 * vert_off[i];
    const int32_t* T = tris + 3 * tri_off[i];
    double br = 0;
    for (int64_t v = 0; v < vert_off[i + 1] - vert_off[i]; ++v)
      br = std::max(br, std::sqrt((double)V[3 * v] * V[3 * v] + (double)V[3 * v + 1] * V[3 * v + 1] +
                                  (double)V[3 * v + 2] * V[3 * v + 2]));
    h.bound_r[i] = round_up_f32(br);
    int64_t slot = slot_off[i];
    int depth = 0;
    auto& nodes = trees[i];
    h.root[i] = (int32_t)node_off[i];
    for (size_t q = 0; q < nodes.size(); ++q) {
      int64_t g = node_off[i] + (int64_t)q;
      auto& nd = nodes[q];
      std::memcpy(&h.node_tri[g * 9], nd.tri, sizeof(nd.tri));
      h.node_delta[g] = nd.delta;
      std::memcpy(&h.node_box[g * 16], nd.box, sizeof(nd.box));
      h.node_level[g] = nd.level;
      depth = std::max(depth, nd.level);
      if (nd.leaf) {
        h.node_child[2 * g] = (int32_t)slot;
        h.node_child[2 * g + 1] = -(int32_t)nd.tris.size();
        for (int t : nd.tris) {
          for (int k = 0; k < 3; ++k) {
            int v = T[3 * t + k];
            h.slot_vid[slot * 3 + k] = (int32_t)(vert_off[i] + v);
            for (int c = 0; c < 3; ++c) h.slot_xyz[slot * 9 + 3 * k + c] = V[3 * v + c];
          }
          h.slot_tri[slot] = t;
          h.slot_particle[slot] = i;
          h.tri_slot[tri_off[i] + t] = (int32_t)slot;
          ++slot;
        }
        while ((slot - slot_off[i]) % 4) ++slot;
      } else {
        h.node_child[2 * g] = (int32_t)(node_off[i] + nd.children.front());
        h.node_child[2 * g + 1] = (int32_t)nd.children.size();
      }
    }
    trees[i].clear();
    trees[i].shrink_to_fit();
#pragma omp critical
    h.max_depth = std::max(h.max_depth, depth);
  }
  return MRDEM_OK;
}

}  // namespace mrdem
