// Host build of the implicit step's device functions (mrdem_step.cuh) for the
// CPU tests: the broad phase driven through the same sequence of steps as its
// kernels (bounds, cells, bucket scan, scatter, count, scan, write and sort),
// the pose update, and the per-contact Hessian block.  Test infrastructure:
// the library itself runs these functions only in its CUDA kernels.
#include <cmath>
#include <vector>

#include "mrdem_step.cuh"

using namespace mrdem;

extern "C" long long hs_broad_phase(int n, const double* poses, const double* bound,
                                    const double* radius, double eps_rel, int* pairs,
                                    double* pair_eps, long long cap, unsigned shuffle) {
  // k_bp_bounds
  BroadGrid g;
  g.lo[0] = g.lo[1] = g.lo[2] = INFINITY;
  double rb = 0.0, rmin = INFINITY;
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) g.lo[k] = fmin(g.lo[k], poses[7 * i + k]);
    rb = fmax(rb, bound[i]);
    rmin = fmin(rmin, bound[i]);
  }
  g.r_max = rb;
  g.classes = bp_classes(rb, rmin);
  for (int k = 0; k < kMaxClasses; ++k) {
    g.h[k] = bp_cell_side(rb, k);
    g.inv_h[k] = 1.0 / g.h[k];
  }
  g.bad = 0;
  int log2_t = 6;
  while ((1LL << log2_t) < 2LL * n) ++log2_t;
  const long long t = 1LL << log2_t;
  std::vector<BroadCell> cell(n);
  std::vector<int32_t> order(n), class_order(n), bucket_end(t, 0), class_end(kMaxClasses, 0),
      cnt(n);
  BroadWork w{cell.data(), order.data(), bucket_end.data(), class_order.data(), class_end.data(),
              log2_t};
  const BroadIn in{poses, bound, radius, eps_rel, n};
  // k_bp_cells
  for (int i = 0; i < n; ++i) {
    cell[i] = bp_cell_of(in, g, i, log2_t);
    ++bucket_end[cell[i].b];
    ++class_end[cell[i].k];
  }
  // k_bp_scan (buckets, classes)
  long long run = 0;
  for (long long b = 0; b < t; ++b) {
    const int c = bucket_end[b];
    bucket_end[b] = (int32_t)run;
    run += c;
  }
  run = 0;
  for (int k = 0; k < kMaxClasses; ++k) {
    const int c = class_end[k];
    class_end[k] = (int32_t)run;
    run += c;
  }
  // k_bp_scatter: the kernel's atomics group a bucket's (and a class's)
  // particles in any order; scatter them in a shuffled order
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  unsigned s = shuffle;
  for (int i = n - 1; i > 0 && shuffle; --i) {
    s = s * 1103515245u + 12345u;
    const int j = (int)(s % (unsigned)(i + 1));
    const int tmp = idx[i];
    idx[i] = idx[j];
    idx[j] = tmp;
  }
  for (int q = 0; q < n; ++q) {
    const int i = idx[q];
    order[bucket_end[cell[i].b]++] = i;
    class_order[class_end[cell[i].k]++] = i;
  }
  // k_bp_count (a warp per particle: the 32 lanes' shares), k_bp_scan
  for (int i = 0; i < n; ++i) {
    int32_t c = 0;
    for (int l = 0; l < 32; ++l) c += bp_visit_lane(in, g, w, i, l, 32, [](int32_t, double) {});
    cnt[i] = c;
  }
  long long total = 0;
  for (int i = 0; i < n; ++i) {
    const int c = cnt[i];
    cnt[i] = (int32_t)total;
    total += c;
  }
  if (total > cap) return total;
  // k_bp_write
  for (int i = 0; i < n; ++i) {
    const long long o = cnt[i], m = (i + 1 < n ? cnt[i + 1] : total) - o;
    long long k = 0;
    // the lanes' candidates one lane after the other, then in order of j
    for (int l = 0; l < 32; ++l)
      bp_visit_lane(in, g, w, i, l, 32, [&](int32_t j, double e) {
        if (k < m) {
          pairs[2 * (o + k) + 1] = j;
          pair_eps[o + k] = e;
        }
        ++k;
      });
    for (long long a = o + 1; a < o + m; ++a) {
      const int j = pairs[2 * a + 1];
      const double e = pair_eps[a];
      long long b = a - 1;
      while (b >= o && pairs[2 * b + 1] > j) {
        pairs[2 * (b + 1) + 1] = pairs[2 * b + 1];
        pair_eps[b + 1] = pair_eps[b];
        --b;
      }
      pairs[2 * (b + 1) + 1] = j;
      pair_eps[b + 1] = e;
    }
    for (long long a = o; a < o + m; ++a) pairs[2 * a] = i;
  }
  return total;
}

extern "C" void hs_move_poses(int n, const double* poses0, const double* vel, double dt,
                              double* out) {
  for (int i = 0; i < n; ++i) move_pose(poses0 + 7 * i, vel + 6 * i, dt, out + 7 * i);
}

extern "C" int hs_contact_hessian(const double* A, const double* B, const double* tA,
                                  const double* tB, double ks, double eps, double* out) {
  V3<double> TA[3], TB[3];
  for (int k = 0; k < 3; ++k) {
    TA[k] = {A[3 * k], A[3 * k + 1], A[3 * k + 2]};
    TB[k] = {B[3 * k], B[3 * k + 1], B[3 * k + 2]};
  }
  return contact_hessian_block(TA, TB, V3<double>{tA[0], tA[1], tA[2]},
                               V3<double>{tB[0], tB[1], tB[2]}, ks, eps, out);
}

extern "C" void hs_picard(int n, const double* vel0, const double* ft, const double* mass,
                          const double* inertia, const double* g, double dt, double* vel,
                          double* norms) {
  norms[0] = norms[1] = 0.0;
  for (int i = 0; i < n; ++i) {
    double out[6], c, s;
    picard_velocity(vel0 + 6 * i, ft + 6 * i, mass[i], inertia[i], g, dt, vel + 6 * i, out, &c,
                    &s);
    for (int k = 0; k < 6; ++k) vel[6 * i + k] = out[k];
    norms[0] = c > norms[0] ? c : norms[0];
    norms[1] = s > norms[1] ? s : norms[1];
  }
}

extern "C" double hs_particle_motion(const double* a, const double* b, double R) {
  return particle_motion(a, b, R);
}

extern "C" void hs_newton_residual(int n, const double* vel0, const double* vel, const double* ft,
                                   const double* mass, const double* inertia, const double* g,
                                   double dt, double* res, double* norms) {
  norms[0] = norms[1] = 0.0;
  for (int i = 0; i < n; ++i) {
    double a, b;
    newton_residual(vel0 + 6 * i, vel + 6 * i, ft + 6 * i, mass[i], inertia[i], g, dt,
                    res + 6 * i, &a, &b);
    norms[0] = a > norms[0] ? a : norms[0];
    norms[1] = b > norms[1] ? b : norms[1];
  }
}

// (M/dt + dt K) p through the conjugate-gradient kernels' per-element
// functions, and their preconditioner diagonal
extern "C" void hs_cg_matvec(int n, long long n_pairs, const int* ab, const double* blocks,
                             const double* mass, const double* inertia, double dt,
                             const double* p, double* ap, double* diag) {
  for (long long i = 0; i < 6LL * n; ++i) {
    ap[i] = cg_mdt(mass, inertia, dt, i) * p[i];
    diag[i] = cg_mdt(mass, inertia, dt, i);
  }
  for (long long q = 0; q < n_pairs; ++q) {
    const int A = ab[2 * q], B = ab[2 * q + 1];
    double ya[6], yb[6], da[6], db[6];
    cg_pair_apply(blocks + 144 * q, p + 6 * A, p + 6 * B, dt, ya, yb);
    cg_pair_diag(blocks + 144 * q, dt, da, db);
    for (int k = 0; k < 6; ++k) {
      ap[6 * A + k] += ya[k];
      ap[6 * B + k] += yb[k];
      diag[6 * A + k] += da[k];
      diag[6 * B + k] += db[k];
    }
  }
}

// The conjugate-gradient sequence of the kernels (init, check, then per
// iteration A p, p.Ap, the step or the negative-curvature step, check,
// direction), serially; returns the iterations, *breakdown the flag.
extern "C" int hs_cg_solve(int n, long long n_pairs, const int* ab, const double* blocks,
                           const double* mass, const double* inertia, double dt,
                           const double* rhs, double* x, int max_iter, double rel_tol,
                           int* breakdown) {
  const long long m = 6LL * n;
  std::vector<double> r(rhs, rhs + m), z(m), p(m), ap(m), diag(m), zero(m, 0.0);
  hs_cg_matvec(n, n_pairs, ab, blocks, mass, inertia, dt, zero.data(), ap.data(), diag.data());
  double rz = 0.0, rr0 = 0.0;
  for (long long i = 0; i < m; ++i) {
    x[i] = 0.0;
    z[i] = r[i] / cg_precond(diag[i], cg_mdt(mass, inertia, dt, i));
    p[i] = z[i];
    rz += r[i] * z[i];
    rr0 += r[i] * r[i];
  }
  *breakdown = 0;
  if (rr0 <= rel_tol * rel_tol * rr0) return 0;
  for (int k = 0; k < max_iter; ++k) {
    hs_cg_matvec(n, n_pairs, ab, blocks, mass, inertia, dt, p.data(), ap.data(), diag.data());
    double pap = 0.0;
    for (long long i = 0; i < m; ++i) pap += p[i] * ap[i];
    if (!(pap > 0.0)) {
      if (k == 0 && pap < 0.0)
        for (long long i = 0; i < m; ++i) x[i] += rz / -pap * p[i];
      *breakdown = 1;
      return k;
    }
    const double alpha = rz / pap;
    double rz1 = 0.0, rr = 0.0;
    for (long long i = 0; i < m; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * ap[i];
      z[i] = r[i] / cg_precond(diag[i], cg_mdt(mass, inertia, dt, i));
      rz1 += r[i] * z[i];
      rr += r[i] * r[i];
    }
    if (rr <= rel_tol * rel_tol * rr0) return k + 1;
    const double beta = rz1 / rz;
    for (long long i = 0; i < m; ++i) p[i] = z[i] + beta * p[i];
    rz = rz1;
  }
  return max_iter;
}

extern "C" void hs_pose_points(const double* pose, int n, const double* v, double* out) {
  double R[9];
  quat_matrix(pose + 3, R);
  for (int i = 0; i < n; ++i) {
    const V3<double> w = pose_point(R, pose, V3<double>{v[3 * i], v[3 * i + 1], v[3 * i + 2]});
    out[3 * i] = w.x;
    out[3 * i + 1] = w.y;
    out[3 * i + 2] = w.z;
  }
}
