// mrdem_geometry.cuh -- triangle-pair geometry of the collision detection.
//
// Two building blocks of Sec. 3 of Noble & Weinzierl (arXiv 2105.12415):
//   * the comparison-based distance ("Direct distance calculation"): six
//     point-to-triangle and nine edge-to-edge closest-point problems, plus the
//     six edge-against-triangle crossing tests that give distance 0 for
//     intersecting triangles; templated on float / double;
//   * the iterative penalty sweep (Eq. 3 functional, Eq. 4 alternating
//     modified Newton, fixed iteration count of the hybrid scheme of
//     Algorithm 4) in float, followed by a certificate: along the final
//     iterate's separation direction u, min_k u.P_k - max_k u.Q_k is a lower
//     bound of the distance, so a pair may be discarded only when that bound
//     exceeds the contact threshold.
// Used by the host hierarchy builder (point-triangle distance) and by every
// kernel.  Compiles as plain C++ when not under nvcc.
#pragma once

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define MRDEM_HD __host__ __device__ __forceinline__
#else
#define MRDEM_HD inline
#endif

namespace mrdem {

template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
MRDEM_HD V3<T> v3(T x, T y, T z) { return {x, y, z}; }
template <typename T>
MRDEM_HD V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
MRDEM_HD V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
MRDEM_HD V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T>
MRDEM_HD T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
MRDEM_HD V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T>
MRDEM_HD T clamp01(T v) { return v < T(0) ? T(0) : (v > T(1) ? T(1) : v); }
// Approximate reciprocal for the sweep (its accuracy only affects how well the
// pairs are pruned, never correctness).
#ifdef __CUDA_ARCH__
#define MRDEM_RCP(x) __fdividef(1.0f, (x))
#define MRDEM_DIV(a, b) __fdividef((a), (b))
#else
#define MRDEM_RCP(x) (1.0f / (x))
#define MRDEM_DIV(a, b) ((a) / (b))
#endif

template <typename T>
MRDEM_HD T my_sqrt(T v) { return sqrt(v); }
template <>
MRDEM_HD float my_sqrt<float>(float v) { return sqrtf(v); }

// Quotient a / b.  In double on the device: a float reciprocal of b refined by
// two Newton-Raphson steps r <- r (2 - b r) (each doubles the correct bits:
// ~23 -> 46 -> 92) and one residual correction of the quotient; about one ulp,
// far cheaper than the correctly rounded division, and exact enough for the
// final distances; divisors outside [1e-30, 1e30] take the ordinary division.
template <typename T>
MRDEM_HD T qdiv(T a, T b) { return a / b; }
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ double qdiv<double>(double a, double b) {
  if (!(fabs(b) > 1e-30 && fabs(b) < 1e30)) return a / b;  // outside the float seed's range
  double r = (double)__frcp_rn((float)b);
  r = fma(r, fma(-b, r, 1.0), r);
  r = fma(r, fma(-b, r, 1.0), r);
  double q = a * r;
  return fma(r, fma(-b, q, a), q);
}
#endif

// Result of a closest-point query between two triangles P and Q.
template <typename T>
struct TriTriResult {
  T d;            // distance
  V3<T> pa, pb;   // closest points on P and Q
  T wa[3], wb[3]; // barycentric weights of pa in P and pb in Q
  int feature;    // which sub-test produced the minimum (codes in mrdem.h)
  bool near_parallel;  // an edge-edge test that set the minimum was near-parallel
};

// Closest point of triangle (a, b, c) to p, classified by the Voronoi region
// of p (vertex, edge or face region), with its barycentric weights.
template <typename T>
MRDEM_HD V3<T> closest_on_triangle(V3<T> p, V3<T> a, V3<T> b, V3<T> c, T w[3]) {
  V3<T> ab = b - a, ac = c - a, ap = p - a;
  T d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= T(0) && d2 <= T(0)) { w[0] = 1; w[1] = 0; w[2] = 0; return a; }
  V3<T> bp = p - b;
  T d3 = dot(ab, bp), d4 = dot(ac, bp);
  if (d3 >= T(0) && d4 <= d3) { w[0] = 0; w[1] = 1; w[2] = 0; return b; }
  T vc = d1 * d4 - d3 * d2;
  if (vc <= T(0) && d1 >= T(0) && d3 <= T(0)) {
    T s = qdiv(d1, d1 - d3);
    w[0] = T(1) - s; w[1] = s; w[2] = 0;
    return a + s * ab;
  }
  V3<T> cp = p - c;
  T d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= T(0) && d5 <= d6) { w[0] = 0; w[1] = 0; w[2] = 1; return c; }
  T vb = d5 * d2 - d1 * d6;
  if (vb <= T(0) && d2 >= T(0) && d6 <= T(0)) {
    T s = qdiv(d2, d2 - d6);
    w[0] = T(1) - s; w[1] = 0; w[2] = s;
    return a + s * ac;
  }
  T va = d3 * d6 - d5 * d4;
  T e43 = d4 - d3, e56 = d5 - d6;
  if (va <= T(0) && e43 >= T(0) && e56 >= T(0)) {
    T s = qdiv(e43, e43 + e56);
    w[0] = 0; w[1] = T(1) - s; w[2] = s;
    return b + s * (c - b);
  }
  T inv = qdiv(T(1), va + vb + vc);
  T v = vb * inv, u = vc * inv;
  w[0] = T(1) - v - u; w[1] = v; w[2] = u;
  return a + v * ab + u * ac;
}

// The same closest point with the region chosen by the same tests in the same
// order but without branches: every quantity is formed, the first region
// whose test holds wins, and one quotient q = num / den gives the point
// a + v ab + w ac (vertex regions: (0,0), (1,0), (0,1); edge ab: (q,0); edge
// ac: (0,q); edge bc: (1-q,q); face: (vb q, vc q) with q = 1/(va+vb+vc)).
// Used where the lanes of a warp evaluate different points.
template <typename T>
MRDEM_HD V3<T> closest_on_triangle_flat(V3<T> p, V3<T> a, V3<T> b, V3<T> c) {
  V3<T> ab = b - a, ac = c - a, ap = p - a, bp = p - b, cp = p - c;
  T d1 = dot(ab, ap), d2 = dot(ac, ap), d3 = dot(ab, bp), d4 = dot(ac, bp);
  T d5 = dot(ab, cp), d6 = dot(ac, cp);
  T vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
  T e43 = d4 - d3, e56 = d5 - d6;
  const T zero(0), one(1);
  int region = 6;
  if (va <= zero && e43 >= zero && e56 >= zero) region = 5;
  if (vb <= zero && d2 >= zero && d6 <= zero) region = 4;
  if (d6 >= zero && d5 <= d6) region = 3;
  if (vc <= zero && d1 >= zero && d3 <= zero) region = 2;
  if (d3 >= zero && d4 <= d3) region = 1;
  if (d1 <= zero && d2 <= zero) region = 0;
  T num = region == 2 ? d1 : (region == 4 ? d2 : (region == 5 ? e43 : (region == 6 ? one : zero)));
  T den = region == 2 ? d1 - d3
        : (region == 4 ? d2 - d6 : (region == 5 ? e43 + e56 : (region == 6 ? va + vb + vc : one)));
  T q = qdiv(num, den);
  T v = region == 1 ? one : (region == 2 ? q : (region == 5 ? one - q : (region == 6 ? vb * q : zero)));
  T w = region == 3 ? one : (region == 4 || region == 5 ? q : (region == 6 ? vc * q : zero));
  return a + v * ab + w * ac;
}

// Closest points of segments [p1, q1] and [p2, q2]: minimise over s, then
// clamp t and re-solve s if t left [0, 1].  Returns the parameters.
// near_parallel is set when |d1 x d2|^2 <= 1e-6 |d1|^2 |d2|^2.
template <typename T>
MRDEM_HD void closest_segments(V3<T> p1, V3<T> q1, V3<T> p2, V3<T> q2, T* s_out, T* t_out,
                               bool* near_parallel) {
  V3<T> d1 = q1 - p1, d2 = q2 - p2, r = p1 - p2;
  T a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  T c = dot(d1, r), b = dot(d1, d2);
  T den = a * e - b * b;
  *near_parallel = den <= T(1e-6) * a * e;
  T s = den > T(0) ? clamp01(qdiv(b * f - c * e, den)) : T(0);
  T t = qdiv(b * s + f, e);
  if (t < T(0)) {
    t = T(0);
    s = clamp01(qdiv(-c, a));
  } else if (t > T(1)) {
    t = T(1);
    s = clamp01(qdiv(b - c, a));
  }
  *s_out = s;
  *t_out = t;
}

// Does segment [p, q] cross the triangle (a, b, c)?  Signed plane distances
// of the endpoints, then an inside test of the crossing point by the three
// edge orientations.  x and the triangle's weights of x are returned.
template <typename T>
MRDEM_HD bool segment_crosses(V3<T> p, V3<T> q, V3<T> a, V3<T> b, V3<T> c, T* t_out, T w[3]) {
  V3<T> n = cross(b - a, c - a);
  T sp = dot(n, p - a), sq = dot(n, q - a);
  if ((sp > T(0) && sq > T(0)) || (sp < T(0) && sq < T(0)) || sp == sq) return false;
  T t = sp / (sp - sq);
  V3<T> x = p + t * (q - p);
  T c0 = dot(cross(c - b, x - b), n);  // weight of a (area opposite a)
  T c1 = dot(cross(a - c, x - c), n);  // weight of b
  T c2 = dot(cross(b - a, x - a), n);  // weight of c
  if (c0 < T(0) || c1 < T(0) || c2 < T(0)) return false;
  T inv = T(1) / (c0 + c1 + c2);
  w[0] = c0 * inv; w[1] = c1 * inv; w[2] = c2 * inv;
  *t_out = t;
  return true;
}

// Comparison-based triangle-triangle distance, fixed test order, first
// minimum kept: crossings of P's edges, crossings of Q's edges, P's vertices
// against Q, Q's vertices against P, then the nine edge pairs.
// With RANK, *second2 receives the squared distance of the best sub-test
// that did not win (a different feature), for near-tie detection.
template <typename T, bool RANK>
MRDEM_HD TriTriResult<T> tri_tri_distance_impl(const V3<T> P[3], const V3<T> Q[3], T* second2) {
  TriTriResult<T> r;
  r.near_parallel = false;
  T w[3], t;
  // the first crossing edge in the fixed order (P's edges, then Q's): its
  // number c, parameter t and the crossed triangle's weights w
  int c = -1;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int e = 0; e < 6; ++e) {
    if (c >= 0) break;
    const int i = e % 3, i1 = i == 2 ? 0 : i + 1;
    const bool hit = e < 3 ? segment_crosses(P[i], P[i1], Q[0], Q[1], Q[2], &t, w)
                           : segment_crosses(Q[i], Q[i1], P[0], P[1], P[2], &t, w);
    if (hit) c = e;
  }
  if (c >= 0) {
    const int i = c % 3, i1 = i == 2 ? 0 : i + 1;
    // weights of the crossing point on its edge: (1 - t) at vertex i, t at i1
    const T e0 = i == 0 ? T(1) - t : (i1 == 0 ? t : T(0));
    const T e1 = i == 1 ? T(1) - t : (i1 == 1 ? t : T(0));
    const T e2 = i == 2 ? T(1) - t : (i1 == 2 ? t : T(0));
    r.d = T(0);
    if (c < 3) {
      r.pa = pick3(P, i) + t * (pick3(P, i1) - pick3(P, i));
      r.pb = r.pa;
      r.wa[0] = e0; r.wa[1] = e1; r.wa[2] = e2;
      r.wb[0] = w[0]; r.wb[1] = w[1]; r.wb[2] = w[2];
    } else {
      r.pb = pick3(Q, i) + t * (pick3(Q, i1) - pick3(Q, i));
      r.pa = r.pb;
      r.wb[0] = e0; r.wb[1] = e1; r.wb[2] = e2;
      r.wa[0] = w[0]; r.wa[1] = w[1]; r.wa[2] = w[2];
    }
    r.feature = 100 + c;
    return r;
  }
  T best2 = T(INFINITY), sec2 = T(INFINITY);
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int k = 0; k < 3; ++k) {
    V3<T> q = closest_on_triangle(P[k], Q[0], Q[1], Q[2], w);
    V3<T> dv = P[k] - q;
    T d2 = dot(dv, dv);
    if (RANK && !(d2 < best2) && d2 < sec2) sec2 = d2;
    if (d2 < best2) {
      if (RANK) sec2 = best2;
      best2 = d2; r.pa = P[k]; r.pb = q; r.feature = k;
      r.wa[0] = r.wa[1] = r.wa[2] = T(0); r.wa[k] = T(1);
      r.wb[0] = w[0]; r.wb[1] = w[1]; r.wb[2] = w[2];
    }
  }
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int k = 0; k < 3; ++k) {
    V3<T> p = closest_on_triangle(Q[k], P[0], P[1], P[2], w);
    V3<T> dv = p - Q[k];
    T d2 = dot(dv, dv);
    if (RANK && !(d2 < best2) && d2 < sec2) sec2 = d2;
    if (d2 < best2) {
      if (RANK) sec2 = best2;
      best2 = d2; r.pa = p; r.pb = Q[k]; r.feature = 3 + k;
      r.wb[0] = r.wb[1] = r.wb[2] = T(0); r.wb[k] = T(1);
      r.wa[0] = w[0]; r.wa[1] = w[1]; r.wa[2] = w[2];
    }
  }
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int i = 0; i < 3; ++i) {
    int i1 = i == 2 ? 0 : i + 1;
  #ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int j = 0; j < 3; ++j) {
      int j1 = j == 2 ? 0 : j + 1;
      T s, u;
      bool par;
      closest_segments(P[i], P[i1], Q[j], Q[j1], &s, &u, &par);
      V3<T> c1 = P[i] + s * (P[i1] - P[i]);
      V3<T> c2 = Q[j] + u * (Q[j1] - Q[j]);
      V3<T> dv = c1 - c2;
      T d2 = dot(dv, dv);
      if (RANK && !(d2 < best2) && d2 < sec2) sec2 = d2;
      if (d2 < best2) {
        if (RANK) sec2 = best2;
        best2 = d2; r.pa = c1; r.pb = c2; r.feature = 6 + 3 * i + j;
        r.near_parallel = par;
        r.wa[0] = r.wa[1] = r.wa[2] = T(0); r.wa[i] = T(1) - s; r.wa[i1] = s;
        r.wb[0] = r.wb[1] = r.wb[2] = T(0); r.wb[j] = T(1) - u; r.wb[j1] = u;
      }
    }
  }
  r.d = my_sqrt(best2);
  if (RANK) *second2 = sec2;
  return r;
}

template <typename T>
MRDEM_HD TriTriResult<T> tri_tri_distance(const V3<T> P[3], const V3<T> Q[3]) {
  return tri_tri_distance_impl<T, false>(P, Q, nullptr);
}

// All fifteen sub-tests of the comparison-based distance without early exit:
// d2[k] is the squared distance of sub-test k (k = feature code 0..14).
// Returns whether an edge of one triangle crosses the other (the six
// edge-against-triangle tests).
template <typename T>
MRDEM_HD bool tri_tri_subtests(const V3<T> P[3], const V3<T> Q[3], T d2[15]) {
  T w[3], t;
  bool crossing = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int i1 = i == 2 ? 0 : i + 1;
    crossing |= segment_crosses(P[i], P[i1], Q[0], Q[1], Q[2], &t, w);
    crossing |= segment_crosses(Q[i], Q[i1], P[0], P[1], P[2], &t, w);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    V3<T> q = closest_on_triangle(P[k], Q[0], Q[1], Q[2], w);
    V3<T> p = closest_on_triangle(Q[k], P[0], P[1], P[2], w);
    d2[k] = dot(P[k] - q, P[k] - q);
    d2[3 + k] = dot(p - Q[k], p - Q[k]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int i1 = i == 2 ? 0 : i + 1;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      int j1 = j == 2 ? 0 : j + 1;
      T s, u;
      bool par;
      closest_segments(P[i], P[i1], Q[j], Q[j1], &s, &u, &par);
      V3<T> dv = (P[i] + s * (P[i1] - P[i])) - (Q[j] + u * (Q[j1] - Q[j]));
      d2[6 + 3 * i + j] = dot(dv, dv);
    }
  }
  return crossing;
}

template <typename T>
MRDEM_HD V3<T> pick3(const V3<T> T3[3], int k) {
  return k == 0 ? T3[0] : (k == 1 ? T3[1] : T3[2]);
}

// Closest points of one sub-test (feature code 0..14) of the
// comparison-based distance, with their barycentric weights in P and Q; the
// squared distance is returned.
template <typename T>
MRDEM_HD T eval_subtest(const V3<T> P[3], const V3<T> Q[3], int f, V3<T>* pa, V3<T>* pb,
                        T wa[3], T wb[3]) {
  T w[3];
  if (f < 3) {
    V3<T> v = pick3(P, f);
    *pa = v;
    *pb = closest_on_triangle(v, Q[0], Q[1], Q[2], w);
    wa[0] = f == 0; wa[1] = f == 1; wa[2] = f == 2;
    wb[0] = w[0]; wb[1] = w[1]; wb[2] = w[2];
  } else if (f < 6) {
    V3<T> v = pick3(Q, f - 3);
    *pa = closest_on_triangle(v, P[0], P[1], P[2], w);
    *pb = v;
    wa[0] = w[0]; wa[1] = w[1]; wa[2] = w[2];
    wb[0] = f == 3; wb[1] = f == 4; wb[2] = f == 5;
  } else {
    int i = (f - 6) / 3, j = (f - 6) - 3 * ((f - 6) / 3);
    int i1 = i == 2 ? 0 : i + 1, j1 = j == 2 ? 0 : j + 1;
    V3<T> a0 = pick3(P, i), a1 = pick3(P, i1), b0 = pick3(Q, j), b1 = pick3(Q, j1);
    T s, u;
    bool par;
    closest_segments(a0, a1, b0, b1, &s, &u, &par);
    *pa = a0 + s * (a1 - a0);
    *pb = b0 + u * (b1 - b0);
    wa[0] = (i == 0) * (T(1) - s) + (i1 == 0) * s;
    wa[1] = (i == 1) * (T(1) - s) + (i1 == 1) * s;
    wa[2] = (i == 2) * (T(1) - s) + (i1 == 2) * s;
    wb[0] = (j == 0) * (T(1) - u) + (j1 == 0) * u;
    wb[1] = (j == 1) * (T(1) - u) + (j1 == 1) * u;
    wb[2] = (j == 2) * (T(1) - u) + (j1 == 2) * u;
  }
  V3<T> dv = *pa - *pb;
  return dot(dv, dv);
}

// Candidate pair for the final distance: both triangles in double,
// relative to the origin o (A's first vertex), and the threshold 2 eps.
struct CandGeom {
  V3<double> P[3], Q[3], o;
  double tau;
};

// FP32 form of the final distance: the fifteen sub-tests in float on the
// rounded coordinates with the error bound err = 2^-15 max|coordinate|; a
// pair clearly beyond 2 eps is dropped; every sub-test within 2 err of the
// float minimum is finished in extended precision and the smallest value is
// the distance (the true minimiser is always among them).
// Float stage of the FP32 form: the fifteen sub-tests on float coordinates
// relative to A's first vertex.  extra_err bounds the error of those
// coordinates beyond their own rounding (e.g. a float rigid transform).
// Returns 0 (beyond 2 eps for sure), -1 (crossing or nearly touching: needs
// the full double test) or 1 (finish in double: the sub-tests whose bit is
// set in *mask are within 2 err of the float minimum and contain the true
// minimiser).
MRDEM_HD int cand_float_stage(const V3<float> Pf[3], const V3<float> Qf[3], double tau,
                              float extra_err, unsigned* mask) {
  float L = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    L = fmaxf(L, fmaxf(fmaxf(fabsf(Pf[k].x), fabsf(Pf[k].y)), fabsf(Pf[k].z)));
    L = fmaxf(L, fmaxf(fmaxf(fabsf(Qf[k].x), fabsf(Qf[k].y)), fabsf(Qf[k].z)));
  }
  float d2[15];
  bool crossing = tri_tri_subtests(Pf, Qf, d2);
  float best2 = d2[0];
#pragma unroll
  for (int k = 1; k < 15; ++k) best2 = fminf(best2, d2[k]);
  float err = ldexpf(L, -15) + extra_err;
  float d32 = sqrtf(best2);
  if (crossing || d32 <= 2.f * err) return -1;
  if ((double)d32 > tau + (double)err) return 0;
  float lim = d32 + 2.f * err;
  float lim2 = lim * lim;
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k < 15; ++k) m |= (d2[k] <= lim2 ? 1u : 0u) << k;
  *mask = m;
  return 1;
}

// Double stage: the smallest of the masked sub-tests, with closest points
// and barycentric weights.
MRDEM_HD double cand_double_stage(const CandGeom& g, unsigned mask, V3<double>& pa,
                                  V3<double>& pb, double* wa, double* wb) {
  double bd2 = 1e300;
  for (int k = 0; k < 15; ++k) {
    if (!((mask >> k) & 1u)) continue;
    V3<double> a, b;
    double xa[3], xb[3];
    double v = eval_subtest(g.P, g.Q, k, &a, &b, xa, xb);
    if (v < bd2) {
      bd2 = v;
      pa = a;
      pb = b;
      if (wa) { wa[0] = xa[0]; wa[1] = xa[1]; wa[2] = xa[2]; }
      if (wb) { wb[0] = xb[0]; wb[1] = xb[1]; wb[2] = xb[2]; }
    }
  }
  return sqrt(bd2);
}

// ---------------------------------------------------------------------------
// Penalty sweep (Sec. 3, Eq. 3/4).  Unknowns x = (a1, b1, a2, b2) with
// t1 = P0 + a1 (P1 - P0) + b1 (P2 - P0), t2 = Q0 + a2 (Q1 - Q0) + b2 (Q2 - Q0),
// J^ = |t1 - t2|^2 / 2.  One iteration:
//   (1) x_k -= dJ^/dx_k / (H^_kk + a_reg)          (all k from the same x)
//   (2) per triangle, with the quadratic one-sided penalty
//       a_iter/2 (max(0,-a)^2 + max(0,a-1)^2 + max(0,-b)^2 + max(0,b-1)^2
//       + max(0,a+b-1)^2) and its Hessian without Dirac terms:
//       a -= a_iter v_a / (a_iter n_a + a_reg), v_a the summed violations
//       containing a, n_a their number (0, 1 or 2).
// a_reg = rho_reg s, a_iter = rho_iter s, s the mean of the four squared edge
// lengths.  Start x = 0; n_iter iterations.
struct SweepConst {
  float rho_reg, rho_iter;
  int n_iter;
};

#ifdef __CUDA_ARCH__
#define MRDEM_SAT(x) __saturatef(x)
#else
#define MRDEM_SAT(x) fminf(fmaxf((x), 0.f), 1.f)
#endif

// One triangle's penalty half-step; c1 = a_it/(a_it + a_reg),
// c2 = a_it/(2 a_it + a_reg).  a - clamp(a, 0, 1) equals
// max(0, a-1) - max(0, -a), and it is non-zero exactly when a violates one of
// its box constraints.
MRDEM_HD void penalty_step(float& a, float& b, float c1, float c2) {
  float ea = a - MRDEM_SAT(a), eb = b - MRDEM_SAT(b);
  float ab1 = (a + b) - 1.f;
  float sm = fmaxf(ab1, 0.f);
  bool on = ab1 > 0.f;
  float ka = (on && ea != 0.f) ? c2 : c1;
  float kb = (on && eb != 0.f) ? c2 : c1;
  a = fmaf(-(ea + sm), ka, a);
  b = fmaf(-(eb + sm), kb, b);
}

// Sweep + certificate for P (vertices p0..p2) against Q.  Returns the lower
// bound gap (NaN when the final separation vector is zero: no bound).
// conv_tol2 = (C eps)^2; *converged tells whether the contact point
// (t1 + t2)/2 moved by at most C eps in the last iteration.  x_out (4 floats)
// receives the final unknowns when not null.  NIT > 0 fixes the iteration
// count at compile time (the loop unrolls); NIT = 0 takes sc.n_iter.
template <bool WANT_CONV, int NIT = 0>
MRDEM_HD float sweep_certificate(V3<float> p0, V3<float> p1, V3<float> p2, V3<float> q0,
                                 V3<float> q1, V3<float> q2, const SweepConst& sc,
                                 float conv_tol2, bool* converged, float* x_out) {
  V3<float> e1 = p1 - p0, e2 = p2 - p0, f1 = q1 - q0, f2 = q2 - q0, d0 = p0 - q0;
  float h1 = dot(e1, e1), h2 = dot(e2, e2), h3 = dot(f1, f1), h4 = dot(f2, f2);
  float s = 0.25f * ((h1 + h2) + (h3 + h4));
  float areg = sc.rho_reg * s, ait = sc.rho_iter * s;
  float i1 = MRDEM_RCP(h1 + areg), i2 = MRDEM_RCP(h2 + areg);
  float i3 = MRDEM_RCP(h3 + areg), i4 = MRDEM_RCP(h4 + areg);
  float c1 = MRDEM_DIV(ait, ait + areg), c2 = MRDEM_DIV(ait, fmaf(2.f, ait, areg));
  float a1 = 0.f, b1 = 0.f, a2 = 0.f, b2 = 0.f;
  float pa1 = 0.f, pb1 = 0.f, pa2 = 0.f, pb2 = 0.f;
  const int n_iter = NIT > 0 ? NIT : sc.n_iter;
  V3<float> r;
#pragma unroll
  for (int it = 0; it < n_iter; ++it) {
    if (WANT_CONV && it == n_iter - 1) { pa1 = a1; pb1 = b1; pa2 = a2; pb2 = b2; }
    if (it == 0) {
      r = d0;  // the start x = 0 of Algorithm 4
    } else {
      r.x = fmaf(-b2, f2.x, fmaf(-a2, f1.x, fmaf(b1, e2.x, fmaf(a1, e1.x, d0.x))));
      r.y = fmaf(-b2, f2.y, fmaf(-a2, f1.y, fmaf(b1, e2.y, fmaf(a1, e1.y, d0.y))));
      r.z = fmaf(-b2, f2.z, fmaf(-a2, f1.z, fmaf(b1, e2.z, fmaf(a1, e1.z, d0.z))));
    }
    float g1 = dot(r, e1), g2 = dot(r, e2), g3 = dot(r, f1), g4 = dot(r, f2);
    a1 = fmaf(-g1, i1, a1);
    b1 = fmaf(-g2, i2, b1);
    a2 = fmaf(g3, i3, a2);  // dJ^/da2 = -r.f1
    b2 = fmaf(g4, i4, b2);
    penalty_step(a1, b1, c1, c2);
    penalty_step(a2, b2, c1, c2);
  }
  r.x = fmaf(-b2, f2.x, fmaf(-a2, f1.x, fmaf(b1, e2.x, fmaf(a1, e1.x, d0.x))));
  r.y = fmaf(-b2, f2.y, fmaf(-a2, f1.y, fmaf(b1, e2.y, fmaf(a1, e1.y, d0.y))));
  r.z = fmaf(-b2, f2.z, fmaf(-a2, f1.z, fmaf(b1, e2.z, fmaf(a1, e1.z, d0.z))));
  if (WANT_CONV) {
    // displacement of (t1 + t2)/2 over the last iteration
    float da1 = a1 - pa1, db1 = b1 - pb1, da2 = a2 - pa2, db2 = b2 - pb2;
    float mx = fmaf(da1, e1.x, fmaf(db1, e2.x, fmaf(da2, f1.x, db2 * f2.x)));
    float my = fmaf(da1, e1.y, fmaf(db1, e2.y, fmaf(da2, f1.y, db2 * f2.y)));
    float mz = fmaf(da1, e1.z, fmaf(db1, e2.z, fmaf(da2, f1.z, db2 * f2.z)));
    *converged = 0.25f * dot(v3(mx, my, mz), v3(mx, my, mz)) <= conv_tol2;
  }
  if (x_out) { x_out[0] = a1; x_out[1] = b1; x_out[2] = a2; x_out[3] = b2; }
#ifdef __CUDA_ARCH__
  float inv = rsqrtf(dot(r, r));
#else
  float inv = 1.f / sqrtf(dot(r, r));
#endif
  // support gap along r, normalised once at the end
  float mp = fminf(dot(r, p0), fminf(dot(r, p1), dot(r, p2)));
  float mq = fmaxf(dot(r, q0), fmaxf(dot(r, q1), dot(r, q2)));
  return (mp - mq) * inv;
}

// Support gap of the two triangles along an axis n (any non-zero vector):
// max over both orientations of (min over one triangle - max over the other),
// divided by |n|.  Like the sweep's certificate it bounds the distance from
// below; along the face normals it is tight for nearly parallel triangles.
MRDEM_HD float axis_gap(V3<float> n, V3<float> p0, V3<float> p1, V3<float> p2, V3<float> q0,
                        V3<float> q1, V3<float> q2) {
  float a0 = dot(n, p0), a1 = dot(n, p1), a2 = dot(n, p2);
  float b0 = dot(n, q0), b1 = dot(n, q1), b2 = dot(n, q2);
  float amin = fminf(a0, fminf(a1, a2)), amax = fmaxf(a0, fmaxf(a1, a2));
  float bmin = fminf(b0, fminf(b1, b2)), bmax = fmaxf(b0, fmaxf(b1, b2));
#ifdef __CUDA_ARCH__
  float inv = rsqrtf(dot(n, n));
#else
  float inv = 1.f / sqrtf(dot(n, n));
#endif
  return fmaxf(amin - bmax, bmin - amax) * inv;
}

}  // namespace mrdem
