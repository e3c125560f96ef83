// mrdem_forces.cu -- penalty forces of a contact set and their adjoint.
//
// Force law of Sec. 2 of Noble & Weinzierl (arXiv 2105.12415): a contact with
// closest points pa (on A's triangle) and pb (on B's), distance d = |pa - pb|
// and |n| = d/2, pushes A along u = (pa - pb)/d with
//   |F| = K_s sqrt(mu) (1 - |n|/eps),  mu = 1/(1/M_A + 1/M_B),
// and B with -F (equal and opposite), applied at the contact point
// (pa + pb)/2.  The energy e(d) = K_s sqrt(mu) eps (1 - d/(2 eps))^2 has
// -e'(d) = |F|, so F = -dE/dt_A.  The adjoint recomputes each contact's
// closest points and barycentric weights in FP64 from the triangles (no state
// kept from the detection) and scatters
//   dE/dv = R^T (w e'(d) (+-u))  for the six vertices,
//   dE/dt = +-e'(d) u, dE/dtheta = (p - t) x (+-e'(d) u),
//   jac  += e''(d) J J^T, J = [u, (pa - t_A) x u, -u, -(pb - t_B) x u].
#include <cuda_runtime.h>

#include <algorithm>

#include "mrdem_geometry.cuh"
#include "mrdem_internal.h"

namespace mrdem {

using D3 = V3<double>;

// helpers (the same layout as the detection kernels use)
__device__ __forceinline__ V3<float> load_vertex(const HierDev& H, int slot, int c) {
  return {__ldg(H.tri + (3 * c + 0) * H.stride + slot), __ldg(H.tri + (3 * c + 1) * H.stride + slot),
          __ldg(H.tri + (3 * c + 2) * H.stride + slot)};
}
__device__ __forceinline__ V3<float> xf_point(const PairXf& X, V3<float> v) {
  return {fmaf(X.R[0], v.x, fmaf(X.R[1], v.y, fmaf(X.R[2], v.z, X.t[0]))),
          fmaf(X.R[3], v.x, fmaf(X.R[4], v.y, fmaf(X.R[5], v.z, X.t[1]))),
          fmaf(X.R[6], v.x, fmaf(X.R[7], v.y, fmaf(X.R[8], v.z, X.t[2])))};
}
__device__ __forceinline__ void load_pairxf(const PairXf* xf, int p, PairXf& X) {
  const float4* q = reinterpret_cast<const float4*>(xf + p);
  float4 a = __ldg(q), b = __ldg(q + 1), cc = __ldg(q + 2), d = __ldg(q + 3);
  X.R[0] = a.x; X.R[1] = a.y; X.R[2] = a.z; X.R[3] = a.w;
  X.R[4] = b.x; X.R[5] = b.y; X.R[6] = b.z; X.R[7] = b.w;
  X.R[8] = cc.x; X.t[0] = cc.y; X.t[1] = cc.z; X.t[2] = cc.w;
  X.tau = d.x; X.margin = d.y;
  X.A = __float_as_int(d.z); X.B = __float_as_int(d.w);
}
// Both triangles of a candidate in A's frame, relative to A's first vertex
// (double, from the double transform).
__device__ __forceinline__ void cand_geom64(const HierDev& H, const PairXf64& X, int sa, int sb,
                                            CandGeom& g) {
  D3 Pb[3], Qb[3];
  for (int q = 0; q < 3; ++q) {
    Pb[q] = {(double)H.tri[(3 * q) * H.stride + sa], (double)H.tri[(3 * q + 1) * H.stride + sa],
             (double)H.tri[(3 * q + 2) * H.stride + sa]};
    Qb[q] = {(double)H.tri[(3 * q) * H.stride + sb], (double)H.tri[(3 * q + 1) * H.stride + sb],
             (double)H.tri[(3 * q + 2) * H.stride + sb]};
  }
  g.o = Pb[0];
  for (int q = 0; q < 3; ++q) {
    g.P[q] = Pb[q] - g.o;
    D3 y = {X.R[0] * Qb[q].x + X.R[1] * Qb[q].y + X.R[2] * Qb[q].z + X.t[0],
            X.R[3] * Qb[q].x + X.R[4] * Qb[q].y + X.R[5] * Qb[q].z + X.t[1],
            X.R[6] * Qb[q].x + X.R[7] * Qb[q].y + X.R[8] * Qb[q].z + X.t[2]};
    g.Q[q] = y - g.o;
  }
  g.tau = 2.0 * X.eps;
}

namespace {

__device__ __forceinline__ void pose_matrix(const double* p, double R[9]) {
  double w = p[3], x = p[4], y = p[5], z = p[6];
  double s = 2.0 / (w * w + x * x + y * y + z * z);
  R[0] = 1.0 - s * (y * y + z * z); R[1] = s * (x * y - w * z);       R[2] = s * (x * z + w * y);
  R[3] = s * (x * y + w * z);       R[4] = 1.0 - s * (x * x + z * z); R[5] = s * (y * z - w * x);
  R[6] = s * (x * z - w * y);       R[7] = s * (y * z + w * x);       R[8] = 1.0 - s * (x * x + y * y);
}
__device__ __forceinline__ D3 mul(const double R[9], D3 v) {
  return {R[0] * v.x + R[1] * v.y + R[2] * v.z, R[3] * v.x + R[4] * v.y + R[5] * v.z,
          R[6] * v.x + R[7] * v.y + R[8] * v.z};
}
__device__ __forceinline__ D3 mul_t(const double R[9], D3 v) {
  return {R[0] * v.x + R[3] * v.y + R[6] * v.z, R[1] * v.x + R[4] * v.y + R[7] * v.z,
          R[2] * v.x + R[5] * v.y + R[8] * v.z};
}
__device__ __forceinline__ void world_tri(const HierDev& H, int slot, const double R[9],
                                          const double* t, D3 T[3]) {
  for (int c = 0; c < 3; ++c) {
    D3 v = {(double)H.tri[(3 * c) * H.stride + slot], (double)H.tri[(3 * c + 1) * H.stride + slot],
            (double)H.tri[(3 * c + 2) * H.stride + slot]};
    D3 w = mul(R, v);
    T[c] = {w.x + t[0], w.y + t[1], w.z + t[2]};
  }
}
__device__ __forceinline__ D3 unit_normal(const D3 T[3]) {
  D3 n = cross(T[1] - T[0], T[2] - T[0]);
  return (1.0 / sqrt(dot(n, n))) * n;
}
__device__ __forceinline__ void add3(double* o, D3 v) {
  atomicAdd(o, v.x);
  atomicAdd(o + 1, v.y);
  atomicAdd(o + 2, v.z);
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) k_forces(HierDev H, const int32_t* __restrict__ ab,
                                                const double* __restrict__ eps,
                                                const double* __restrict__ poses,
                                                mrdem_contacts c, const double* __restrict__ mass,
                                                const double* __restrict__ com, double k_s,
                                                double* ft, double* energy, int64_t n_pairs) {
  int64_t n = *c.count;
  if (n > c.capacity) n = c.capacity;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    double e_k = 0.0;
    int p = k < n ? c.pair[k] : -1;
    if (p >= 0 && p < n_pairs) {
      int A = ab[2 * p], B = ab[2 * p + 1];
      double e = eps[p], d = c.dist[k];
      double mu = 1.0 / (1.0 / mass[A] + 1.0 / mass[B]);
      double ks = k_s * sqrt(mu);
      D3 pa = {c.point_a[3 * k], c.point_a[3 * k + 1], c.point_a[3 * k + 2]};
      D3 pb = {c.point_b[3 * k], c.point_b[3 * k + 1], c.point_b[3 * k + 2]};
      double RA[9], RB[9];
      pose_matrix(poses + 7 * (int64_t)A, RA);
      pose_matrix(poses + 7 * (int64_t)B, RB);
      D3 u;
      if (d > 0.0) {
        u = (1.0 / d) * (pa - pb);
      } else {
        D3 T[3];
        int slot = H.tri_slot[H.tri_off[A] + c.tri_a[k]];
        world_tri(H, slot, RA, poses + 7 * (int64_t)A, T);
        u = -1.0 * unit_normal(T);
      }
      double s = 1.0 - d / (2.0 * e);
      D3 F = (ks * s) * u;
      e_k = ks * e * s * s;
      if (ft) {
        D3 xc = 0.5 * (pa + pb);
        D3 cA = mul(RA, {com[3 * A], com[3 * A + 1], com[3 * A + 2]});
        D3 cB = mul(RB, {com[3 * B], com[3 * B + 1], com[3 * B + 2]});
        cA = {cA.x + poses[7 * (int64_t)A], cA.y + poses[7 * (int64_t)A + 1], cA.z + poses[7 * (int64_t)A + 2]};
        cB = {cB.x + poses[7 * (int64_t)B], cB.y + poses[7 * (int64_t)B + 1], cB.z + poses[7 * (int64_t)B + 2]};
        add3(ft + 6 * (int64_t)A, F);
        add3(ft + 6 * (int64_t)A + 3, cross(xc - cA, F));
        add3(ft + 6 * (int64_t)B, -1.0 * F);
        add3(ft + 6 * (int64_t)B + 3, cross(xc - cB, -1.0 * F));
      }
    }
    if (energy) {
      double w = warp_sum(e_k);
      if ((threadIdx.x & 31) == 0 && w != 0.0) atomicAdd(energy, w);
    }
  }
}

// Adjoint: one thread per contact.  Closest points and barycentric weights
// are recomputed from the triangles in A's frame (per-pair transforms from the
// setup pass): float sub-tests select the minimising sub-test(s), which are
// finished in double (the detection's FP32 form); crossing or nearly touching
// pairs use the full double test.  Gauss-Newton blocks of contacts that share
// a pair within a warp are summed in shared memory before one set of atomics
// per pair.
constexpr int kGradThreads = 128;
__global__ void __launch_bounds__(kGradThreads) k_grad(HierDev H, const PairXf* __restrict__ xf,
                                                       const PairXf64* __restrict__ xf64,
                                                       const double* __restrict__ poses,
                                                       mrdem_contacts c,
                                                       const double* __restrict__ mass, double k_s,
                                                       double scale, float* dverts, double* dpose,
                                                       double* jac, int64_t n_pairs) {
  __shared__ double sJ[kGradThreads / 32][32][13];  // 12 Jacobian entries and the weight e''
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t n = *c.count;
  if (n > c.capacity) n = c.capacity;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    int p = k < n ? c.pair[k] : -1;
    bool ok = p >= 0 && p < n_pairs;
    double J[12], h = 0.0;
    if (ok) ok = xf64[p].valid != 0;
    if (ok) {
      const PairXf64& X64 = xf64[p];
      const int A = X64.A, B = X64.B;
      const double e = X64.eps;
      int sa = H.tri_slot[H.tri_off[A] + c.tri_a[k]];
      int sb = H.tri_slot[H.tri_off[B] + c.tri_b[k]];
      // float stage on float coordinates relative to A's first vertex
      PairXf X;
      load_pairxf(xf, p, X);
      V3<float> a0 = load_vertex(H, sa, 0), a1 = load_vertex(H, sa, 1), a2 = load_vertex(H, sa, 2);
      V3<float> Pf[3] = {{0.f, 0.f, 0.f}, a1 - a0, a2 - a0};
      V3<float> Qf[3] = {xf_point(X, load_vertex(H, sb, 0)) - a0, xf_point(X, load_vertex(H, sb, 1)) - a0,
                         xf_point(X, load_vertex(H, sb, 2)) - a0};
      unsigned mask = 0;
      int res = cand_float_stage(Pf, Qf, 1e300, X.margin, &mask);
      CandGeom g;
      cand_geom64(H, X64, sa, sb, g);
      double d, wa[3], wb[3];
      D3 pa, pb;
      if (res == 1) {
        d = cand_double_stage(g, mask, pa, pb, wa, wb);
      } else {
        TriTriResult<double> r = tri_tri_distance(g.P, g.Q);
        d = r.d; pa = r.pa; pb = r.pb;
        for (int q = 0; q < 3; ++q) { wa[q] = r.wa[q]; wb[q] = r.wb[q]; }
      }
      ok = d <= 2.0 * e;
      if (ok) {
        double mu = 1.0 / (1.0 / mass[A] + 1.0 / mass[B]);
        double ks = k_s * sqrt(mu);
        // direction in A's frame, then the world
        D3 uA;
        if (d > 0.0) {
          uA = (1.0 / d) * (pa - pb);
        } else {
          D3 nn = cross(g.P[1] - g.P[0], g.P[2] - g.P[0]);
          uA = (-1.0 / sqrt(dot(nn, nn))) * nn;
        }
        D3 paw = mul(X64.RA, pa + g.o), pbw = mul(X64.RA, pb + g.o);
        paw = {paw.x + X64.tA[0], paw.y + X64.tA[1], paw.z + X64.tA[2]};
        pbw = {pbw.x + X64.tA[0], pbw.y + X64.tA[1], pbw.z + X64.tA[2]};
        D3 u = mul(X64.RA, uA);
        double de = -ks * (1.0 - d / (2.0 * e)) * scale;
        D3 gv = de * u;
        if (dverts) {
          // A's body frame: R_A^T g = de uA; B's body frame: R_rel^T of that
          D3 gA = de * uA;
          D3 gB = mul_t(X64.R, gA);
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
          add3(dpose + 6 * (int64_t)A, gv);
          add3(dpose + 6 * (int64_t)A + 3, cross(ra, gv));
          add3(dpose + 6 * (int64_t)B, -1.0 * gv);
          add3(dpose + 6 * (int64_t)B + 3, cross(rb, -1.0 * gv));
        }
        D3 c1 = cross(ra, u), c2 = cross(rb, u);
        J[0] = u.x; J[1] = u.y; J[2] = u.z; J[3] = c1.x; J[4] = c1.y; J[5] = c1.z;
        J[6] = -u.x; J[7] = -u.y; J[8] = -u.z; J[9] = -c2.x; J[10] = -c2.y; J[11] = -c2.z;
        h = ks / (2.0 * e) * scale;
      }
    }
    if (jac) {
      // group the warp's contacts by pair; each group's 78 distinct block
      // entries are summed by the lanes in turn and added once
      for (int q = 0; q < 12; ++q) sJ[w][lane][q] = ok ? J[q] : 0.0;
      sJ[w][lane][12] = ok ? h : 0.0;
      __syncwarp();
      unsigned pending = __ballot_sync(0xffffffffu, ok);
      int mykey = ok ? p : -1;
      while (pending) {
        int leader = __ffs(pending) - 1;
        int key = __shfl_sync(0xffffffffu, mykey, leader);
        unsigned grp = __ballot_sync(0xffffffffu, ok && mykey == key);
        pending &= ~grp;
        for (int e2 = lane; e2 < 78; e2 += 32) {
          // e2 -> (r, q) with r <= q in the upper triangle of 12 x 12
          int r = 0, rem = e2;
          while (rem >= 12 - r) { rem -= 12 - r; ++r; }
          int q = r + rem;
          double acc = 0.0;
          unsigned gm = grp;
          while (gm) {
            int l = __ffs(gm) - 1;
            gm &= gm - 1;
            acc += sJ[w][l][12] * sJ[w][l][r] * sJ[w][l][q];
          }
          double* o = jac + 144 * (int64_t)key;
          atomicAdd(o + 12 * r + q, acc);
          if (q != r) atomicAdd(o + 12 * q + r, acc);
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace

int launch_forces(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                  const double* eps, const double* poses, const mrdem_contacts* con,
                  const double* mass, const double* com, double k_s, double* ft, double* energy,
                  cudaStream_t s) {
  if (!ft && !energy) return MRDEM_OK;
  ProfScope ps(c, K_FORCES, s);
  k_forces<<<c->n_sms * 8, 256, 0, s>>>(hier->dev, ab, eps, poses, *con, mass, com, k_s, ft,
                                         energy, n_pairs);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_grad(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                const double* eps, const double* poses, const mrdem_contacts* con,
                const double* mass, double k_s, double scale, float* dverts, double* dpose,
                double* jac, cudaStream_t s) {
  if (!dverts && !dpose && !jac) return MRDEM_OK;
  if (n_pairs == 0) return MRDEM_OK;
  // per-pair transforms of this call's poses (no root test)
  int st = setup_pairs(c, hier, n_pairs, ab, eps, poses, s);
  if (st != MRDEM_OK) return st;
  ProfScope ps(c, K_GRAD, s);
  k_grad<<<c->n_sms * 8, kGradThreads, 0, s>>>(hier->dev, c->xf, c->xf64, poses, *con, mass, k_s,
                                                scale, dverts, dpose, jac, n_pairs);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
