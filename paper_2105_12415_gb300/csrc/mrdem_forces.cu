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

#include "mrdem_device.cuh"

namespace mrdem {


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
  // per-pair transforms of this call's poses (no root test), then the
  // closest points of every contact and the scatter
  int st = setup_pairs(c, hier, n_pairs, ab, eps, poses, s);
  if (st != MRDEM_OK) return st;
  return launch_grad_closest(c, hier, n_pairs, ab, poses, con, mass, k_s, scale, dverts, dpose,
                             jac, s);
}

}  // namespace mrdem
