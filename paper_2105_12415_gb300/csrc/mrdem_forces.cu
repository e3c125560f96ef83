// mrdem_forces.cu -- penalty forces of a contact set and their adjoint.
//
// Force law of Sec. 2 of Noble & Weinzierl (arXiv 2105.12415): a contact with
// closest points pa (on A's triangle) and pb (on B's), distance d = |pa - pb|
// and |n| = d/2, pushes A along u = (pa - pb)/d with
//   |F| = K_s sqrt(mu) (1 - |n|/eps),  mu = 1/(1/M_A + 1/M_B),
// and B with -F (equal and opposite), applied at the contact point
// (pa + pb)/2.  The energy e(d) = K_s sqrt(mu) eps (1 - d/(2 eps))^2 has
// -e'(d) = |F|, so F = -dE/dt_A.  The adjoint takes each contact's distance
// and world closest points as the detection wrote them (the forward pass
// keeps what the backward pass needs), recomputes only the barycentric
// weights of the closest points in FP64 from the body-frame triangles, and
// scatters
//   dE/dv = R^T (w e'(d) (+-u))  for the six vertices,
//   dE/dt = +-e'(d) u, dE/dtheta = (p - t) x (+-e'(d) u),
//   jac  += e''(d) J J^T, J = [u, (pa - t_A) x u, -u, -(pb - t_B) x u].
// Per-pair outputs (forces, pose gradients, Jacobian blocks) are summed over
// the contacts of a pair within a warp first, one atomic per group.
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
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ D3 mul_t(const double R[9], D3 v) {
  return {R[0] * v.x + R[3] * v.y + R[6] * v.z, R[1] * v.x + R[4] * v.y + R[7] * v.z,
          R[2] * v.x + R[5] * v.y + R[8] * v.z};
}
__device__ __forceinline__ D3 body_vertex(const HierDev& H, int slot, int c) {
  return {(double)H.tri[(3 * c) * H.stride + slot], (double)H.tri[(3 * c + 1) * H.stride + slot],
          (double)H.tri[(3 * c + 2) * H.stride + slot]};
}
// Barycentric weights of a point x of the triangle V (least squares in the
// triangle's plane; a degenerate triangle puts all weight on V0).
__device__ __forceinline__ void barycentric(const D3 V[3], D3 x, double w[3]) {
  D3 e1 = V[1] - V[0], e2 = V[2] - V[0], r = x - V[0];
  double d11 = dot(e1, e1), d12 = dot(e1, e2), d22 = dot(e2, e2);
  double r1 = dot(r, e1), r2 = dot(r, e2);
  double den = d11 * d22 - d12 * d12;
  if (!(den > 0.0)) {
    w[0] = 1.0; w[1] = 0.0; w[2] = 0.0;
    return;
  }
  double inv = 1.0 / den;
  w[1] = (d22 * r1 - d12 * r2) * inv;
  w[2] = (d11 * r2 - d12 * r1) * inv;
  w[0] = 1.0 - w[1] - w[2];
}
// Unit direction of a contact in the world frame: (pa - pb)/d, at d = 0
// minus the outward unit normal of A's triangle.
__device__ __forceinline__ D3 contact_dir(const HierDev& H, double d, D3 pa, D3 pb, int slot_a,
                                          const double RA[9]) {
  if (d > 0.0) return (1.0 / d) * (pa - pb);
  D3 V[3] = {body_vertex(H, slot_a, 0), body_vertex(H, slot_a, 1), body_vertex(H, slot_a, 2)};
  D3 n = cross(V[1] - V[0], V[2] - V[0]);
  return mul(RA, (-1.0 / sqrt(dot(n, n))) * n);
}

// Per-particle frames, once per call: R (row-major), t and the world centre
// of mass (zero without com), 16 doubles per particle.  The contact kernels
// read them instead of rebuilding both rotation matrices for every contact.
constexpr int kFrame = 16;
__global__ void __launch_bounds__(256) k_frames(int n, const double* __restrict__ poses,
                                                const double* __restrict__ com, double* fr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* p = poses + 7 * (int64_t)i;
  double R[9];
  pose_matrix(p, R);
  double* o = fr + kFrame * (int64_t)i;
  for (int q = 0; q < 9; ++q) o[q] = R[q];
  o[9] = p[0]; o[10] = p[1]; o[11] = p[2];
  D3 c = com ? mul(R, {com[3 * i], com[3 * i + 1], com[3 * i + 2]}) : D3{0.0, 0.0, 0.0};
  o[12] = c.x + p[0]; o[13] = c.y + p[1]; o[14] = c.z + p[2];
  o[15] = 0.0;
}
__device__ __forceinline__ void frame_R(const double* fr, int i, double R[9]) {
  const double2* f = reinterpret_cast<const double2*>(fr + kFrame * (int64_t)i);
  for (int q = 0; q < 4; ++q) {
    double2 v = __ldg(f + q);
    R[2 * q] = v.x;
    R[2 * q + 1] = v.y;
  }
  R[8] = __ldg(fr + kFrame * (int64_t)i + 8);
}
__device__ __forceinline__ D3 frame_vec(const double* fr, int i, int at) {
  const double* f = fr + kFrame * (int64_t)i + at;
  return {__ldg(f), __ldg(f + 1), __ldg(f + 2)};
}

constexpr int kForceThreads = 128;

__global__ void __launch_bounds__(kForceThreads) k_forces(
    HierDev H, const int32_t* __restrict__ ab, const double* __restrict__ eps, mrdem_contacts c,
    const double* __restrict__ mass, const double* __restrict__ fr, double k_s, double* ft,
    double* energy, int64_t n_pairs) {
  __shared__ double sF[kForceThreads / 32][32][9];  // F, (x - c_A) x F, (x - c_B) x (-F)
  double(*F9)[9] = sF[threadIdx.x >> 5];
  const int lane = lane_id();
  int64_t n = *c.count;
  if (n > c.capacity) n = c.capacity;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    double e_k = 0.0;
    int p = k < n ? c.pair[k] : -1;
    bool ok = p >= 0 && p < n_pairs;
    if (ok) {
      int A = ab[2 * p], B = ab[2 * p + 1];
      double e = eps[p], d = c.dist[k];
      const double mA = mass[A], mB = mass[B];
      double ks = k_s * sqrt(mA * mB / (mA + mB));
      D3 pa = {c.point_a[3 * k], c.point_a[3 * k + 1], c.point_a[3 * k + 2]};
      D3 pb = {c.point_b[3 * k], c.point_b[3 * k + 1], c.point_b[3 * k + 2]};
      D3 u;
      if (d > 0.0) {
        u = (1.0 / d) * (pa - pb);
      } else {
        double RA[9];
        frame_R(fr, A, RA);
        u = contact_dir(H, d, pa, pb, H.tri_slot[H.tri_off[A] + c.tri_a[k]], RA);
      }
      double s = 1.0 - d / (2.0 * e);
      D3 F = (ks * s) * u;
      e_k = ks * e * s * s;
      D3 xc = 0.5 * (pa + pb);
      D3 cA = frame_vec(fr, A, 12), cB = frame_vec(fr, B, 12);
      D3 tA = cross(xc - cA, F), tB = cross(xc - cB, -1.0 * F);
      F9[lane][0] = F.x; F9[lane][1] = F.y; F9[lane][2] = F.z;
      F9[lane][3] = tA.x; F9[lane][4] = tA.y; F9[lane][5] = tA.z;
      F9[lane][6] = tB.x; F9[lane][7] = tB.y; F9[lane][8] = tB.z;
    }
    if (ft) {
      __syncwarp();
      warp_group_sums(
          ok, p, 9, [&](int q) { return [&, q](int l) { return F9[l][q]; }; },
          [&](int pk, int q, double v) {
            int A = ab[2 * pk], B = ab[2 * pk + 1];
            if (q < 3) {
              atomicAdd(ft + 6 * (int64_t)A + q, v);
              atomicAdd(ft + 6 * (int64_t)B + q, -v);
            } else if (q < 6) {
              atomicAdd(ft + 6 * (int64_t)A + q, v);
            } else {
              atomicAdd(ft + 6 * (int64_t)B + q - 3, v);
            }
          },
          [](int) {});
    }
    if (energy) {
      double w = warp_sum(e_k);
      if (lane == 0 && w != 0.0) atomicAdd(energy, w);
    }
  }
}

// Adjoint, one thread per contact.  Per lane in shared memory: the Gauss-
// Newton vector W = (u, (pa - t_A) x u, (pb - t_B) x u), e''(d) W, and the
// pose gradient (e' u, (pa - t_A) x e' u, (pb - t_B) x (-e' u)).  The 12-row
// J = (W0, W1, -W0, -W2) makes J J^T a signed copy of the 9x9 Gram matrix of
// W, so a pair's block needs 45 sums, one FMA per contact each.
constexpr int kGradThreads = 128;
struct GradSmem {
  double w[32][9];
  double hw[32][9];
  double g[32][9];
  double gram[45];
  double one;
};
// Row of the 12 pose unknowns -> (index into W, sign).
__device__ __forceinline__ int w_index(int r, double& sgn) {
  sgn = r < 6 ? 1.0 : -1.0;
  return r < 6 ? r : (r < 9 ? r - 6 : r - 3);
}
// Upper-triangle index of (i, j), i <= j < 9, and its inverse.
__device__ __forceinline__ int gram_index(int i, int j) { return i * 9 - (i * (i - 1)) / 2 + (j - i); }
__device__ __forceinline__ void gram_pair(int e, int& i, int& j) {
  i = 0;
  while (e >= 9 - i) {
    e -= 9 - i;
    ++i;
  }
  j = i + e;
}

__global__ void __launch_bounds__(kGradThreads) k_grad(
    HierDev H, const int32_t* __restrict__ ab, const double* __restrict__ eps,
    const double* __restrict__ fr, mrdem_contacts c, const double* __restrict__ mass,
    double k_s, double scale, float* dverts, double* dpose, double* jac, int64_t n_pairs) {
  __shared__ GradSmem smem[kGradThreads / 32];
  GradSmem& S = smem[threadIdx.x >> 5];
  const int lane = lane_id();
  if (lane == 0) S.one = 1.0;
  __syncwarp();
  int64_t n = *c.count;
  if (n > c.capacity) n = c.capacity;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    int64_t k = base + threadIdx.x;
    int p = k < n ? c.pair[k] : -1;
    bool ok = p >= 0 && p < n_pairs;
    double d = 0.0, e = 0.0;
    if (ok) {
      e = eps[p];
      d = c.dist[k];
      ok = d <= 2.0 * e;
    }
    if (ok) {
      int A = ab[2 * p], B = ab[2 * p + 1];
      const double mA = mass[A], mB = mass[B];
      const double ks = k_s * sqrt(mA * mB / (mA + mB));
      const double inv2e = 0.5 / e;
      D3 pa = {c.point_a[3 * k], c.point_a[3 * k + 1], c.point_a[3 * k + 2]};
      D3 pb = {c.point_b[3 * k], c.point_b[3 * k + 1], c.point_b[3 * k + 2]};
      double RA[9], RB[9];
      frame_R(fr, A, RA);
      frame_R(fr, B, RB);
      int sa = H.tri_slot[H.tri_off[A] + c.tri_a[k]];
      int sb = H.tri_slot[H.tri_off[B] + c.tri_b[k]];
      D3 u = contact_dir(H, d, pa, pb, sa, RA);
      D3 gv = (-ks * (1.0 - d * inv2e) * scale) * u;
      D3 ra = pa - frame_vec(fr, A, 9), rb = pb - frame_vec(fr, B, 9);
      if (dverts) {
        // body-frame closest points and their weights; the gradient of a
        // body-frame vertex is R^T of the world one
        D3 VA[3] = {body_vertex(H, sa, 0), body_vertex(H, sa, 1), body_vertex(H, sa, 2)};
        D3 VB[3] = {body_vertex(H, sb, 0), body_vertex(H, sb, 1), body_vertex(H, sb, 2)};
        double wa[3], wb[3];
        barycentric(VA, mul_t(RA, ra), wa);
        barycentric(VB, mul_t(RB, rb), wb);
        D3 gA = mul_t(RA, gv), gB = mul_t(RB, gv);
        for (int v = 0; v < 3; ++v) {
          int64_t ia = 3 * (int64_t)H.vid[v * H.stride + sa], ib = 3 * (int64_t)H.vid[v * H.stride + sb];
          atomicAdd(dverts + ia, (float)(wa[v] * gA.x));
          atomicAdd(dverts + ia + 1, (float)(wa[v] * gA.y));
          atomicAdd(dverts + ia + 2, (float)(wa[v] * gA.z));
          atomicAdd(dverts + ib, (float)(-wb[v] * gB.x));
          atomicAdd(dverts + ib + 1, (float)(-wb[v] * gB.y));
          atomicAdd(dverts + ib + 2, (float)(-wb[v] * gB.z));
        }
      }
      D3 c1 = cross(ra, u), c2 = cross(rb, u);
      D3 t1 = cross(ra, gv), t2 = cross(rb, -1.0 * gv);
      const double W[9] = {u.x, u.y, u.z, c1.x, c1.y, c1.z, c2.x, c2.y, c2.z};
      const double h = ks * inv2e * scale;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        S.w[lane][q] = W[q];
        S.hw[lane][q] = h * W[q];
      }
      double* g = S.g[lane];
      g[0] = gv.x; g[1] = gv.y; g[2] = gv.z; g[3] = t1.x; g[4] = t1.y; g[5] = t1.z;
      g[6] = t2.x; g[7] = t2.y; g[8] = t2.z;
    }
    if (!dpose && !jac) continue;
    __syncwarp();
    const int q0 = jac ? 0 : 45, q1 = dpose ? 54 : 45;
    warp_group_sums(
        ok, p, q1 - q0,
        [&](int q) {
          q += q0;
          // Gram sums read (hw_i, w_j) of each lane; pose sums (g_q, 1)
          int i, j;
          gram_pair(q < 45 ? q : 0, i, j);
          const double* x = q < 45 ? &S.hw[0][i] : &S.g[0][q - 45];
          const double* y = q < 45 ? &S.w[0][j] : &S.one;
          const int ys = q < 45 ? 9 : 0;
          return [x, y, ys](int l) { return x[9 * l] * y[ys * l]; };
        },
        [&](int pk, int q, double v) {
          q += q0;
          if (q < 45) {
            S.gram[q] = v;
            return;
          }
          q -= 45;
          int A = ab[2 * pk], B = ab[2 * pk + 1];
          if (q < 3) {
            atomicAdd(dpose + 6 * (int64_t)A + q, v);
            atomicAdd(dpose + 6 * (int64_t)B + q, -v);
          } else if (q < 6) {
            atomicAdd(dpose + 6 * (int64_t)A + q, v);
          } else {
            atomicAdd(dpose + 6 * (int64_t)B + q - 3, v);
          }
        },
        [&](int pk) {
          if (!jac) return;
          double* o = jac + 144 * (int64_t)pk;
          for (int x = lane; x < 144; x += 32) {
            double sr, sq;
            int i = w_index(x / 12, sr), j = w_index(x % 12, sq);
            atomicAdd(o + x, sr * sq * S.gram[i <= j ? gram_index(i, j) : gram_index(j, i)]);
          }
        });
  }
}

}  // namespace

static int ensure_frames(mrdem_ctx* c, int64_t n) {
  if (n <= c->cap_frames) return MRDEM_OK;
  cudaFree(c->frames);
  c->frames = nullptr;
  c->cap_frames = 0;
  if (cudaMalloc(&c->frames, sizeof(double) * kFrame * n) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_OOM;
  }
  c->cap_frames = n;
  return MRDEM_OK;
}

static int launch_frames(mrdem_ctx* c, const mrdem_hier* hier, const double* poses,
                         const double* com, cudaStream_t s) {
  int n = hier->dev.n_particles;
  int st = ensure_frames(c, n);
  if (st) return st;
  if (n > 0) k_frames<<<(n + 255) / 256, 256, 0, s>>>(n, poses, com, c->frames);
  return MRDEM_OK;
}

int launch_forces(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                  const double* eps, const double* poses, const mrdem_contacts* con,
                  const double* mass, const double* com, double k_s, double* ft, double* energy,
                  cudaStream_t s) {
  if (!ft && !energy) return MRDEM_OK;
  ProfScope ps(c, K_FORCES, s);
  int st = launch_frames(c, hier, poses, com, s);
  if (st) return st;
  k_forces<<<c->n_sms * 16, kForceThreads, 0, s>>>(hier->dev, ab, eps, *con, mass, c->frames,
                                                    k_s, ft, energy, n_pairs);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_grad(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                const double* eps, const double* poses, const mrdem_contacts* con,
                const double* mass, double k_s, double scale, float* dverts, double* dpose,
                double* jac, cudaStream_t s) {
  if (!dverts && !dpose && !jac) return MRDEM_OK;
  if (n_pairs == 0) return MRDEM_OK;
  ProfScope ps(c, K_GRAD, s);
  int st = launch_frames(c, hier, poses, nullptr, s);
  if (st) return st;
  k_grad<<<c->n_sms * 16, kGradThreads, 0, s>>>(hier->dev, ab, eps, c->frames, *con, mass, k_s,
                                                 scale, dverts, dpose, jac, n_pairs);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
