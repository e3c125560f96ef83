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
// weights of the closest points (in float: the vertex gradient is a float
// output) from the body-frame triangles, and scatters
//   dE/dv = R^T (w e'(d) (+-u))  for the six vertices,
//   dE/dt = +-e'(d) u, dE/dtheta = (p - t) x (+-e'(d) u),
//   jac  += e''(d) J J^T, J = [u, (pa - t_A) x u, -u, -(pb - t_B) x u].
// Per-pair outputs (forces, pose gradients, Jacobian blocks) are summed over
// the contacts of a pair within a warp first, one atomic per group.  Both
// kernels reduce their FP64 inputs to the differences the formulas need
// (closest points minus each other and minus the particles' positions or
// centres of mass) in FP64, round those to double-float by integer
// operations (mrdem_split.cuh) and do the rest, the per-pair sums included,
// in double-float on the FP32 units; the sums are rounded to double for the
// atomics.  The energy stays in FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "mrdem_device.cuh"
#include "mrdem_split.cuh"

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


// Unit direction of a contact in the world frame: (pa - pb)/d, at d = 0
// minus the outward unit normal of A's triangle.
__device__ __forceinline__ D3 contact_dir(const HierDev& H, double d, D3 pa, D3 pb, int slot_a,
                                          const double RA[9]) {
  if (d > 0.0) return (1.0 / d) * (pa - pb);
  D3 V[3];
  load_tri64(H, slot_a, V);
  D3 n = cross(V[1] - V[0], V[2] - V[0]);
  return mul(RA, (-1.0 / sqrt(dot(n, n))) * n);
}

// Per-call tables built once by k_frames: per particle R (row-major), t and
// the world centre of mass (zero without com), 16 doubles, and R again in
// float (12 floats); per pair K_s sqrt(mu) and 1/(2 eps).  The contact
// kernels read them instead of rebuilding rotations and dividing per contact.
constexpr int kFrame = 16, kFrameF = 12;
struct Tables {
  double* fr;   // [n_particles * kFrame]
  float* frf;   // [n_particles * kFrameF]
  double2* pc;  // [n_pairs]
};
__global__ void __launch_bounds__(64) k_frames(int n, int64_t n_pairs,
                                                const double* __restrict__ poses,
                                                const double* __restrict__ com,
                                                const int32_t* __restrict__ ab,
                                                const double* __restrict__ eps,
                                                const double* __restrict__ mass, double k_s,
                                                Tables T) {
  wait_prior_grid();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double* p = poses + 7 * i;
    double R[9];
    pose_matrix(p, R);
    double* o = T.fr + kFrame * i;
    float* of = T.frf + kFrameF * i;
    for (int q = 0; q < 9; ++q) {
      o[q] = R[q];
      of[q] = (float)R[q];
    }
    of[9] = of[10] = of[11] = 0.f;
    o[9] = p[0]; o[10] = p[1]; o[11] = p[2];
    D3 c = com ? mul(R, {com[3 * i], com[3 * i + 1], com[3 * i + 2]}) : D3{0.0, 0.0, 0.0};
    o[12] = c.x + p[0]; o[13] = c.y + p[1]; o[14] = c.z + p[2];
    o[15] = 0.0;
  }
  if (i < n_pairs) {
    int A = ab[2 * i], B = ab[2 * i + 1];
    double ks = 0.0;
    if (A >= 0 && A < n && B >= 0 && B < n) {
      const double mA = mass[A], mB = mass[B];
      ks = k_s * sqrt(mA * mB / (mA + mB));
    }
    T.pc[i] = make_double2(ks, 0.5 / eps[i]);
  }
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
__device__ __forceinline__ void frame_Rf(const float* frf, int i, float R[9]) {
  const float4* f = reinterpret_cast<const float4*>(frf + kFrameF * (int64_t)i);
  float4 a = __ldg(f), b = __ldg(f + 1), c = __ldg(f + 2);
  R[0] = a.x; R[1] = a.y; R[2] = a.z; R[3] = a.w; R[4] = b.x; R[5] = b.y; R[6] = b.z;
  R[7] = b.w; R[8] = c.x;
}
__device__ __forceinline__ D3 frame_vec(const double* fr, int i, int at) {
  const double* f = fr + kFrame * (int64_t)i + at;
  return {__ldg(f), __ldg(f + 1), __ldg(f + 2)};
}
// float helpers of the vertex gradient (a float output)
__device__ __forceinline__ F3 mul_tf(const float R[9], F3 v) {
  return {fmaf(R[0], v.x, fmaf(R[3], v.y, R[6] * v.z)), fmaf(R[1], v.x, fmaf(R[4], v.y, R[7] * v.z)),
          fmaf(R[2], v.x, fmaf(R[5], v.y, R[8] * v.z))};
}
// Barycentric weights of a point x of triangle V, in float: least squares in
// the triangle's plane; a degenerate triangle puts all weight on V0.
__device__ __forceinline__ void barycentric_f(const F3 V[3], F3 x, float w[3]) {
  F3 e1 = V[1] - V[0], e2 = V[2] - V[0], r = x - V[0];
  float d11 = dot(e1, e1), d12 = dot(e1, e2), d22 = dot(e2, e2);
  float r1 = dot(r, e1), r2 = dot(r, e2);
  float den = d11 * d22 - d12 * d12;
  if (!(den > 0.f)) {
    w[0] = 1.f; w[1] = 0.f; w[2] = 0.f;
    return;
  }
  float inv = 1.f / den;
  w[1] = (d22 * r1 - d12 * r2) * inv;
  w[2] = (d11 * r2 - d12 * r1) * inv;
  w[0] = 1.f - w[1] - w[2];
}

constexpr int kForceThreads = 128;

__global__ void __launch_bounds__(kForceThreads) k_forces(
    HierDev H, const int32_t* __restrict__ ab, const double* __restrict__ eps, mrdem_contacts c,
    const double2* __restrict__ pc, const double* __restrict__ fr, double* ft, double* energy,
    int64_t n_pairs) {
  wait_prior_grid();
  __shared__ dd sF[kForceThreads / 32][32][9];  // F, (x - c_A) x F, (x - c_B) x (-F)
  dd(*F9)[9] = sF[threadIdx.x >> 5];
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
      const double2 kc = __ldg(pc + p);  // K_s sqrt(mu), 1/(2 eps)
      const double ks = kc.x;
      D3 pa = {c.point_a[3 * k], c.point_a[3 * k + 1], c.point_a[3 * k + 2]};
      D3 pb = {c.point_b[3 * k], c.point_b[3 * k + 1], c.point_b[3 * k + 2]};
      // double-float from here on (the FP64 inputs reduced to differences
      // first): u, F and the torques about the centres of mass, with the
      // lever arms x - c_A = (pa - c_A) - (pa - pb)/2 and
      // x - c_B = (pb - c_B) + (pa - pb)/2
      const V3<dd> diff = split_double(pa - pb);
      V3<dd> u;
      if (d > 0.0) {
        u = (dd(1.f) / split_double(d)) * diff;
      } else {
        double RA[9];
        frame_R(fr, A, RA);
        u = split_double(contact_dir(H, d, pa, pb, H.tri_slot[H.tri_off[A] + c.tri_a[k]], RA));
      }
      const double s = 1.0 - d * kc.y;
      const V3<dd> F = split_double(ks * s) * u;
      e_k = ks * e * s * s;
      const V3<dd> half = {dd(0.5f * diff.x.hi, 0.5f * diff.x.lo), dd(0.5f * diff.y.hi, 0.5f * diff.y.lo),
                           dd(0.5f * diff.z.hi, 0.5f * diff.z.lo)};
      const V3<dd> la = split_double(pa - frame_vec(fr, A, 12)) - half;
      const V3<dd> lb = split_double(pb - frame_vec(fr, B, 12)) + half;
      const V3<dd> tA = cross(la, F), tB = cross(F, lb);  // (x - c_B) x (-F)
      F9[lane][0] = F.x; F9[lane][1] = F.y; F9[lane][2] = F.z;
      F9[lane][3] = tA.x; F9[lane][4] = tA.y; F9[lane][5] = tA.z;
      F9[lane][6] = tB.x; F9[lane][7] = tB.y; F9[lane][8] = tB.z;
    }
    if (ft) {
      __syncwarp();
      warp_group_sums<dd>(
          ok, p, 9, [&](int q) { return [&, q](int l) { return F9[l][q]; }; },
          [&](int pk, int q, dd sum) {
            const double v = to_double(sum);
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

// Adjoint, one thread per contact, in double-float on the FP32 units (the
// FP64 rate of this part is about 1/61 of its FP32 rate, and this kernel
// was bound by it): the FP64 inputs are first reduced to the differences
// the formulas need (closest points minus each other and minus the
// particles' positions, and the two scalar coefficients) and rounded to
// double-float once; the direction u, the lever arms, the Gauss-Newton
// vector W = (u, (pa - t_A) x u, (pb - t_B) x u), e''(d) W, the
// pose-gradient terms (e' u, (pa - t_A) x e' u, (pb - t_B) x (-e' u)) and
// the per-pair sums over a warp's contacts then run in double-float
// (relative error about 2^-44 per operation), and each sum is rounded to
// double for its atomic.  The 12-row J = (W0, W1, -W0, -W2) makes J J^T a
// signed copy of the 9x9 Gram matrix of W, so a pair's block needs 45 sums.
constexpr int kGradThreads = 128;
struct GradSmem {
  dd w[32][9];
  dd hw[32][9];
  dd g[32][9];
  double gram[45];
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
    const double* __restrict__ fr, const float* __restrict__ frf, const double2* __restrict__ pc,
    mrdem_contacts c, double scale, float* dverts, double* dpose, double* jac, int64_t n_pairs) {
  wait_prior_grid();
  __shared__ GradSmem smem[kGradThreads / 32];
  GradSmem& S = smem[threadIdx.x >> 5];
  const int lane = lane_id();
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
      const double2 kc = __ldg(pc + p);  // K_s sqrt(mu), 1/(2 eps)
      const double ks = kc.x, inv2e = kc.y;
      D3 pa = {c.point_a[3 * k], c.point_a[3 * k + 1], c.point_a[3 * k + 2]};
      D3 pb = {c.point_b[3 * k], c.point_b[3 * k + 1], c.point_b[3 * k + 2]};
      int sa = H.tri_slot[H.tri_off[A] + c.tri_a[k]];
      int sb = H.tri_slot[H.tri_off[B] + c.tri_b[k]];
      V3<dd> u;
      if (d > 0.0) {
        u = (dd(1.f) / split_double(d)) * split_double(pa - pb);
      } else {
        double RA[9];
        frame_R(fr, A, RA);
        u = split_double(contact_dir(H, d, pa, pb, sa, RA));
      }
      const V3<dd> gv = split_double(-ks * (1.0 - d * inv2e) * scale) * u;
      const V3<dd> ra = split_double(pa - frame_vec(fr, A, 9));
      const V3<dd> rb = split_double(pb - frame_vec(fr, B, 9));
      if (dverts) {
        // a float output: body-frame closest points and their weights in
        // float from the world offsets; the gradient of a body-frame vertex
        // is R^T of the world one
        float RA[9], RB[9];
        frame_Rf(frf, A, RA);
        frame_Rf(frf, B, RB);
        F3 VA[3], VB[3];
        load_tri(H, sa, VA);
        load_tri(H, sb, VB);
        float wa[3], wb[3];
        barycentric_f(VA, mul_tf(RA, F3{ra.x.hi, ra.y.hi, ra.z.hi}), wa);
        barycentric_f(VB, mul_tf(RB, F3{rb.x.hi, rb.y.hi, rb.z.hi}), wb);
        const F3 g = {gv.x.hi, gv.y.hi, gv.z.hi};
        const F3 gA = mul_tf(RA, g), gB = mul_tf(RB, g);
        for (int v = 0; v < 3; ++v) {
          int64_t ia = 3 * (int64_t)H.vid[v * H.stride + sa], ib = 3 * (int64_t)H.vid[v * H.stride + sb];
          atomicAdd(dverts + ia, wa[v] * gA.x);
          atomicAdd(dverts + ia + 1, wa[v] * gA.y);
          atomicAdd(dverts + ia + 2, wa[v] * gA.z);
          atomicAdd(dverts + ib, -wb[v] * gB.x);
          atomicAdd(dverts + ib + 1, -wb[v] * gB.y);
          atomicAdd(dverts + ib + 2, -wb[v] * gB.z);
        }
      }
      const V3<dd> c1 = cross(ra, u), c2 = cross(rb, u);
      const V3<dd> t1 = cross(ra, gv), t2 = cross(gv, rb);  // (pb - t_B) x (-e' u)
      const dd h = split_double(ks * inv2e * scale);
      const dd W[9] = {u.x, u.y, u.z, c1.x, c1.y, c1.z, c2.x, c2.y, c2.z};
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        S.w[lane][q] = W[q];
        S.hw[lane][q] = h * W[q];
      }
      dd* g = S.g[lane];
      g[0] = gv.x; g[1] = gv.y; g[2] = gv.z; g[3] = t1.x; g[4] = t1.y; g[5] = t1.z;
      g[6] = t2.x; g[7] = t2.y; g[8] = t2.z;
    }
    if (!dpose && !jac) continue;
    __syncwarp();
    const int q0 = jac ? 0 : 45, q1 = dpose ? 54 : 45;
    warp_group_sums<dd>(
        ok, p, q1 - q0,
        [&](int q) {
          q += q0;
          // Gram sums read (hw_i, w_j) of each lane; pose sums g_q
          int i, j;
          gram_pair(q < 45 ? q : 0, i, j);
          const dd* x = q < 45 ? &S.hw[0][i] : &S.g[0][q - 45];
          const dd* y = &S.w[0][j];
          const bool prod = q < 45;
          return [x, y, prod](int l) { return prod ? x[9 * l] * y[9 * l] : x[9 * l]; };
        },
        [&](int pk, int q, dd sum) {
          const double v = to_double(sum);
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

// Forces and the adjoint keep their tables in separate buffers (which = 0
// or 1), so that the two calls may run concurrently on two streams.
static int ensure_tables(mrdem_ctx* c, int which, int64_t n, int64_t n_pairs, Tables* T) {
  // doubles: frames, then pair constants (2 each); floats after them
  const int64_t nd = kFrame * n + 2 * n_pairs, nf = kFrameF * n;
  const int64_t need = nd + (nf + 1) / 2;
  double*& buf = which ? c->frames_grad : c->frames;
  int64_t& cap = which ? c->cap_frames_grad : c->cap_frames;
  if (need > cap) {
    cudaFree(buf);
    buf = nullptr;
    cap = 0;
    if (cudaMalloc(&buf, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      return MRDEM_ERR_OOM;
    }
    cap = need;
  }
  T->fr = buf;
  T->pc = reinterpret_cast<double2*>(buf + kFrame * n);
  T->frf = reinterpret_cast<float*>(buf + nd);
  return MRDEM_OK;
}

static int launch_tables(mrdem_ctx* c, int which, const mrdem_hier* hier, int64_t n_pairs,
                         const int32_t* ab, const double* eps, const double* poses,
                         const double* mass, const double* com, double k_s, Tables* T,
                         cudaStream_t s) {
  int n = hier->dev.n_particles;
  int st = ensure_tables(c, which, n, n_pairs, T);
  if (st) return st;
  int64_t m = std::max<int64_t>(n, n_pairs);
  if (m > 0)
    launch_after(k_frames, (unsigned)((m + 63) / 64), 64, 0, s, n, n_pairs, poses, com, ab, eps,
                 mass, k_s, *T);
  return MRDEM_OK;
}

int launch_forces(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                  const double* eps, const double* poses, const mrdem_contacts* con,
                  const double* mass, const double* com, double k_s, double* ft, double* energy,
                  cudaStream_t s) {
  if (!ft && !energy) return MRDEM_OK;
  ProfScope ps(c, K_FORCES, s);
  Tables T;
  int st = launch_tables(c, 0, hier, n_pairs, ab, eps, poses, mass, com, k_s, &T, s);
  if (st) return st;
  launch_after(k_forces, c->n_sms * 16, kForceThreads, 0, s, hier->dev, ab, eps, *con,
               (const double2*)T.pc, (const double*)T.fr, ft, energy, n_pairs);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

int launch_grad(mrdem_ctx* c, const mrdem_hier* hier, int64_t n_pairs, const int32_t* ab,
                const double* eps, const double* poses, const mrdem_contacts* con,
                const double* mass, double k_s, double scale, float* dverts, double* dpose,
                double* jac, cudaStream_t s) {
  if (!dverts && !dpose && !jac) return MRDEM_OK;
  if (n_pairs == 0) return MRDEM_OK;
  ProfScope ps(c, K_GRAD, s);
  Tables T;
  int st = launch_tables(c, 1, hier, n_pairs, ab, eps, poses, mass, nullptr, k_s, &T, s);
  if (st) return st;
  launch_after(k_grad, c->n_sms * 16, kGradThreads, 0, s, hier->dev, ab, eps, (const double*)T.fr,
               (const float*)T.frf, (const double2*)T.pc, *con, scale, dverts, dpose, jac,
               n_pairs);
  return cudaGetLastError() == cudaSuccess ? MRDEM_OK : MRDEM_ERR_CUDA;
}

}  // namespace mrdem
