// mrdem_api.cpp -- the C ABI declared in include/mrdem.h: contexts, parameter
// validation, hierarchy build/upload/export and argument checks in front of
// the kernel launchers.  No exception crosses the boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <new>

#include "mrdem_internal.h"

using namespace mrdem;

namespace {

// The FP32 exact pass packs a candidate's index and a sub-test number (4
// bits) into one int32 work item.
constexpr int64_t kMaxCandidates = (int64_t)1 << 27;

bool one_of(int32_t v, std::initializer_list<int32_t> allowed) {
  for (int32_t a : allowed)
    if (v == a) return true;
  return false;
}

bool params_ok(const mrdem_params& p) {
  return p.n_iter >= 1 && p.n_iter <= 64 && p.rho_reg > 0.f && p.rho_iter > 0.f && p.conv_c > 0.f &&
         p.fanout >= 2 && p.fanout <= 8 && p.leaf_max >= 1 && p.leaf_max <= 32 && p.leaf_min >= 1 &&
         p.kmeans_iters >= 0 && p.cap_level > 0 && p.cap_tiles > 0 && p.cap_candidates > 0 &&
         p.cap_level < (int64_t)1 << 31 && p.cap_tiles < (int64_t)1 << 31 &&
         p.cap_candidates < kMaxCandidates && p.cap_sweep > 0 && p.cap_sweep < (int64_t)1 << 31 &&
         one_of(p.tile_warps, {2, 4, 8}) && one_of(p.sweep_warps, {2, 4, 8}) &&
         one_of(p.level_warps, {2, 4, 8}) && one_of(p.exact_threads, {64, 128, 256}) &&
         one_of(p.expand_items, {8, 16, 32}) && one_of(p.node_threads, {128, 256}) &&
         one_of(p.level_kernel, {0, 1, 2});
}

void free_lists(mrdem_ctx* c) {
  cudaFree(c->level_list[0]);
  cudaFree(c->level_list[1]);
  cudaFree(c->tiles);
  cudaFree(c->cands);
  cudaFree(c->sweep);
  c->sweep = nullptr;
  cudaFree(c->acc);
  cudaFree(c->items_pt);
  cudaFree(c->items_ee);
  cudaFree(c->res_pt);
  cudaFree(c->res_ee);
  cudaFree(c->items_cx);
  cudaFree(c->res_cx);
  cudaFree(c->d2_pt);
  c->d2_pt = c->d2_ee = c->d2_cx = nullptr;
  c->acc = nullptr;
  c->items_pt = c->items_ee = c->items_cx = nullptr;
  c->res_pt = c->res_ee = c->res_cx = nullptr;
  c->cap_items = 0;
  c->level_list[0] = c->level_list[1] = nullptr;
  c->tiles = nullptr;
  c->cands = nullptr;
  c->cap_level = c->cap_tiles = c->cap_cands = c->cap_sweep = 0;
}

int alloc_lists(mrdem_ctx* c, int64_t lv, int64_t ti, int64_t ca, int64_t sw) {
  free_lists(c);
  if (cudaMalloc(&c->level_list[0], sizeof(int4) * lv) != cudaSuccess ||
      cudaMalloc(&c->level_list[1], sizeof(int4) * lv) != cudaSuccess ||
      cudaMalloc(&c->tiles, sizeof(TileItem) * ti) != cudaSuccess ||
      cudaMalloc(&c->cands, sizeof(int3) * ca) != cudaSuccess ||
      cudaMalloc(&c->sweep, sizeof(int4) * sw) != cudaSuccess ||
      cudaMalloc(&c->acc, sizeof(AccRec) * ca) != cudaSuccess ||
      cudaMalloc(&c->items_pt, sizeof(int) * 2 * ca) != cudaSuccess ||
      cudaMalloc(&c->items_ee, sizeof(int) * 2 * ca) != cudaSuccess ||
      cudaMalloc(&c->res_pt, sizeof(ItemRes) * 2 * ca) != cudaSuccess ||
      cudaMalloc(&c->res_ee, sizeof(ItemRes) * 2 * ca) != cudaSuccess ||
      cudaMalloc(&c->items_cx, sizeof(int) * 2 * ca) != cudaSuccess ||
      cudaMalloc(&c->res_cx, sizeof(ItemRes) * 2 * ca) != cudaSuccess ||
      cudaMalloc(&c->d2_pt, sizeof(dd) * 3 * 2 * ca) != cudaSuccess) {
    cudaGetLastError();
    free_lists(c);
    return MRDEM_ERR_OOM;
  }
  c->cap_level = lv;
  c->cap_tiles = ti;
  c->cap_cands = ca;
  c->cap_sweep = sw;
  c->cap_items = 2 * ca;
  c->d2_ee = c->d2_pt + 2 * ca;
  c->d2_cx = c->d2_ee + 2 * ca;
  return MRDEM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(d);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool contacts_ok(const mrdem_contacts* c) {
  return c && c->capacity >= 0 && c->count &&
         (c->capacity == 0 || (c->pair && c->tri_a && c->tri_b && c->dist && c->point_a && c->point_b));
}

}  // namespace

extern "C" {

void mrdem_default_params(mrdem_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n_iter = 4;
  p->rho_reg = 1.0f;
  p->rho_iter = 100.0f;
  p->conv_c = 1.0f;
  p->fanout = 8;
  p->leaf_max = 32;
  p->leaf_min = 16;
  p->kmeans_iters = 3;
  p->cap_level = (int64_t)1 << 24;
  p->cap_tiles = (int64_t)1 << 24;
  p->cap_candidates = (int64_t)1 << 20;
  p->tile_warps = 8;
  p->sweep_warps = 4;
  p->level_warps = 8;
  p->exact_threads = 128;
  p->expand_items = 32;
  p->node_threads = 256;
  p->level_kernel = 0;
  p->cap_sweep = (int64_t)1 << 25;
}

const char* mrdem_status_string(int s) {
  switch (s) {
    case MRDEM_OK: return "ok";
    case MRDEM_ERR_INVALID: return "invalid argument";
    case MRDEM_ERR_OOM: return "out of memory";
    case MRDEM_ERR_CUDA: return "CUDA runtime error";
    case MRDEM_ERR_CAPACITY: return "work list or contact buffer capacity exceeded";
    case MRDEM_ERR_NONFINITE: return "non-finite pose or eps (or eps <= 0)";
    default: return "unknown status";
  }
}

int mrdem_create(mrdem_ctx** out, int device, const mrdem_params* p) {
  if (!out) return MRDEM_ERR_INVALID;
  *out = nullptr;
  mrdem_params prm;
  if (p) prm = *p; else mrdem_default_params(&prm);
  if (!params_ok(prm)) return MRDEM_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  DeviceGuard g(device);
  mrdem_ctx* c = new (std::nothrow) mrdem_ctx();
  if (!c) return MRDEM_ERR_OOM;
  c->device = device;
  c->params = prm;
  cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device);
  int st = alloc_lists(c, prm.cap_level, prm.cap_tiles, prm.cap_candidates, prm.cap_sweep);
  if (st == MRDEM_OK &&
      (cudaMalloc(&c->counters, sizeof(unsigned long long) * CNT_TOTAL) != cudaSuccess ||
       cudaMalloc(&c->status, sizeof(unsigned long long) * ST_TOTAL) != cudaSuccess ||
       cudaMemset(c->status, 0, sizeof(unsigned long long) * ST_TOTAL) != cudaSuccess))
    st = MRDEM_ERR_OOM;
  if (st != MRDEM_OK) {
    cudaGetLastError();
    mrdem_destroy(c);
    return st;
  }
  *out = c;
  return MRDEM_OK;
}

int mrdem_destroy(mrdem_ctx* c) {
  if (!c) return MRDEM_OK;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  for (auto& r : c->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  free_lists(c);
  cudaFree(c->xf);
  cudaFree(c->xf64);
  cudaFree(c->xfdd);
  cudaFree(c->pair_cnt);
  cudaFree(c->tmp_i);
  cudaFree(c->tmp_d);
  cudaFree(c->tmp_count);
  cudaFree(c->merge_seg);
  cudaFree(c->merge_mem);
  cudaFree(c->broad_mem);
  cudaFree(c->cg_mem);
  cudaFree(c->refine_mem);
  cudaFree(c->frames);
  cudaFree(c->frames_grad);
  cudaFree(c->as_status);
  if (c->merge_side) cudaStreamDestroy(c->merge_side);
  for (cudaEvent_t e : c->merge_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(c->counters);
  cudaFree(c->status);
  delete c;
  return MRDEM_OK;
}

int mrdem_get_params(const mrdem_ctx* c, mrdem_params* out) {
  if (!c || !out) return MRDEM_ERR_INVALID;
  *out = c->params;
  return MRDEM_OK;
}

int mrdem_set_params(mrdem_ctx* c, const mrdem_params* p) {
  if (!c || !p) return MRDEM_ERR_INVALID;
  mrdem_params n = *p;
  n.cap_level = c->params.cap_level;
  n.cap_tiles = c->params.cap_tiles;
  n.cap_candidates = c->params.cap_candidates;
  n.cap_sweep = c->params.cap_sweep;
  if (!params_ok(n)) return MRDEM_ERR_INVALID;
  c->params = n;
  c->n_occ = 0;  // launch shapes may have changed
  for (bool& t : c->tuned_ok) t = false;  // tuned shapes belong to the old parameters
  return MRDEM_OK;
}

int mrdem_reserve(mrdem_ctx* c, int64_t lv, int64_t ti, int64_t ca, int64_t sw) {
  if (!c || lv < 0 || ti < 0 || ca < 0 || sw < 0) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  lv = lv ? lv : c->cap_level;
  ti = ti ? ti : c->cap_tiles;
  ca = ca ? ca : c->cap_cands;
  sw = sw ? sw : c->cap_sweep;
  if (lv >= (int64_t)1 << 31 || ti >= (int64_t)1 << 31 || ca >= kMaxCandidates ||
      sw >= (int64_t)1 << 31)
    return MRDEM_ERR_INVALID;
  if (cudaDeviceSynchronize() != cudaSuccess) return MRDEM_ERR_CUDA;
  int st = alloc_lists(c, lv, ti, ca, sw);
  if (st == MRDEM_OK) {
    c->params.cap_level = lv;
    c->params.cap_tiles = ti;
    c->params.cap_candidates = ca;
    c->params.cap_sweep = sw;
  }
  return st;
}

int mrdem_build_hierarchy_host(const mrdem_params* params, int32_t n, const int64_t* vert_off,
                               const float* verts, const int64_t* tri_off, const int32_t* tris,
                               mrdem_hier** out) {
  if (!out) return MRDEM_ERR_INVALID;
  *out = nullptr;
  mrdem_params prm;
  if (params) prm = *params; else mrdem_default_params(&prm);
  try {
    mrdem_hier* h = new mrdem_hier();
    int st = build_hierarchy_host(prm, n, vert_off, verts, tri_off, tris, &h->h);
    if (st != MRDEM_OK) {
      delete h;
      return st;
    }
    *out = h;
    return MRDEM_OK;
  } catch (const std::bad_alloc&) {
    return MRDEM_ERR_OOM;
  } catch (...) {
    return MRDEM_ERR_INVALID;
  }
}

int mrdem_hier_upload(mrdem_ctx* c, mrdem_hier* hier) {
  if (!c || !hier) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  const HierHost& h = hier->h;
  if (hier->d_mem) {
    cudaFree(hier->d_mem);
    hier->d_mem = nullptr;
    hier->ctx = nullptr;
  }
  int64_t stride = (h.n_tri_pad + 31) / 32 * 32;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t sz_geo = al(sizeof(float4) * 3 * h.n_nodes), sz_child = al(sizeof(int2) * h.n_nodes);
  size_t sz_sph = al(sizeof(float4) * h.n_nodes), sz_nrm = sz_sph, sz_tsph = al(sizeof(float4) * stride);
  size_t sz_tri = al(sizeof(float4) * 3 * stride), sz_vid = al(sizeof(int32_t) * 3 * stride);
  size_t sz_slot = al(sizeof(int32_t) * stride), sz_ts = al(sizeof(int32_t) * h.n_tri);
  size_t sz_off = al(sizeof(int64_t) * (h.n_particles + 1));
  size_t sz_root = al(sizeof(int32_t) * h.n_particles), sz_br = al(sizeof(float) * h.n_particles);
  size_t sz_box = al(sizeof(float4) * 4 * h.n_nodes), sz_boxw = al(sizeof(float4) * h.n_nodes);
  size_t sz_up = al(sizeof(int2) * h.n_nodes);
  size_t total = sz_geo + sz_child + sz_tri + sz_vid + sz_slot + sz_ts + sz_off + sz_root + sz_br +
                 sz_sph + sz_nrm + sz_tsph + sz_box + sz_boxw + sz_up;
  char* base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_OOM;
  }
  try {
    std::vector<char> buf(total, 0);
    char* p = buf.data();
    size_t o_geo = 0, o_child = o_geo + sz_geo, o_tri = o_child + sz_child, o_vid = o_tri + sz_tri;
    size_t o_slot = o_vid + sz_vid, o_ts = o_slot + sz_slot, o_off = o_ts + sz_ts;
    size_t o_root = o_off + sz_off, o_br = o_root + sz_root, o_sph = o_br + sz_br;
    size_t o_nrm = o_sph + sz_sph, o_tsph = o_nrm + sz_nrm, o_box = o_tsph + sz_tsph;
    size_t o_boxw = o_box + sz_box, o_up = o_boxw + sz_boxw;
    // parent and level of every node (the active sets of the implicit step
    // find a pair's parent pair from them)
    int2* up = (int2*)(p + o_up);
    for (int64_t n = 0; n < h.n_nodes; ++n) up[n] = make_int2(-1, h.node_level[n]);
    for (int64_t n = 0; n < h.n_nodes; ++n) {
      const int32_t b = h.node_child[2 * n], cnt = h.node_child[2 * n + 1];
      for (int32_t k = 0; k < cnt; ++k) up[b + k].x = (int)n;
    }
    float4* geo = (float4*)(p + o_geo);
    for (int64_t n = 0; n < h.n_nodes; ++n) {
      const float* t = &h.node_tri[9 * n];
      geo[3 * n + 0] = make_float4(t[0], t[1], t[2], h.node_delta[n]);
      geo[3 * n + 1] = make_float4(t[3], t[4], t[5], 0.f);
      geo[3 * n + 2] = make_float4(t[6], t[7], t[8], 0.f);
    }
    // node spheres: centroid of the surrogate triangle and the largest vertex
    // distance plus delta, computed in double and rounded up
    float4* sph = (float4*)(p + o_sph);
    for (int64_t n = 0; n < h.n_nodes; ++n) {
      const float* t = &h.node_tri[9 * n];
      double c[3];
      for (int k = 0; k < 3; ++k) c[k] = ((double)t[k] + (double)t[3 + k] + (double)t[6 + k]) / 3.0;
      double r2 = 0;
      for (int v = 0; v < 3; ++v) {
        double d2 = 0;
        for (int k = 0; k < 3; ++k) d2 += ((double)t[3 * v + k] - c[k]) * ((double)t[3 * v + k] - c[k]);
        r2 = std::max(r2, d2);
      }
      double r = (std::sqrt(r2) + (double)h.node_delta[n]) * (1.0 + 1e-6) + 1e-30;
      sph[n] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)r);
    }
    // surrogate planes: unit normal and offset in double, stored in float
    // (a zero normal for a degenerate surrogate makes every plane test pass)
    float4* nrm = (float4*)(p + o_nrm);
    for (int64_t n = 0; n < h.n_nodes; ++n) {
      const float* t = &h.node_tri[9 * n];
      double e1[3], e2[3], nn[3];
      for (int k = 0; k < 3; ++k) {
        e1[k] = (double)t[3 + k] - (double)t[k];
        e2[k] = (double)t[6 + k] - (double)t[k];
      }
      nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
      nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
      nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
      double l = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
      double e = std::sqrt(std::max(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2],
                                    e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
      if (!(l > 1e-9 * e * e)) {
        nrm[n] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      for (int k = 0; k < 3; ++k) nn[k] /= l;
      nrm[n] = make_float4((float)nn[0], (float)nn[1], (float)nn[2],
                           (float)(nn[0] * t[0] + nn[1] * t[1] + nn[2] * t[2]));
    }
    // oriented boxes: (c.xyz, h0) (u0.xyz, h1) (u1.xyz, h2) (u2.xyz, 0)
    float4* box = (float4*)(p + o_box);
    float4* boxw = (float4*)(p + o_boxw);
    for (int64_t n = 0; n < h.n_nodes; ++n) {
      const float* b = &h.node_box[16 * n];
      box[4 * n + 0] = make_float4(b[0], b[1], b[2], b[12]);
      box[4 * n + 1] = make_float4(b[3], b[4], b[5], b[13]);
      box[4 * n + 2] = make_float4(b[6], b[7], b[8], b[14]);
      box[4 * n + 3] = make_float4(b[9], b[10], b[11], 0.f);
      // half width along each own axis u_s: sum_k h_k |u_s . u_k| of the
      // stored float values, in double, rounded up (1 + 1e-12 covers the
      // double rounding)
      float w[3];
      for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) {
          const double dk = (double)b[3 + 3 * a] * b[3 + 3 * k] + (double)b[4 + 3 * a] * b[4 + 3 * k] +
                            (double)b[5 + 3 * a] * b[5 + 3 * k];
          acc += (double)b[12 + k] * std::fabs(dk);
        }
        acc *= 1.0 + 1e-12;
        float f = (float)acc;
        if ((double)f < acc) f = std::nextafter(f, INFINITY);
        w[a] = f;
      }
      boxw[n] = make_float4(w[0], w[1], w[2], 0.f);
    }
    std::memcpy(p + o_child, h.node_child.data(), sizeof(int32_t) * 2 * h.n_nodes);
    float* tri = (float*)(p + o_tri);
    int32_t* vid = (int32_t*)(p + o_vid);
    float4* tsph = (float4*)(p + o_tsph);
    for (int64_t s = 0; s < h.n_tri_pad; ++s) {
      for (int k = 0; k < 9; ++k) tri[12 * s + k] = h.slot_xyz[9 * s + k];
      tri[12 * s + 9] = tri[12 * s + 10] = tri[12 * s + 11] = 0.f;
      for (int k = 0; k < 3; ++k) vid[k * stride + s] = h.slot_vid[3 * s + k];
      // bounding sphere of the triangle: centroid, largest vertex distance,
      // in double and rounded up (padding slots get an empty sphere)
      const float* t = &h.slot_xyz[9 * s];
      double c[3], r2 = 0;
      for (int k = 0; k < 3; ++k) c[k] = ((double)t[k] + (double)t[3 + k] + (double)t[6 + k]) / 3.0;
      for (int v = 0; v < 3; ++v) {
        double d2 = 0;
        for (int k = 0; k < 3; ++k) d2 += ((double)t[3 * v + k] - c[k]) * ((double)t[3 * v + k] - c[k]);
        r2 = std::max(r2, d2);
      }
      tsph[s] = make_float4((float)c[0], (float)c[1], (float)c[2],
                            (float)(std::sqrt(r2) * (1.0 + 1e-6) + 1e-30));
    }
    for (int64_t s = h.n_tri_pad; s < stride; ++s) tsph[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t s = h.n_tri_pad; s < stride; ++s)
      for (int k = 0; k < 3; ++k) vid[k * stride + s] = -1;
    int32_t* st = (int32_t*)(p + o_slot);
    for (int64_t s = 0; s < stride; ++s) st[s] = s < h.n_tri_pad ? h.slot_tri[s] : -1;
    std::memcpy(p + o_ts, h.tri_slot.data(), sizeof(int32_t) * h.n_tri);
    std::memcpy(p + o_off, h.tri_off.data(), sizeof(int64_t) * (h.n_particles + 1));
    std::memcpy(p + o_root, h.root.data(), sizeof(int32_t) * h.n_particles);
    std::memcpy(p + o_br, h.bound_r.data(), sizeof(float) * h.n_particles);
    if (cudaMemcpy(base, buf.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(base);
      cudaGetLastError();
      return MRDEM_ERR_CUDA;
    }
    HierDev& d = hier->dev;
    d.node_geo = (const float4*)(base + o_geo);
    d.node_child = (const int2*)(base + o_child);
    d.tri = (const float4*)(base + o_tri);
    d.vid = (const int32_t*)(base + o_vid);
    d.slot_tri = (const int32_t*)(base + o_slot);
    d.tri_slot = (const int32_t*)(base + o_ts);
    d.tri_off = (const int64_t*)(base + o_off);
    d.root = (const int32_t*)(base + o_root);
    d.node_up = (const int2*)(base + o_up);
    d.n_nodes = h.n_nodes;
    d.bound_r = (const float*)(base + o_br);
    d.node_sph = (const float4*)(base + o_sph);
    d.node_nrm = (const float4*)(base + o_nrm);
    d.tri_sph = (const float4*)(base + o_tsph);
    d.node_box = (const float4*)(base + o_box);
    d.node_boxw = (const float4*)(base + o_boxw);
    d.stride = stride;
    d.n_tri = h.n_tri;
    d.n_particles = h.n_particles;
  } catch (const std::bad_alloc&) {
    cudaFree(base);
    return MRDEM_ERR_OOM;
  }
  hier->d_mem = base;
  hier->ctx = c;
  return MRDEM_OK;
}

int mrdem_build_hierarchy(mrdem_ctx* c, int32_t n, const int64_t* vert_off, const float* verts,
                          const int64_t* tri_off, const int32_t* tris, mrdem_hier** out) {
  if (!c || !out) return MRDEM_ERR_INVALID;
  int st = mrdem_build_hierarchy_host(&c->params, n, vert_off, verts, tri_off, tris, out);
  if (st != MRDEM_OK) return st;
  st = mrdem_hier_upload(c, *out);
  if (st != MRDEM_OK) {
    mrdem_hier_destroy(*out);
    *out = nullptr;
  }
  return st;
}

int mrdem_build_hierarchy_device(mrdem_ctx* c, int32_t n, const int64_t* vert_off,
                                 const float* verts, const int64_t* tri_off, const int32_t* tris,
                                 mrdem_hier** out, double* build_ms) {
  if (!c || !out) return MRDEM_ERR_INVALID;
  *out = nullptr;
  DeviceGuard g(c->device);
  mrdem_hier* hh = new (std::nothrow) mrdem_hier();
  if (!hh) return MRDEM_ERR_OOM;
  int st = build_hierarchy_device(c->params, n, vert_off, verts, tri_off, tris, &hh->h, build_ms);
  if (st == MRDEM_OK) st = mrdem_hier_upload(c, hh);
  if (st != MRDEM_OK) {
    mrdem_hier_destroy(hh);
    return st;
  }
  *out = hh;
  return MRDEM_OK;
}

int mrdem_hier_destroy(mrdem_hier* h) {
  if (!h) return MRDEM_OK;
  if (h->d_mem) {
    DeviceGuard g(h->ctx ? h->ctx->device : 0);
    cudaFree(h->d_mem);
  }
  delete h;
  return MRDEM_OK;
}

int mrdem_hier_get_info(const mrdem_hier* hier, mrdem_hier_info* out) {
  if (!hier || !out) return MRDEM_ERR_INVALID;
  const HierHost& h = hier->h;
  out->n_particles = h.n_particles;
  out->max_depth = h.max_depth;
  out->n_nodes = h.n_nodes;
  out->n_tri = h.n_tri;
  out->n_tri_pad = h.n_tri_pad;
  out->n_verts = h.n_verts;
  return MRDEM_OK;
}

int mrdem_hier_export(const mrdem_hier* hier, float* node_tri, float* node_delta,
                      int32_t* node_child, int32_t* node_level, int32_t* root, int32_t* slot_tri,
                      int32_t* slot_particle) {
  if (!hier) return MRDEM_ERR_INVALID;
  const HierHost& h = hier->h;
  if (node_tri) std::copy(h.node_tri.begin(), h.node_tri.end(), node_tri);
  if (node_delta) std::copy(h.node_delta.begin(), h.node_delta.end(), node_delta);
  if (node_child) std::copy(h.node_child.begin(), h.node_child.end(), node_child);
  if (node_level) std::copy(h.node_level.begin(), h.node_level.end(), node_level);
  if (root) std::copy(h.root.begin(), h.root.end(), root);
  if (slot_tri) std::copy(h.slot_tri.begin(), h.slot_tri.end(), slot_tri);
  if (slot_particle) std::copy(h.slot_particle.begin(), h.slot_particle.end(), slot_particle);
  return MRDEM_OK;
}

int mrdem_hier_export_boxes(const mrdem_hier* hier, float* node_box) {
  if (!hier || !node_box) return MRDEM_ERR_INVALID;
  std::copy(hier->h.node_box.begin(), hier->h.node_box.end(), node_box);
  return MRDEM_OK;
}

static int check_pair_args(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                           const double* eps, const double* poses) {
  if (!c || !h || n_pairs < 0 || n_pairs >= (int64_t)1 << 31) return MRDEM_ERR_INVALID;
  if (h->ctx != c || !h->d_mem) return MRDEM_ERR_INVALID;
  if (n_pairs > 0 && (!ab || !eps || !poses)) return MRDEM_ERR_INVALID;
  return MRDEM_OK;
}

int mrdem_detect(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                 const double* eps, const double* poses, int32_t precision,
                 const mrdem_contacts* out, int64_t* stats, mrdem_stream s) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!contacts_ok(out) || (precision != MRDEM_PREC_FP32 && precision != MRDEM_PREC_FP64))
    return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_detect(c, h, n_pairs, ab, eps, poses, precision, out, stats, (cudaStream_t)s);
}

int mrdem_autotune(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                   const double* eps, const double* poses, int32_t precision,
                   const mrdem_contacts* out, int32_t reps, int32_t* chosen, double* ms) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!contacts_ok(out) || (precision != MRDEM_PREC_FP32 && precision != MRDEM_PREC_FP64) ||
      reps < 1 || reps > 1000 || n_pairs < 1)
    return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return autotune(c, h, n_pairs, ab, eps, poses, precision, out, reps, chosen, ms);
}

static int decode_status(const unsigned long long* st, int64_t* required) {
  if (required) {
    required[0] = (int64_t)st[ST_REQ_LEVEL];
    required[1] = (int64_t)st[ST_REQ_TILES];
    required[2] = (int64_t)st[ST_REQ_CANDS];
    required[3] = (int64_t)st[ST_REQ_CONTACTS];
    required[4] = (int64_t)st[ST_REQ_SWEEP];
  }
  if (st[ST_NONFINITE]) return MRDEM_ERR_NONFINITE;
  if (st[ST_REQ_LEVEL] || st[ST_REQ_TILES] || st[ST_REQ_CANDS] || st[ST_REQ_CONTACTS] ||
      st[ST_REQ_SWEEP] || st[ST_REQ_ACTIVE])
    return MRDEM_ERR_CAPACITY;
  return MRDEM_OK;
}

int mrdem_check(mrdem_ctx* c, mrdem_stream s, int64_t* required) {
  if (!c) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  unsigned long long st[ST_TOTAL];
  if (cudaStreamSynchronize((cudaStream_t)s) != cudaSuccess ||
      cudaMemcpy(st, c->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(st)) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  return decode_status(st, required);
}

int mrdem_status_async(mrdem_ctx* c, uint64_t* host_words, mrdem_stream s) {
  static_assert(MRDEM_STATUS_WORDS == ST_TOTAL, "status words");
  if (!c || !host_words) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  const size_t bytes = sizeof(unsigned long long) * ST_TOTAL;
  if (cudaMemcpyAsync(host_words, c->status, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)s) !=
          cudaSuccess ||
      cudaMemsetAsync(c->status, 0, bytes, (cudaStream_t)s) != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  return MRDEM_OK;
}

int mrdem_status_decode(const uint64_t* host_words, int64_t* required) {
  if (!host_words) return MRDEM_ERR_INVALID;
  return decode_status(reinterpret_cast<const unsigned long long*>(host_words), required);
}

int mrdem_contact_forces(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                         const double* eps, const double* poses, const mrdem_contacts* con,
                         const double* mass, const double* com, double k_s, double* ft,
                         double* energy, mrdem_stream s) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!contacts_ok(con) || !mass || !com || !(k_s >= 0)) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_forces(c, h, n_pairs, ab, eps, poses, con, mass, com, k_s, ft, energy,
                       (cudaStream_t)s);
}

int mrdem_contact_grad(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                       const double* eps, const double* poses, const mrdem_contacts* con,
                       const double* mass, double k_s, double scale, float* dverts,
                       double* dpose, double* jac, mrdem_stream s) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!contacts_ok(con) || !mass || !(k_s >= 0)) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_grad(c, h, n_pairs, ab, eps, poses, con, mass, k_s, scale, dverts, dpose, jac,
                     (cudaStream_t)s);
}

int mrdem_detect_plain_fp64(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                            const double* eps, const double* poses, const mrdem_contacts* out,
                            mrdem_stream s) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!contacts_ok(out)) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_plain(c, h, n_pairs, ab, eps, poses, out, (cudaStream_t)s);
}

int mrdem_triangle_distance(mrdem_ctx* c, int64_t n, const double* P, const double* Q,
                            const double* eps, int32_t precision, double* dist, double* pa,
                            double* pb, int32_t* feature, float* sx, float* sgap, int32_t* sconv,
                            mrdem_stream s) {
  if (!c || n < 0 || n >= (int64_t)1 << 40) return MRDEM_ERR_INVALID;
  if (n > 0 && (!P || !Q || !eps)) return MRDEM_ERR_INVALID;
  if (precision != MRDEM_PREC_FP32 && precision != MRDEM_PREC_FP64) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_triangle_distance(c, n, P, Q, eps, precision, dist, pa, pb, feature, sx, sgap,
                                  sconv, (cudaStream_t)s);
}

int mrdem_merge_contacts(mrdem_ctx* c, int64_t n_pairs, const double* eps,
                         const mrdem_contacts* in, const mrdem_contacts* out, int32_t* members,
                         mrdem_stream s) {
  if (!c || n_pairs < 0 || n_pairs >= (int64_t)1 << 31) return MRDEM_ERR_INVALID;
  if (!contacts_ok(in) || !contacts_ok(out) || (n_pairs > 0 && !eps)) return MRDEM_ERR_INVALID;
  if (in->capacity >= (int64_t)1 << 31 || out->capacity >= (int64_t)1 << 31)
    return MRDEM_ERR_INVALID;
  // the output buffers may not overlap the input's
  const void* ip[] = {in->count, in->pair, in->tri_a, in->tri_b, in->dist, in->point_a, in->point_b};
  const void* op[] = {out->count, out->pair, out->tri_a, out->tri_b, out->dist, out->point_a,
                      out->point_b, members};
  for (const void* a : ip)
    for (const void* b : op)
      if (a && a == b) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_merge(c, n_pairs, eps, in, out, members, (cudaStream_t)s);
}

int mrdem_broad_phase(mrdem_ctx* c, int32_t n, const double* poses, const double* bound,
                      const double* radius, double eps_rel, int32_t* pairs, double* pair_eps,
                      int64_t cap, int64_t* count, mrdem_stream s) {
  if (!c || n < 0 || n > ((int32_t)1 << 26) || !count || cap < 0 || cap >= (int64_t)1 << 31)
    return MRDEM_ERR_INVALID;
  if (!(eps_rel >= 0.0) || !std::isfinite(eps_rel)) return MRDEM_ERR_INVALID;
  if (n > 0 && (!poses || !bound || !radius)) return MRDEM_ERR_INVALID;
  if (cap > 0 && (!pairs || !pair_eps)) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_broad_phase(c, n, poses, bound, radius, eps_rel, pairs, pair_eps, cap, count,
                            (cudaStream_t)s);
}

int mrdem_move_poses(mrdem_ctx* c, int32_t n, const double* poses0, const double* vel, double dt,
                     double* poses, mrdem_stream s) {
  if (!c || n < 0 || !std::isfinite(dt)) return MRDEM_ERR_INVALID;
  if (n > 0 && (!poses0 || !vel || !poses)) return MRDEM_ERR_INVALID;
  if (n > 0 && (const void*)vel == (const void*)poses) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_move_poses(c, n, poses0, vel, dt, poses, (cudaStream_t)s);
}

int mrdem_twist_grad(mrdem_ctx* c, int32_t n, const double* twist, const double* grad_pose,
                     double* out, mrdem_stream s) {
  if (!c || n < 0) return MRDEM_ERR_INVALID;
  if (n > 0 && (!twist || !grad_pose || !out)) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_twist_grad(c, n, twist, grad_pose, out, (cudaStream_t)s);
}

int mrdem_picard_update(mrdem_ctx* c, int32_t n, const double* vel0, const double* force_torque,
                        const double* mass, const double* inertia, const double* gravity,
                        double dt, double* vel, double* norms, mrdem_stream s) {
  if (!c || n < 0 || !gravity || !norms || !std::isfinite(dt)) return MRDEM_ERR_INVALID;
  if (n > 0 && (!vel0 || !force_torque || !mass || !inertia || !vel)) return MRDEM_ERR_INVALID;
  if (n > 0 && (vel == vel0 || vel == force_torque)) return MRDEM_ERR_INVALID;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(gravity[k])) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_picard_update(c, n, vel0, force_torque, mass, inertia, gravity, dt, vel, norms,
                              (cudaStream_t)s);
}

int mrdem_contact_hessian(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                          const double* eps, const double* poses, const mrdem_contacts* con,
                          const double* mass, double k_s, double* blocks, int64_t* skipped,
                          mrdem_stream s) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!contacts_ok(con) || !mass || !(k_s >= 0) || !std::isfinite(k_s)) return MRDEM_ERR_INVALID;
  if (n_pairs > 0 && !blocks) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_contact_hessian(c, h, n_pairs, ab, eps, poses, con, mass, k_s, blocks, skipped,
                                (cudaStream_t)s);
}

int mrdem_newton_residual(mrdem_ctx* c, int32_t n, const double* vel0, const double* vel,
                          const double* force_torque, const double* mass, const double* inertia,
                          const double* gravity, double dt, double* res, double* norms,
                          mrdem_stream s) {
  if (!c || n < 0 || !gravity || !norms || !(dt > 0.0) || !std::isfinite(dt))
    return MRDEM_ERR_INVALID;
  if (n > 0 && (!vel0 || !vel || !force_torque || !mass || !inertia || !res))
    return MRDEM_ERR_INVALID;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(gravity[k])) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_newton_residual(c, n, vel0, vel, force_torque, mass, inertia, gravity, dt, res,
                                norms, (cudaStream_t)s);
}

int mrdem_newton_solve(mrdem_ctx* c, int32_t n, int64_t n_pairs, const int32_t* ab,
                       const double* blocks, const double* mass, const double* inertia, double dt,
                       const double* rhs, double* x, int32_t max_iter, double rel_tol,
                       int32_t check_every, double* info, mrdem_stream s) {
  if (!c || n < 0 || n > ((int32_t)1 << 26) || n_pairs < 0 || n_pairs >= (int64_t)1 << 31 ||
      !info || !(dt > 0.0) || !std::isfinite(dt) || max_iter < 0 || max_iter > 100000 ||
      !(rel_tol >= 0.0) || !std::isfinite(rel_tol) || check_every < 0)
    return MRDEM_ERR_INVALID;
  if (n > 0 && (!mass || !inertia || !rhs || !x)) return MRDEM_ERR_INVALID;
  if (n_pairs > 0 && (!ab || !blocks)) return MRDEM_ERR_INVALID;
  if (n > 0 && (const void*)rhs == (const void*)x) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_newton_solve(c, n, n_pairs, ab, blocks, mass, inertia, dt, rhs, x, max_iter,
                             rel_tol, check_every, info, (cudaStream_t)s);
}

int mrdem_vel_axpy(mrdem_ctx* c, int64_t m, double a, const double* x, const double* y,
                   double* out, mrdem_stream s) {
  if (!c || m < 0 || !std::isfinite(a)) return MRDEM_ERR_INVALID;
  if (m > 0 && (!x || !y || !out)) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_vel_axpy(c, m, a, x, y, out, (cudaStream_t)s);
}

int mrdem_refine_contacts(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                          const double* eps, const double* poses, const mrdem_contacts* cand,
                          const mrdem_contacts* out, mrdem_stream s) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!contacts_ok(cand) || !contacts_ok(out)) return MRDEM_ERR_INVALID;
  if (cand->capacity >= (int64_t)1 << 31 || out->capacity >= (int64_t)1 << 31)
    return MRDEM_ERR_INVALID;
  const void* ip[] = {cand->count, cand->pair, cand->tri_a, cand->tri_b, cand->dist,
                      cand->point_a, cand->point_b};
  const void* op[] = {out->count, out->pair, out->tri_a, out->tri_b, out->dist, out->point_a,
                      out->point_b};
  for (const void* a : ip)
    for (const void* b : op)
      if (a && a == b) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_refine_contacts(c, h, n_pairs, ab, eps, poses, cand, out, (cudaStream_t)s);
}

int mrdem_motion_bound(mrdem_ctx* c, int32_t n, const double* poses_ref, const double* poses,
                       const double* bound, double* out, mrdem_stream s) {
  if (!c || n < 0 || !out) return MRDEM_ERR_INVALID;
  if (n > 0 && (!poses_ref || !poses || !bound)) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_motion_bound(c, n, poses_ref, poses, bound, out, (cudaStream_t)s);
}

static bool active_ok(const mrdem_active_set* a) {
  return a && a->count && a->capacity >= 0 && a->capacity < ((int64_t)1 << 31) &&
         (a->capacity == 0 || (a->item && ((uintptr_t)a->item & 15) == 0));
}

int mrdem_active_set_init(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs,
                          const int32_t* ab, const mrdem_active_set* out, mrdem_stream s) {
  if (!c || !h || h->ctx != c || !h->d_mem || n_pairs < 0 || !active_ok(out) ||
      out->capacity < n_pairs || (n_pairs > 0 && !ab))
    return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_active_init(c, h, n_pairs, ab, out, (cudaStream_t)s);
}

int mrdem_active_set_step(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                          const double* eps, const double* poses, int precision,
                          const mrdem_active_set* in, const mrdem_active_set* out,
                          const mrdem_contacts* contacts, const mrdem_contacts* sur,
                          int64_t* counts, mrdem_stream s) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!active_ok(in) || !active_ok(out) || !contacts_ok(contacts) || !contacts_ok(sur) ||
      (precision != MRDEM_PREC_FP32 && precision != MRDEM_PREC_FP64))
    return MRDEM_ERR_INVALID;
  if (in->item == out->item || in->count == out->count || contacts->count == sur->count ||
      (contacts->pair && contacts->pair == sur->pair))
    return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_active_step(c, h, n_pairs, ab, eps, poses, precision, in, out, contacts, sur,
                            counts, (cudaStream_t)s);
}

int mrdem_surrogate_forces(mrdem_ctx* c, const mrdem_hier* h, int64_t n_pairs, const int32_t* ab,
                           const double* eps, const double* poses, const mrdem_contacts* sur,
                           const double* mass, const double* com, double k_s, double weight,
                           double* ft, double* energy, mrdem_stream s) {
  int st = check_pair_args(c, h, n_pairs, ab, eps, poses);
  if (st) return st;
  if (!contacts_ok(sur) || !mass || !com || !ft || !(k_s >= 0) || !(weight >= 0) ||
      !(weight <= 1))
    return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  return launch_surrogate_forces(c, h, n_pairs, ab, eps, poses, sur, mass, com, k_s, weight, ft,
                                 energy, (cudaStream_t)s);
}

static const char* kKernelNames[K_COUNT] = {
    "k_setup", "k_expand", "k_sweep_nodes", "k_tile",  "k_sweep_fine", "k_exact",
    "k_exact64", "k_forces", "k_grad",       "k_plain", "k_tridist", "k_sort",
    "k_merge", "k_broad", "k_step", "k_hessian", "k_cg"};

int mrdem_profile(mrdem_ctx* c, int32_t enable) {
  if (!c) return MRDEM_ERR_INVALID;
  c->prof = enable != 0;
  return MRDEM_OK;
}

int mrdem_profile_read(mrdem_ctx* c, int32_t n_max, const char** names, double* ms,
                       int64_t* launches, int32_t* n_out) {
  if (!c || n_max < 0) return MRDEM_ERR_INVALID;
  DeviceGuard g(c->device);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return MRDEM_ERR_CUDA;
  }
  double tot[K_COUNT] = {0};
  int64_t cnt[K_COUNT] = {0};
  for (auto& r : c->prof_recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      tot[r.kernel] += t;
      cnt[r.kernel] += 1;
    }
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  cudaGetLastError();
  c->prof_recs.clear();
  int n = 0;
  for (int k = 0; k < K_COUNT && n < n_max; ++k) {
    if (!cnt[k]) continue;
    if (names) names[n] = kKernelNames[k];
    if (ms) ms[n] = tot[k];
    if (launches) launches[n] = cnt[k];
    ++n;
  }
  if (n_out) *n_out = n;
  return MRDEM_OK;
}

}  // extern "C"
