"""PyTorch-facing wrappers over the C ABI (memory, streams, autograd).

Every step of the detection, the forces and the adjoint runs in libmrdem's
CUDA kernels; this module only allocates torch tensors, passes pointers and
the current CUDA stream, and grows buffers when the library reports that a
work list overflowed.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

PRECISION = {"fp32": L.MRDEM_PREC_FP32, "fp64": L.MRDEM_PREC_FP64}


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return C.c_void_p(a.ctypes.data)


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _need(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class Context:
    """A library context on one CUDA device (owns the device work lists)."""

    def __init__(self, device: int = 0, params: L.mrdem_params | None = None, **overrides):
        lib = L.load()
        p = params if params is not None else L.default_params()
        for k, v in overrides.items():
            setattr(p, k, v)
        h = C.c_void_p()
        L.check(lib.mrdem_create(C.byref(h), int(device), C.byref(p)), "mrdem_create")
        self.handle = h
        self.device = int(device)

    @property
    def params(self) -> L.mrdem_params:
        p = L.mrdem_params()
        L.check(L.load().mrdem_get_params(self.handle, C.byref(p)), "mrdem_get_params")
        return p

    def set_params(self, **kw):
        p = self.params
        for k, v in kw.items():
            setattr(p, k, v)
        L.check(L.load().mrdem_set_params(self.handle, C.byref(p)), "mrdem_set_params")

    def reserve(self, cap_level=0, cap_tiles=0, cap_candidates=0, cap_sweep=0):
        L.check(L.load().mrdem_reserve(self.handle, int(cap_level), int(cap_tiles),
                                       int(cap_candidates), int(cap_sweep)), "mrdem_reserve")

    def profile(self, enable: bool):
        L.check(L.load().mrdem_profile(self.handle, int(bool(enable))), "mrdem_profile")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the previous read."""
        n_max = 16
        names = (C.c_char_p * n_max)()
        ms = np.zeros(n_max)
        cnt = np.zeros(n_max, np.int64)
        n = C.c_int32()
        L.check(L.load().mrdem_profile_read(self.handle, n_max, names, _np_ptr(ms), _np_ptr(cnt),
                                            C.byref(n)), "mrdem_profile_read")
        return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(n.value)}

    def close(self):
        if getattr(self, "handle", None):
            L.load().mrdem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """Surrogate trees of a set of particle meshes (host arrays, optionally on a device)."""

    def __init__(self, handle, keep=None):
        self.handle = handle
        self._keep = keep

    @staticmethod
    def _arrays(vert_off, verts, tri_off, tris):
        vo = np.ascontiguousarray(vert_off, np.int64)
        v = np.ascontiguousarray(verts, np.float32)
        to = np.ascontiguousarray(tri_off, np.int64)
        t = np.ascontiguousarray(tris, np.int32)
        return vo, v, to, t

    @classmethod
    def build_host(cls, vert_off, verts, tri_off, tris, params: L.mrdem_params | None = None):
        vo, v, to, t = cls._arrays(vert_off, verts, tri_off, tris)
        h = C.c_void_p()
        p = params if params is not None else L.default_params()
        L.check(L.load().mrdem_build_hierarchy_host(C.byref(p), len(vo) - 1, _np_ptr(vo), _np_ptr(v),
                                                   _np_ptr(to), _np_ptr(t), C.byref(h)),
                "mrdem_build_hierarchy_host")
        return cls(h)

    @classmethod
    def build(cls, ctx: Context, vert_off, verts, tri_off, tris):
        vo, v, to, t = cls._arrays(vert_off, verts, tri_off, tris)
        h = C.c_void_p()
        L.check(L.load().mrdem_build_hierarchy(ctx.handle, len(vo) - 1, _np_ptr(vo), _np_ptr(v),
                                              _np_ptr(to), _np_ptr(t), C.byref(h)),
                "mrdem_build_hierarchy")
        return cls(h, keep=ctx)

    @classmethod
    def build_device(cls, ctx: Context, vert_off, verts, tri_off, tris):
        """Trees built on ctx's GPU (mrdem_build_hierarchy_device).  verts
        (float32 [nv, 3]) and tris (int32 [nt, 3], local indices) are device
        tensors; the offsets are host arrays.  Returns the hierarchy; its
        build_ms attribute is the device part's time."""
        vo = np.ascontiguousarray(vert_off, np.int64)
        to = np.ascontiguousarray(tri_off, np.int64)
        _need(verts, torch.float32, (int(vo[-1]), 3), "verts")
        _need(tris, torch.int32, (int(to[-1]), 3), "tris")
        h = C.c_void_p()
        ms = C.c_double()
        L.check(L.load().mrdem_build_hierarchy_device(ctx.handle, len(vo) - 1, _np_ptr(vo), _p(verts),
                                                     _np_ptr(to), _p(tris), C.byref(h),
                                                     C.byref(ms)),
                "mrdem_build_hierarchy_device")
        out = cls(h, keep=ctx)
        out.build_ms = ms.value
        return out

    @classmethod
    def from_scene_device(cls, ctx: Context, scene):
        dev = torch.device("cuda", ctx.device)
        verts = torch.as_tensor(np.ascontiguousarray(scene.verts, np.float32), device=dev)
        tris = torch.as_tensor(np.ascontiguousarray(scene.tris, np.int32), device=dev)
        return cls.build_device(ctx, scene.vert_off, verts, scene.tri_off, tris)

    @classmethod
    def from_scene(cls, ctx: Context | None, scene, params=None):
        if ctx is None:
            return cls.build_host(scene.vert_off, scene.verts, scene.tri_off, scene.tris, params)
        return cls.build(ctx, scene.vert_off, scene.verts, scene.tri_off, scene.tris)

    def upload(self, ctx: Context):
        L.check(L.load().mrdem_hier_upload(ctx.handle, self.handle), "mrdem_hier_upload")
        self._keep = ctx

    def info(self) -> dict:
        i = L.mrdem_hier_info()
        L.check(L.load().mrdem_hier_get_info(self.handle, C.byref(i)), "mrdem_hier_get_info")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def export(self) -> dict:
        i = self.info()
        nn, ns, n = i["n_nodes"], i["n_tri_pad"], i["n_particles"]
        out = dict(node_tri=np.empty((nn, 9), np.float32), node_delta=np.empty(nn, np.float32),
                   node_child=np.empty((nn, 2), np.int32), node_level=np.empty(nn, np.int32),
                   root=np.empty(n, np.int32), slot_tri=np.empty(ns, np.int32),
                   slot_particle=np.empty(ns, np.int32))
        L.check(L.load().mrdem_hier_export(self.handle, *[_np_ptr(out[k]) for k in (
            "node_tri", "node_delta", "node_child", "node_level", "root", "slot_tri",
            "slot_particle")]), "mrdem_hier_export")
        out["node_box"] = np.empty((nn, 16), np.float32)
        L.check(L.load().mrdem_hier_export_boxes(self.handle, _np_ptr(out["node_box"])),
                "mrdem_hier_export_boxes")
        return out

    def close(self):
        if getattr(self, "handle", None):
            L.load().mrdem_hier_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Contacts:
    """Caller-owned contact buffers on the device."""

    def __init__(self, capacity: int, device):
        self.device = torch.device(device)
        self.count = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.resize(capacity)

    def resize(self, capacity: int):
        capacity = max(int(capacity), 1)
        d = self.device
        self.capacity = capacity
        self.pair = torch.empty(capacity, dtype=torch.int32, device=d)
        self.tri_a = torch.empty(capacity, dtype=torch.int32, device=d)
        self.tri_b = torch.empty(capacity, dtype=torch.int32, device=d)
        self.dist = torch.empty(capacity, dtype=torch.float64, device=d)
        self.point_a = torch.empty((capacity, 3), dtype=torch.float64, device=d)
        self.point_b = torch.empty((capacity, 3), dtype=torch.float64, device=d)

    def struct(self) -> L.mrdem_contacts:
        return L.mrdem_contacts(self.capacity, self.count.data_ptr(), self.pair.data_ptr(),
                                self.tri_a.data_ptr(), self.tri_b.data_ptr(), self.dist.data_ptr(),
                                self.point_a.data_ptr(), self.point_b.data_ptr())

    def n(self) -> int:
        return min(int(self.count.item()), self.capacity)

    def to_numpy(self, sort=True) -> dict:
        n = self.n()
        out = dict(pair=self.pair[:n].cpu().numpy(), ta=self.tri_a[:n].cpu().numpy(),
                   tb=self.tri_b[:n].cpu().numpy(), d=self.dist[:n].cpu().numpy(),
                   pa=self.point_a[:n].cpu().numpy(), pb=self.point_b[:n].cpu().numpy())
        if sort:
            o = np.lexsort((out["tb"], out["ta"], out["pair"]))
            out = {k: v[o] for k, v in out.items()}
        return out


def _pair_args(hier, pairs, eps, poses, n_particles):
    P = pairs.shape[0]
    _need(pairs, torch.int32, (P, 2), "pairs")
    _need(eps, torch.float64, (P,), "eps")
    _need(poses, torch.float64, (n_particles, 7), "poses")
    return P


def detect(ctx: Context, hier: Hierarchy, pairs, eps, poses, precision="fp32", contacts=None,
           stats=None, check=True, stream=None, max_retries=4):
    """Contact set of every pair (Algorithm 5).  With check=True the call
    synchronises, grows overflowing buffers and repeats (so it is not
    capturable); with check=False it only enqueues work."""
    info = hier.info()
    P = _pair_args(hier, pairs, eps, poses, info["n_particles"])
    if contacts is None:
        contacts = Contacts(max(1024, 64 * P), pairs.device)
    if stats is None:
        stats = torch.zeros(L.MRDEM_STAT_COUNT, dtype=torch.int64, device=pairs.device)
    lib = L.load()
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    for _ in range(max_retries + 1):
        cs = contacts.struct()
        L.check(lib.mrdem_detect(ctx.handle, hier.handle, P, _p(pairs), _p(eps), _p(poses), prec,
                                 C.byref(cs), _p(stats), _stream(stream)), "mrdem_detect")
        if not check:
            return contacts, stats
        req = np.zeros(5, np.int64)
        st = lib.mrdem_check(ctx.handle, _stream(stream), _np_ptr(req))
        if st == L.MRDEM_OK:
            return contacts, stats
        if st != L.MRDEM_ERR_CAPACITY:
            L.check(st, "mrdem_detect")
        prm = ctx.params
        grow = lambda need, cap: int(need * 1.25) + 1024 if need > cap else 0  # noqa: E731
        lv, ti, ca = grow(req[0], prm.cap_level), grow(req[1], prm.cap_tiles), grow(req[2], prm.cap_candidates)
        sw = grow(req[4], prm.cap_sweep)
        if lv or ti or ca or sw:
            ctx.reserve(lv, ti, ca, sw)
        if req[3] > contacts.capacity:
            contacts.resize(int(req[3] * 1.25) + 1024)
    raise L.MrdemError(L.MRDEM_ERR_CAPACITY, "mrdem_detect (retries exhausted)")


TUNED_FIELDS = ("level_warps", "expand_items", "node_threads", "tile_warps", "sweep_warps",
                "exact_threads", "level_kernel")


def autotune(ctx: Context, hier: Hierarchy, pairs, eps, poses, precision="fp32", contacts=None,
             reps=3):
    """Pick the detection kernels' launch shapes for this GPU and this batch's
    size class (mrdem_autotune); later detections of that size class use
    them.  A checked detection runs first, so the lists are large enough.
    Returns {"chosen": {field: value}, "ms_default": t0, "ms_tuned": t1}."""
    contacts, _ = detect(ctx, hier, pairs, eps, poses, precision, contacts=contacts)
    P = _pair_args(hier, pairs, eps, poses, hier.info()["n_particles"])
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    chosen = np.zeros(len(TUNED_FIELDS), np.int32)
    ms = np.zeros(2)
    cs = contacts.struct()
    L.check(L.load().mrdem_autotune(ctx.handle, hier.handle, P, _p(pairs), _p(eps), _p(poses), prec,
                                    C.byref(cs), int(reps), _np_ptr(chosen), _np_ptr(ms)),
            "mrdem_autotune")
    return {"chosen": dict(zip(TUNED_FIELDS, (int(v) for v in chosen))),
            "ms_default": float(ms[0]), "ms_tuned": float(ms[1])}


def detect_plain_fp64(ctx, hier, pairs, eps, poses, contacts=None, stream=None):
    """The plain GPU form: FP64 brute force, one launch per pair (baseline)."""
    info = hier.info()
    P = _pair_args(hier, pairs, eps, poses, info["n_particles"])
    if contacts is None:
        contacts = Contacts(max(1024, 64 * P), pairs.device)
    lib = L.load()
    for _ in range(4):
        cs = contacts.struct()
        L.check(lib.mrdem_detect_plain_fp64(ctx.handle, hier.handle, P, _p(pairs), _p(eps),
                                            _p(poses), C.byref(cs), _stream(stream)),
                "mrdem_detect_plain_fp64")
        req = np.zeros(5, np.int64)
        st = lib.mrdem_check(ctx.handle, _stream(stream), _np_ptr(req))
        if st == L.MRDEM_OK:
            return contacts
        if st != L.MRDEM_ERR_CAPACITY:
            L.check(st, "mrdem_detect_plain_fp64")
        contacts.resize(int(req[3] * 1.25) + 1024)
    raise L.MrdemError(L.MRDEM_ERR_CAPACITY, "mrdem_detect_plain_fp64")


def merge_contacts(ctx: Context, eps, contacts: Contacts, out: Contacts | None = None,
                   members=None, check=True, stream=None, max_retries=4):
    """Redundant-contact merge (Sec. 2): per pair, contacts whose contact
    points lie closer than the pair's eps, taken transitively, become one
    contact at their mean points.  Returns (merged contacts, members): the
    list grouped by pair and ordered by the representatives' (tri_a, tri_b),
    and per entry the number of contacts merged into it (int32).  With
    check=True the call synchronises, grows an overflowing output and
    repeats; with check=False it only enqueues work."""
    P = eps.shape[0]
    _need(eps, torch.float64, (P,), "eps")
    if out is None:
        out = Contacts(max(1024, contacts.capacity), contacts.device)
    lib = L.load()
    for _ in range(max_retries + 1):
        if members is None or members.shape[0] < out.capacity:
            members = torch.empty(out.capacity, dtype=torch.int32, device=out.device)
        cin, cout = contacts.struct(), out.struct()
        L.check(lib.mrdem_merge_contacts(ctx.handle, P, _p(eps), C.byref(cin), C.byref(cout),
                                         _p(members), _stream(stream)), "mrdem_merge_contacts")
        if not check:
            return out, members
        req = np.zeros(5, np.int64)
        st = lib.mrdem_check(ctx.handle, _stream(stream), _np_ptr(req))
        if st == L.MRDEM_OK:
            return out, members
        if st != L.MRDEM_ERR_CAPACITY:
            L.check(st, "mrdem_merge_contacts")
        out.resize(int(req[3] * 1.25) + 1024)
    raise L.MrdemError(L.MRDEM_ERR_CAPACITY, "mrdem_merge_contacts (retries exhausted)")


def contact_forces(ctx, hier, pairs, eps, poses, contacts, mass, com, k_s=1000.0, force_torque=None,
                   energy=None, stream=None):
    n = hier.info()["n_particles"]
    P = _pair_args(hier, pairs, eps, poses, n)
    _need(mass, torch.float64, (n,), "mass")
    _need(com, torch.float64, (n, 3), "com")
    if force_torque is None:
        force_torque = torch.zeros((n, 6), dtype=torch.float64, device=pairs.device)
    if energy is None:
        energy = torch.zeros(1, dtype=torch.float64, device=pairs.device)
    cs = contacts.struct()
    L.check(L.load().mrdem_contact_forces(ctx.handle, hier.handle, P, _p(pairs), _p(eps), _p(poses),
                                          C.byref(cs), _p(mass), _p(com), float(k_s),
                                          _p(force_torque), _p(energy), _stream(stream)),
            "mrdem_contact_forces")
    return force_torque, energy


def contact_grad(ctx, hier, pairs, eps, poses, contacts, mass, k_s=1000.0, scale=1.0,
                 want_verts=True, want_pose=True, want_jac=False, stream=None):
    info = hier.info()
    n = info["n_particles"]
    P = _pair_args(hier, pairs, eps, poses, n)
    _need(mass, torch.float64, (n,), "mass")
    d = pairs.device
    gv = torch.zeros((info["n_verts"], 3), dtype=torch.float32, device=d) if want_verts else None
    gp = torch.zeros((n, 6), dtype=torch.float64, device=d) if want_pose else None
    jac = torch.zeros((P, 12, 12), dtype=torch.float64, device=d) if want_jac else None
    cs = contacts.struct()
    L.check(L.load().mrdem_contact_grad(ctx.handle, hier.handle, P, _p(pairs), _p(eps), _p(poses),
                                        C.byref(cs), _p(mass), float(k_s), float(scale), _p(gv),
                                        _p(gp), _p(jac), _stream(stream)), "mrdem_contact_grad")
    return gv, gp, jac


def triangle_distance(ctx, P, Q, eps, precision="fp64", sweep=True, stream=None):
    """Exact distance (and the float sweep diagnostics) of explicit triangle pairs."""
    n = P.shape[0]
    _need(P, torch.float64, (n, 9), "P")
    _need(Q, torch.float64, (n, 9), "Q")
    _need(eps, torch.float64, (n,), "eps")
    d = P.device
    out = dict(d=torch.empty(n, dtype=torch.float64, device=d),
               pa=torch.empty((n, 3), dtype=torch.float64, device=d),
               pb=torch.empty((n, 3), dtype=torch.float64, device=d),
               feature=torch.empty(n, dtype=torch.int32, device=d))
    if sweep:
        out.update(x=torch.empty((n, 4), dtype=torch.float32, device=d),
                   gap=torch.empty(n, dtype=torch.float32, device=d),
                   converged=torch.empty(n, dtype=torch.int32, device=d))
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    L.check(L.load().mrdem_triangle_distance(ctx.handle, n, _p(P), _p(Q), _p(eps), prec,
                                             _p(out["d"]), _p(out["pa"]), _p(out["pb"]),
                                             _p(out["feature"]), _p(out.get("x")),
                                             _p(out.get("gap")), _p(out.get("converged")),
                                             _stream(stream)), "mrdem_triangle_distance")
    return out


def contact_hessian(ctx, hier, pairs, eps, poses, contacts, mass, k_s=1000.0, blocks=None,
                    stream=None):
    """Per pair, the 12x12 second derivatives of its contacts' energy in the
    two pose twists (closest points free).  Returns (blocks float64
    [P, 12, 12], skipped: device int64 count of contacts between parallel
    features)."""
    n = hier.info()["n_particles"]
    P = _pair_args(hier, pairs, eps, poses, n)
    _need(mass, torch.float64, (n,), "mass")
    if blocks is None:
        blocks = torch.zeros((P, 12, 12), dtype=torch.float64, device=pairs.device)
    _need(blocks, torch.float64, (P, 12, 12), "blocks")
    skipped = torch.zeros(1, dtype=torch.int64, device=pairs.device)
    cs = contacts.struct()
    L.check(L.load().mrdem_contact_hessian(ctx.handle, hier.handle, P, _p(pairs), _p(eps),
                                           _p(poses), C.byref(cs), _p(mass), float(k_s),
                                           _p(blocks), _p(skipped), _stream(stream)),
            "mrdem_contact_hessian")
    return blocks, skipped


# ---- implicit time step (Algorithm 3)

G_DEFAULT = (0.0, 0.0, -9.81)


def broad_phase(ctx: Context, poses, bound, radius, eps_rel=0.01, cap=None, stream=None,
                max_retries=4):
    """Candidate particle pairs of a many-particle scene (uniform-grid broad
    phase): every i < j with |c_i - c_j| <= R_i + R_j + 2 eps_ij,
    eps_ij = eps_rel * 2 * min(r_i, r_j).  poses [n, 7], bound R [n] and
    radius r [n]: float64 on the device.  Returns (pairs int32 [P, 2] ordered
    by (i, j), eps float64 [P]).  Synchronises to read the count; grows the
    output and repeats when it overflows."""
    n = poses.shape[0]
    _need(poses, torch.float64, (n, 7), "poses")
    _need(bound, torch.float64, (n,), "bound")
    _need(radius, torch.float64, (n,), "radius")
    dev = poses.device
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    cap = int(cap) if cap is not None else max(1024, 16 * n)
    lib = L.load()
    for _ in range(max_retries + 1):
        pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
        eps = torch.empty(cap, dtype=torch.float64, device=dev)
        L.check(lib.mrdem_broad_phase(ctx.handle, n, _p(poses), _p(bound), _p(radius),
                                      float(eps_rel), _p(pairs), _p(eps), cap, _p(count),
                                      _stream(stream)), "mrdem_broad_phase")
        L.check(lib.mrdem_check(ctx.handle, _stream(stream), None), "mrdem_broad_phase")
        total = int(count.item())
        if total <= cap:
            return pairs[:total], eps[:total]
        cap = total
    raise L.MrdemError(L.MRDEM_ERR_CAPACITY, "mrdem_broad_phase (retries exhausted)")


def move_poses(ctx: Context, poses0, vel, dt, out=None, stream=None):
    """Poses after a step dt at velocities vel [n, 6] (v, omega; world
    frame): centre + dt v, orientation turned by the rotation vector
    dt omega (left multiplication)."""
    n = poses0.shape[0]
    _need(poses0, torch.float64, (n, 7), "poses0")
    _need(vel, torch.float64, (n, 6), "vel")
    if out is None:
        out = torch.empty_like(poses0)
    _need(out, torch.float64, (n, 7), "out")
    L.check(L.load().mrdem_move_poses(ctx.handle, n, _p(poses0), _p(vel), float(dt), _p(out),
                                      _stream(stream)), "mrdem_move_poses")
    return out


def picard_update(ctx: Context, vel0, force_torque, mass, inertia, dt, vel, norms=None,
                  gravity=G_DEFAULT, stream=None):
    """One Picard update in place: vel <- (v0 + dt (F / m + g),
    omega0 + dt tau / I).  Returns norms (device float64 [2]):
    (max |new - old|, max |new|)."""
    n = vel0.shape[0]
    for t, name in ((vel0, "vel0"), (force_torque, "force_torque"), (vel, "vel")):
        _need(t, torch.float64, (n, 6), name)
    _need(mass, torch.float64, (n,), "mass")
    _need(inertia, torch.float64, (n,), "inertia")
    if norms is None:
        norms = torch.empty(2, dtype=torch.float64, device=vel0.device)
    g = (C.c_double * 3)(*[float(x) for x in gravity])
    L.check(L.load().mrdem_picard_update(ctx.handle, n, _p(vel0), _p(force_torque), _p(mass),
                                         _p(inertia), C.cast(g, C.c_void_p), float(dt), _p(vel),
                                         _p(norms), _stream(stream)), "mrdem_picard_update")
    return norms


def refine_contacts(ctx, hier, pairs, eps, poses, candidates, out=None, stream=None,
                    max_retries=4):
    """Contacts (d <= 2 eps, exact FP64 distance) among the triangle pairs
    listed in `candidates`, at `poses`, in the list's order.  Synchronises to
    check the output's capacity; grows it and repeats on overflow."""
    n = hier.info()["n_particles"]
    P = _pair_args(hier, pairs, eps, poses, n)
    if out is None:
        out = Contacts(max(1024, candidates.capacity), pairs.device)
    lib = L.load()
    for _ in range(max_retries + 1):
        cin, cout = candidates.struct(), out.struct()
        L.check(lib.mrdem_refine_contacts(ctx.handle, hier.handle, P, _p(pairs), _p(eps),
                                          _p(poses), C.byref(cin), C.byref(cout),
                                          _stream(stream)), "mrdem_refine_contacts")
        req = np.zeros(5, np.int64)
        st = lib.mrdem_check(ctx.handle, _stream(stream), _np_ptr(req))
        if st == L.MRDEM_OK:
            return out
        if st != L.MRDEM_ERR_CAPACITY:
            L.check(st, "mrdem_refine_contacts")
        out.resize(int(req[3] * 1.25) + 1024)
    raise L.MrdemError(L.MRDEM_ERR_CAPACITY, "mrdem_refine_contacts (retries exhausted)")


def motion_bound(ctx, poses_ref, poses, bound, out=None, stream=None):
    """Largest displacement of any particle point between two poses (device
    float64 [1]): |t - t_ref| + rotation angle * bound."""
    n = poses.shape[0]
    _need(poses_ref, torch.float64, (n, 7), "poses_ref")
    _need(poses, torch.float64, (n, 7), "poses")
    _need(bound, torch.float64, (n,), "bound")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=poses.device)
    L.check(L.load().mrdem_motion_bound(ctx.handle, n, _p(poses_ref), _p(poses), _p(bound),
                                        _p(out), _stream(stream)), "mrdem_motion_bound")
    return out


class KeptCandidates:
    """Contacts at a sequence of nearby poses from one candidate list: the
    triangle pairs within 2 (eps + w) at the poses of the last detection,
    refined by exact FP64 distances at the poses asked for, and detected
    again when a point has moved more than w since (mrdem_motion_bound);
    the contact set equals a detection at eps at every call."""

    def __init__(self, ctx, hier, pairs, eps, margin, bound, precision="fp32"):
        n = hier.info()["n_particles"]
        _need(bound, torch.float64, (n,), "bound")
        self.ctx, self.hier, self.pairs, self.eps, self.bound = ctx, hier, pairs, eps, bound
        self.margin, self.precision = float(margin), precision
        self.eps_w = eps + self.margin
        self.cand = self.ref = self.motion = None
        self.stats = torch.zeros(L.MRDEM_STAT_COUNT, dtype=torch.int64, device=pairs.device)
        self.detections = 0

    def contacts(self, poses, out=None):
        fresh = self.cand is None
        if not fresh:
            self.motion = motion_bound(self.ctx, self.ref, poses, self.bound, out=self.motion)
            fresh = self.motion.item() > self.margin
        if fresh:
            self.cand, _ = detect(self.ctx, self.hier, self.pairs, self.eps_w, poses,
                                  self.precision, contacts=self.cand, stats=self.stats)
            self.ref = poses.clone()
            self.detections += 1
        return refine_contacts(self.ctx, self.hier, self.pairs, self.eps, poses, self.cand,
                               out=out)


def implicit_euler_step(ctx: Context, hier: Hierarchy, poses0, vel0, mass, inertia, pairs, eps,
                        dt, gravity=G_DEFAULT, k_s=1000.0, precision="fp32", tol=1e-13,
                        max_iter=200, contacts=None, graph=False, cache_margin=None,
                        bound=None):
    """One implicit Euler step by Picard iteration (Algorithm 3): starting
    from vel0, repeat: move the particles from poses0 by dt times the guessed
    velocities, detect the contacts of the candidate pairs there, compute the
    contact forces and torques (about the body origins), and update the
    guess; stop when max |new - guess| <= tol * max |new|.  All arithmetic
    runs in the library's kernels; the loop reads two numbers per iteration.
    With graph=True the iteration (pose update, detection, forces, velocity
    update) is captured once into a CUDA graph after a first checked
    iteration and replayed; a work-list overflow found by the per-iteration
    status check restores the velocities, runs that iteration again through
    the checked path (which grows the lists) and captures anew.
    With cache_margin = w (and bound, the particles' bounding radii) the
    candidate triangle pairs are detected once at eps + w and kept; each
    iteration checks that no point moved more than w from where the
    candidates were detected (detecting again if one did) and takes its
    contacts from the kept list by exact FP64 distances (the active set
    kept across iterations, Alg. 6's idea, with the same contact set);
    graph is then not used.
    Returns (poses, vel, iterations, history of the relative change)."""
    lib = L.load()
    n = poses0.shape[0]
    dev = poses0.device
    P = pairs.shape[0]
    vel = vel0.clone()
    prev = torch.empty_like(vel)
    poses = torch.empty_like(poses0)
    com = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    ft = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    norms = torch.empty(2, dtype=torch.float64, device=dev)
    stats = torch.zeros(L.MRDEM_STAT_COUNT, dtype=torch.int64, device=dev)
    state = {"contacts": contacts, "graph": None}

    kept = (KeptCandidates(ctx, hier, pairs, eps, cache_margin, bound, precision)
            if cache_margin is not None else None)

    def body_cached():
        move_poses(ctx, poses0, vel, dt, out=poses)
        ft.zero_()
        if P:
            state["contacts"] = kept.contacts(poses, out=state["contacts"])
            contact_forces(ctx, hier, pairs, eps, poses, state["contacts"], mass, com, k_s,
                           force_torque=ft, energy=energy)
        picard_update(ctx, vel0, ft, mass, inertia, dt, vel, norms, gravity)

    def body(checked):
        move_poses(ctx, poses0, vel, dt, out=poses)
        ft.zero_()
        if P:
            state["contacts"], _ = detect(ctx, hier, pairs, eps, poses, precision,
                                          contacts=state["contacts"], stats=stats,
                                          check=checked)
            contact_forces(ctx, hier, pairs, eps, poses, state["contacts"], mass, com, k_s,
                           force_torque=ft, energy=energy)
        picard_update(ctx, vel0, ft, mass, inertia, dt, vel, norms, gravity)

    hist = []
    it = 0
    for it in range(1, max_iter + 1):
        if cache_margin is not None:
            body_cached()
        elif not graph or it == 1:
            body(True)
        else:
            if state["graph"] is None:
                g = torch.cuda.CUDAGraph()
                side = torch.cuda.Stream()
                side.wait_stream(torch.cuda.current_stream())
                prev.copy_(vel)
                with torch.cuda.graph(g, stream=side):
                    body(False)
                torch.cuda.current_stream().wait_stream(side)
                vel.copy_(prev)   # capturing does not run the work
                state["graph"] = g
            prev.copy_(vel)
            state["graph"].replay()
            st = lib.mrdem_check(ctx.handle, _stream(None), None)
            if st == L.MRDEM_ERR_CAPACITY:
                vel.copy_(prev)
                body(True)
                state["graph"] = None
            elif st != L.MRDEM_OK:
                L.check(st, "implicit_euler_step")
        change, scale = norms.tolist()
        scale += 1e-300
        hist.append(change / scale)
        if change <= tol * scale:
            break
    move_poses(ctx, poses0, vel, dt, out=poses)
    return poses, vel, it, hist


class ActiveSets:
    """Caller-owned active sets of Algorithm 6 on the device: item
    [capacity, 4] int32 (pair, node_a, node_b, flags), count one int64
    (mrdem_active_set)."""

    def __init__(self, capacity: int, device):
        self.device = torch.device(device)
        self.count = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.resize(capacity)

    def resize(self, capacity: int):
        self.capacity = max(int(capacity), 1)
        self.item = torch.empty((self.capacity, 4), dtype=torch.int32, device=self.device)

    def struct(self) -> L.mrdem_active_set:
        return L.mrdem_active_set(self.capacity, self.count.data_ptr(), self.item.data_ptr())

    def n(self) -> int:
        return min(int(self.count.item()), self.capacity)

    def to_numpy(self):
        return self.item[:self.n()].cpu().numpy()


def active_sets_init(ctx: Context, hier: Hierarchy, pairs, out=None, stream=None):
    """The initial active sets of Algorithm 6: the two roots of every pair."""
    P = pairs.shape[0]
    _need(pairs, torch.int32, (P, 2), "pairs")
    if out is None or out.capacity < P:
        out = ActiveSets(max(1024, 16 * P), pairs.device)
    st = out.struct()
    L.check(L.load().mrdem_active_set_init(ctx.handle, hier.handle, P, _p(pairs), C.byref(st),
                                           _stream(stream)), "mrdem_active_set_init")
    return out


def active_sets_step(ctx: Context, hier: Hierarchy, pairs, eps, poses, sets_in, sets_out=None,
                     precision="fp32", contacts=None, surrogate=None, counts=None, check=True,
                     stream=None, max_retries=4):
    """One detection of Algorithm 6 on the active sets sets_in at poses: the
    fine contacts of the listed pairs of leaves, the surrogate contacts, and
    the next active sets in sets_out (widened and narrowed;
    mrdem_active_set_step).  counts: int64 [4] on the device (items widened,
    groups narrowed, pairs of leaves compared, surrogate contacts).  With
    check=True the call synchronises, grows overflowing buffers and repeats.
    Returns (sets_out, contacts, surrogate, counts)."""
    info = hier.info()
    P = _pair_args(hier, pairs, eps, poses, info["n_particles"])
    dev = pairs.device
    if sets_out is None:
        sets_out = ActiveSets(max(sets_in.capacity, 1024), dev)
    if contacts is None:
        contacts = Contacts(max(1024, 64 * P), dev)
    if surrogate is None:
        surrogate = Contacts(max(1024, 4 * P), dev)
    if counts is None:
        counts = torch.zeros(4, dtype=torch.int64, device=dev)
    lib = L.load()
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    for _ in range(max_retries + 1):
        si, so, cs, ss = sets_in.struct(), sets_out.struct(), contacts.struct(), surrogate.struct()
        L.check(lib.mrdem_active_set_step(ctx.handle, hier.handle, P, _p(pairs), _p(eps),
                                          _p(poses), prec, C.byref(si), C.byref(so),
                                          C.byref(cs), C.byref(ss), _p(counts),
                                          _stream(stream)), "mrdem_active_set_step")
        if not check:
            return sets_out, contacts, surrogate, counts
        req = np.zeros(5, np.int64)
        st = lib.mrdem_check(ctx.handle, _stream(stream), _np_ptr(req))
        if st == L.MRDEM_OK:
            return sets_out, contacts, surrogate, counts
        if st != L.MRDEM_ERR_CAPACITY:
            L.check(st, "mrdem_active_set_step")
        prm = ctx.params
        grow = lambda need, cap: int(need * 1.25) + 1024 if need > cap else 0  # noqa: E731
        ti, ca = grow(req[1], prm.cap_tiles), grow(req[2], prm.cap_candidates)
        sw = grow(req[4], prm.cap_sweep)
        if ti or ca or sw:
            ctx.reserve(0, ti, ca, sw)
        if req[3] > contacts.capacity:
            contacts.resize(int(req[3] * 1.25) + 1024)
        if int(surrogate.count.item()) > surrogate.capacity:
            surrogate.resize(int(surrogate.count.item() * 1.25) + 1024)
        if int(sets_out.count.item()) > sets_out.capacity:
            sets_out.resize(int(sets_out.count.item() * 1.25) + 1024)
    raise L.MrdemError(L.MRDEM_ERR_CAPACITY, "mrdem_active_set_step (retries exhausted)")


def surrogate_forces(ctx, hier, pairs, eps, poses, surrogate, mass, com, k_s=1000.0, weight=0.25,
                     force_torque=None, energy=None, stream=None):
    """Forces and torques of surrogate contacts (mrdem_surrogate_forces),
    accumulated into force_torque [n, 6] and energy [1]."""
    n = hier.info()["n_particles"]
    P = _pair_args(hier, pairs, eps, poses, n)
    _need(mass, torch.float64, (n,), "mass")
    _need(com, torch.float64, (n, 3), "com")
    if force_torque is None:
        force_torque = torch.zeros((n, 6), dtype=torch.float64, device=pairs.device)
    if energy is None:
        energy = torch.zeros(1, dtype=torch.float64, device=pairs.device)
    ss = surrogate.struct()
    L.check(L.load().mrdem_surrogate_forces(ctx.handle, hier.handle, P, _p(pairs), _p(eps),
                                            _p(poses), C.byref(ss), _p(mass), _p(com), float(k_s),
                                            float(weight), _p(force_torque), _p(energy),
                                            _stream(stream)), "mrdem_surrogate_forces")
    return force_torque, energy


def implicit_euler_step_multires(ctx: Context, hier: Hierarchy, poses0, vel0, mass, inertia,
                                 pairs, eps, dt, gravity=G_DEFAULT, k_s=1000.0, precision="fp32",
                                 tol=1e-13, max_iter=200, weight=0.25):
    """One implicit Euler step by the multiresolution Picard iteration of
    Algorithm 6: every pair's active set starts at the two roots and is kept
    across the iterations; each iteration moves the particles from poses0
    by dt times the guessed velocities, tests the active sets there
    (mrdem_active_set_step: fine contacts of the pairs of leaves in contact
    range, surrogate contacts of the other pairs in range, which are widened
    to their children, and narrowing of groups certainly apart), applies
    the fine contacts' forces and the surrogate contacts' forces weighted by
    `weight`, and updates the guess.  It stops when max |new - guess| <=
    tol * max |new| and the iteration widened and narrowed nothing; the
    result is then the plain implicit Euler step's fixed point.  One host
    synchronisation per iteration.  Returns (poses, vel, iterations,
    history of the relative change, per-iteration record)."""
    n = poses0.shape[0]
    dev = poses0.device
    P = pairs.shape[0]
    vel = vel0.clone()
    poses = torch.empty_like(poses0)
    com = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    ft = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    norms = torch.empty(2, dtype=torch.float64, device=dev)
    counts = torch.zeros(4, dtype=torch.int64, device=dev)
    sets = [active_sets_init(ctx, hier, pairs), None] if P else [None, None]
    contacts = surrogate = None
    hist, record = [], []
    it = 0
    for it in range(1, max_iter + 1):
        move_poses(ctx, poses0, vel, dt, out=poses)
        ft.zero_()
        items = 0
        if P:
            items = sets[0].n()
            sets[1], contacts, surrogate, counts = active_sets_step(
                ctx, hier, pairs, eps, poses, sets[0], sets[1], precision, contacts, surrogate,
                counts)
            contact_forces(ctx, hier, pairs, eps, poses, contacts, mass, com, k_s,
                           force_torque=ft, energy=energy)
            surrogate_forces(ctx, hier, pairs, eps, poses, surrogate, mass, com, k_s, weight,
                             force_torque=ft, energy=energy)
            sets.reverse()
        picard_update(ctx, vel0, ft, mass, inertia, dt, vel, norms, gravity)
        change, scale = norms.tolist()
        c = counts.tolist() if P else [0, 0, 0, 0]
        scale += 1e-300
        hist.append(change / scale)
        record.append(dict(items=items, widened=c[0], narrowed=c[1], leaf_pairs=c[2],
                           surrogate=c[3], contacts=contacts.n() if P else 0))
        if change <= tol * scale and c[0] == 0 and c[1] == 0:
            break
    move_poses(ctx, poses0, vel, dt, out=poses)
    return poses, vel, it, hist, record


def newton_residual(ctx, vel0, vel, force_torque, mass, inertia, dt, res=None, norms=None,
                    gravity=G_DEFAULT, stream=None):
    """Residual M (vel - vel0)/dt - (F, tau) - (m g, 0) of the implicit Euler
    equations; returns (res [n, 6], norms (max |res|, max |M vel|/dt))."""
    n = vel0.shape[0]
    for t, name in ((vel0, "vel0"), (vel, "vel"), (force_torque, "force_torque")):
        _need(t, torch.float64, (n, 6), name)
    _need(mass, torch.float64, (n,), "mass")
    _need(inertia, torch.float64, (n,), "inertia")
    if res is None:
        res = torch.empty_like(vel0)
    if norms is None:
        norms = torch.empty(2, dtype=torch.float64, device=vel0.device)
    g = (C.c_double * 3)(*[float(x) for x in gravity])
    L.check(L.load().mrdem_newton_residual(ctx.handle, n, _p(vel0), _p(vel), _p(force_torque),
                                           _p(mass), _p(inertia), C.cast(g, C.c_void_p),
                                           float(dt), _p(res), _p(norms), _stream(stream)),
            "mrdem_newton_residual")
    return res, norms


def newton_solve(ctx, pairs, blocks, mass, inertia, dt, rhs, x=None, max_iter=200, rel_tol=1e-12,
                 info=None, stream=None, check_every=0):
    """x with (M/dt + dt K) x = rhs by preconditioned conjugate gradients (K
    the pair blocks); returns (x [n, 6], info (iterations, relative
    residual, breakdown flag, |rhs|))."""
    n = rhs.shape[0]
    P = pairs.shape[0]
    _need(rhs, torch.float64, (n, 6), "rhs")
    _need(blocks, torch.float64, (P, 12, 12), "blocks")
    if x is None:
        x = torch.empty_like(rhs)
    if info is None:
        info = torch.empty(4, dtype=torch.float64, device=rhs.device)
    L.check(L.load().mrdem_newton_solve(ctx.handle, n, P, _p(pairs), _p(blocks), _p(mass),
                                        _p(inertia), float(dt), _p(rhs), _p(x), int(max_iter),
                                        float(rel_tol), int(check_every), _p(info),
                                        _stream(stream)),
            "mrdem_newton_solve")
    return x, info


def implicit_euler_step_newton(ctx: Context, hier: Hierarchy, poses0, vel0, mass, inertia, pairs,
                               eps, dt, gravity=G_DEFAULT, k_s=1000.0, precision="fp32",
                               tol=1e-13, max_iter=50, cg_iter=200, cg_tol=1e-12, contacts=None,
                               cache_margin=None, bound=None, stiffness="hessian"):
    """One implicit Euler step by Newton's method in the velocities, on the
    same equations as the Picard iteration: residual
    r = M (V - V0)/dt - (F, tau)(moved geometry) - (m g, 0), Jacobian
    M/dt + dt K with K the contact Hessian blocks (closest points free), the
    linear system solved by conjugate gradients, each step halved until
    max |r| drops (backtracking).  Stops when max |r| <= tol max |M V|/dt.
    With cache_margin = w (and bound) the residuals take their contacts from
    candidates kept across the step (KeptCandidates).  stiffness="gauss-newton"
    uses the adjoint's 12x12 Gauss-Newton blocks e''(d) J J^T (closest points
    frozen; positive semi-definite, so the solve never meets negative
    curvature, but the iteration converges only linearly) instead of the
    contact Hessian.
    Returns (poses, vel, iterations, stats: CG iterations and line-search
    halvings per Newton iteration).  A step that no halving makes descend
    (30 halvings without a lower max |r|) is not taken: the iteration stops
    at the previous V and that iteration's stats say line_search_failed."""
    if stiffness not in ("hessian", "gauss-newton"):
        raise ValueError(f"stiffness must be 'hessian' or 'gauss-newton', not {stiffness!r}")
    lib = L.load()
    n = poses0.shape[0]
    dev = poses0.device
    P = pairs.shape[0]
    V = vel0.clone()
    Vt = torch.empty_like(V)
    poses = torch.empty_like(poses0)
    com = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    ft = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    res = torch.empty((n, 6), dtype=torch.float64, device=dev)
    norms = torch.empty(2, dtype=torch.float64, device=dev)
    blocks = torch.zeros((P, 12, 12), dtype=torch.float64, device=dev)
    x = torch.empty((n, 6), dtype=torch.float64, device=dev)
    info = torch.empty(4, dtype=torch.float64, device=dev)
    state = {"contacts": contacts}
    kept = (KeptCandidates(ctx, hier, pairs, eps, cache_margin, bound, precision)
            if cache_margin is not None else None)

    def residual(Vc):
        move_poses(ctx, poses0, Vc, dt, out=poses)
        ft.zero_()
        if P:
            if kept is not None:
                state["contacts"] = kept.contacts(poses, out=state["contacts"])
            else:
                state["contacts"], _ = detect(ctx, hier, pairs, eps, poses, precision,
                                              contacts=state["contacts"])
            contact_forces(ctx, hier, pairs, eps, poses, state["contacts"], mass, com, k_s,
                           force_torque=ft, energy=energy)
        newton_residual(ctx, vel0, Vc, ft, mass, inertia, dt, res, norms, gravity)
        return norms.tolist()

    rn, sc = residual(V)
    stats = []
    it = 0
    for it in range(1, max_iter + 1):
        if rn <= tol * (sc + 1e-300):
            break
        if P and stiffness == "gauss-newton":
            _, _, jac = contact_grad(ctx, hier, pairs, eps, poses, state["contacts"], mass, k_s,
                                     want_verts=False, want_pose=False, want_jac=True)
            blocks.copy_(jac)
        elif P:
            blocks.zero_()
            contact_hessian(ctx, hier, pairs, eps, poses, state["contacts"], mass, k_s,
                            blocks=blocks)
        newton_solve(ctx, pairs, blocks, mass, inertia, dt, res, x, cg_iter, cg_tol, info,
                     check_every=16)
        cg = info.tolist()
        lam, halvings, descended = 1.0, 0, False
        while True:
            L.check(lib.mrdem_vel_axpy(ctx.handle, 6 * n, -lam, _p(x), _p(V), _p(Vt), None),
                    "mrdem_vel_axpy")
            rt, st = residual(Vt)
            if rt < rn:
                descended = True
                break
            if lam < 2.0 ** -30:
                break
            lam *= 0.5
            halvings += 1
        stats.append({"cg_iterations": int(cg[0]), "cg_residual": cg[1], "cg_breakdown": cg[2] != 0,
                      "halvings": halvings, "line_search_failed": not descended})
        if not descended:
            # keep V; the contacts of the last trial are stale, so the
            # residual is evaluated at V once more before returning
            residual(V)
            break
        V, Vt = Vt, V
        rn, sc = rt, st
    move_poses(ctx, poses0, V, dt, out=poses)
    return poses, V, it, stats


class ContactProblem:
    """Everything the energy of a particle batch depends on, resident on the device."""

    def __init__(self, ctx, hier, pairs, eps, poses, mass, com, k_s=1000.0, precision="fp32"):
        self.ctx, self.hier = ctx, hier
        self.pairs, self.eps, self.poses, self.mass, self.com = pairs, eps, poses, mass, com
        self.k_s, self.precision = float(k_s), precision
        self.contacts = None

    @classmethod
    def from_scene(cls, ctx, hier, scene, device, precision="fp32", k_s=1000.0):
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)  # noqa: E731
        prob = cls(ctx, hier, t(scene.pairs, torch.int32), t(scene.eps, torch.float64),
                   t(scene.poses, torch.float64), t(scene.mass, torch.float64),
                   t(scene.com, torch.float64), k_s, precision)
        prob.set_mesh(scene.vert_off, t(scene.verts, torch.float32), scene.tri_off,
                      t(scene.tris, torch.int32))
        return prob

    def set_mesh(self, vert_off, verts, tri_off, tris):
        """The meshes the hierarchy was built from (host offsets, device
        float32 vertices and int32 local triangles): ContactEnergy rebuilds
        the trees from other vertex values with them."""
        self.mesh = (np.ascontiguousarray(vert_off, np.int64), verts.contiguous(),
                     np.ascontiguousarray(tri_off, np.int64), tris.contiguous())

    def detect(self, stats=None, check=True, stream=None):
        self.contacts, st = detect(self.ctx, self.hier, self.pairs, self.eps, self.poses,
                                   self.precision, contacts=self.contacts, stats=stats,
                                   check=check, stream=stream)
        return self.contacts, st

    def forces(self, stream=None):
        return contact_forces(self.ctx, self.hier, self.pairs, self.eps, self.poses, self.contacts,
                              self.mass, self.com, self.k_s, stream=stream)

    def grad(self, scale=1.0, want_jac=False, stream=None):
        return contact_grad(self.ctx, self.hier, self.pairs, self.eps, self.poses, self.contacts,
                            self.mass, self.k_s, scale, want_jac=want_jac, stream=stream)

    # ---- one step of the batch: detection, forces and energy, adjoint
    def _outputs(self, want_verts, want_pose, want_jac):
        info = self.hier.info()
        n, P, d = info["n_particles"], self.pairs.shape[0], self.pairs.device
        o = getattr(self, "_out", None)
        if o is None:
            o = self._out = dict(
                ft=torch.zeros((n, 6), dtype=torch.float64, device=d),
                energy=torch.zeros(1, dtype=torch.float64, device=d),
                gv=torch.zeros((info["n_verts"], 3), dtype=torch.float32, device=d),
                gp=torch.zeros((n, 6), dtype=torch.float64, device=d),
                jac=torch.zeros((P, 12, 12), dtype=torch.float64, device=d),
                stats=torch.zeros(L.MRDEM_STAT_COUNT, dtype=torch.int64, device=d))
        if self.contacts is None:
            self.contacts = Contacts(max(1024, 64 * P), d)
        return (o["ft"], o["energy"], o["gv"] if want_verts else None,
                o["gp"] if want_pose else None, o["jac"] if want_jac else None, o["stats"])

    def _enqueue(self, scale, want_verts, want_pose, want_jac, host_in=None, host_out=None):
        lib = L.load()
        ft, energy, gv, gp, jac, stats = self._outputs(want_verts, want_pose, want_jac)
        for k, t in (host_in or {}).items():
            getattr(self, k).copy_(t, non_blocking=True)
        for t in (ft, energy, gv, gp, jac):
            if t is not None:
                t.zero_()
        P, s = self.pairs.shape[0], _stream(None)
        prec = PRECISION[self.precision] if isinstance(self.precision, str) else int(self.precision)
        cs = self.contacts.struct()
        h, c = self.hier.handle, self.ctx.handle
        L.check(lib.mrdem_detect(c, h, P, _p(self.pairs), _p(self.eps), _p(self.poses), prec,
                                 C.byref(cs), _p(stats), s), "mrdem_detect")
        # forces and the adjoint both read the contacts: the adjoint runs on a
        # second stream beside the forces (each call keeps its own tables)
        want_grad = gv is not None or gp is not None or jac is not None
        if want_grad:
            side = getattr(self, "_side", None)
            if side is None:
                side = self._side = torch.cuda.Stream(device=self.pairs.device)
            side.wait_stream(torch.cuda.current_stream())
        L.check(lib.mrdem_contact_forces(c, h, P, _p(self.pairs), _p(self.eps), _p(self.poses),
                                         C.byref(cs), _p(self.mass), _p(self.com), self.k_s,
                                         _p(ft), _p(energy), s), "mrdem_contact_forces")
        if want_grad:
            L.check(lib.mrdem_contact_grad(c, h, P, _p(self.pairs), _p(self.eps), _p(self.poses),
                                           C.byref(cs), _p(self.mass), self.k_s, float(scale),
                                           _p(gv), _p(gp), _p(jac), C.c_void_p(side.cuda_stream)),
                    "mrdem_contact_grad")
            torch.cuda.current_stream().wait_stream(side)
        if host_out:
            src = dict(ft=ft, energy=energy, gv=gv, gp=gp, jac=jac, count=self.contacts.count)
            for k, t in host_out.items():
                t.copy_(src[k], non_blocking=True)
        # the status words to pinned host memory at the end of the step (no
        # synchronisation of their own: the step's one synchronisation covers them)
        if getattr(self, "_status_host", None) is None:
            self._status_host = torch.zeros(L.MRDEM_STATUS_WORDS, dtype=torch.int64).pin_memory()
        L.check(lib.mrdem_status_async(c, C.c_void_p(self._status_host.data_ptr()), s),
                "mrdem_status_async")

    def _check_and_grow(self):
        """Status of the work just enqueued (synchronises the stream once and
        decodes the status words the step copied to the host): True if it
        completed, False after growing an overflowing list."""
        lib = L.load()
        req = np.zeros(5, np.int64)
        torch.cuda.current_stream().synchronize()
        st = lib.mrdem_status_decode(C.c_void_p(self._status_host.data_ptr()), _np_ptr(req))
        if st == L.MRDEM_OK:
            return True
        if st != L.MRDEM_ERR_CAPACITY:
            L.check(st, "ContactProblem.step")
        prm = self.ctx.params
        grow = lambda need, cap: int(need * 1.25) + 1024 if need > cap else 0  # noqa: E731
        lv, ti, ca = grow(req[0], prm.cap_level), grow(req[1], prm.cap_tiles), grow(req[2], prm.cap_candidates)
        sw = grow(req[4], prm.cap_sweep)
        if lv or ti or ca or sw:
            self.ctx.reserve(lv, ti, ca, sw)
        if req[3] > self.contacts.capacity:
            self.contacts.resize(int(req[3] * 1.25) + 1024)
        self._graph = None
        return False

    def step(self, scale=1.0, want_verts=True, want_pose=True, want_jac=False, graph=True,
             max_retries=4, host_in=None, host_out=None):
        """Detection, forces and energy, and the adjoint of the whole batch in
        one call on the current stream.  The status is checked once, at the end
        (one synchronisation); after a list overflow the lists grow and the
        step runs again.  host_in: None, or a dict of pinned host tensors
        (keys among "poses", "pairs", "eps", "mass", "com", shaped like the
        problem's) copied into the problem's inputs at the start of every
        step; host_out: None, or a dict of pinned host tensors (keys among
        "ft", "energy", "gv", "gp", "jac", "count") that receive those
        results before the synchronisation.  Both copies are part of the
        step's graph, so a host caller's step is one replay and one
        synchronisation.  With graph=True the sequence is captured once into a
        CUDA graph (captured again after a list grows or the flags change) and
        replayed, so the inputs must be updated in place (pairs, eps, poses,
        mass, com keep their storage).  Returns tensors owned by the problem,
        overwritten by the next step: (contacts, force_torque, energy,
        dE_dverts, dE_dpose, jac, stats)."""
        io = tuple(sorted((k, t.data_ptr()) for k, t in (host_in or {}).items())) + \
            tuple(sorted((k, t.data_ptr()) for k, t in (host_out or {}).items()))
        key = (float(scale), bool(want_verts), bool(want_pose), bool(want_jac), io)
        run = (scale, want_verts, want_pose, want_jac, host_in, host_out)
        for _ in range(max_retries + 1):
            g = getattr(self, "_graph", None)
            if not graph:
                self._enqueue(*run)
            elif g is not None and self._graph_key == key:
                g.replay()
            else:
                # an uncaptured run first: it sizes the scratch the graph will use
                self._enqueue(*run)
                if not self._check_and_grow():
                    continue
                g = torch.cuda.CUDAGraph()
                side = torch.cuda.Stream()
                side.wait_stream(torch.cuda.current_stream())
                with torch.cuda.graph(g, stream=side):
                    self._enqueue(*run)
                torch.cuda.current_stream().wait_stream(side)
                self._graph, self._graph_key = g, key
                g.replay()
            if self._check_and_grow():
                ft, energy, gv, gp, jac, stats = self._outputs(want_verts, want_pose, want_jac)
                return self.contacts, ft, energy, gv, gp, jac, stats
        raise L.MrdemError(L.MRDEM_ERR_CAPACITY, "ContactProblem.step (retries exhausted)")


def twist_grad(ctx: Context, twist, grad_pose, out=None, stream=None):
    """Gradient in the twist of poses moved by it (mrdem_twist_grad)."""
    n = twist.shape[0]
    _need(twist, torch.float64, (n, 6), "twist")
    _need(grad_pose, torch.float64, (n, 6), "grad_pose")
    if out is None:
        out = torch.empty_like(grad_pose)
    L.check(L.load().mrdem_twist_grad(ctx.handle, n, _p(twist), _p(grad_pose), _p(out),
                                      _stream(stream)), "mrdem_twist_grad")
    return out


class ContactEnergy(torch.autograd.Function):
    """E(verts, twist) = sum over the contacts of K_s sqrt(mu) eps (1 - d/(2 eps))^2
    at the geometry the two inputs give.

    verts: body-frame vertices [n_verts, 3] (float32 or float64; the meshes are
    their float32 values, as the library stores every mesh).  twist: [n, 6]
    float64, per particle a world translation v and a rotation vector w: the
    pose moves to centre + v and orientation exp(w) R (mrdem_move_poses with
    dt = 1).  Forward: when verts differ from the problem's meshes, the
    surrogate trees are rebuilt from them on the GPU
    (mrdem_build_hierarchy_device), then the poses are moved, the contacts
    detected and the energy summed.  Backward: the adjoint kernel at that
    geometry gives dE/dverts and dE/dpose (a translation and a left rotation
    increment about each particle origin); the rotation part goes through the
    exponential map's left Jacobian (mrdem_twist_grad)."""

    @staticmethod
    def forward(fctx, verts, twist, problem: ContactProblem):
        ctx = problem.ctx
        hier = problem.hier
        v32 = verts.detach().to(torch.float32).contiguous()
        mesh = getattr(problem, "mesh", None)
        if mesh is None or not torch.equal(v32, mesh[1]):
            if mesh is None:
                raise ValueError("ContactEnergy: the problem has no meshes (set_mesh) to "
                                 "rebuild the trees from new vertices")
            hier = Hierarchy.build_device(ctx, mesh[0], v32, mesh[2], mesh[3])
        tw = twist.detach().to(torch.float64).contiguous()
        poses = move_poses(ctx, problem.poses, tw, 1.0)
        contacts, _ = detect(ctx, hier, problem.pairs, problem.eps, poses, problem.precision)
        _, energy = contact_forces(ctx, hier, problem.pairs, problem.eps, poses, contacts,
                                   problem.mass, problem.com, problem.k_s)
        fctx.state = (hier, poses, contacts, tw, problem, verts.dtype)
        return energy[0].clone()

    @staticmethod
    def backward(fctx, g):
        hier, poses, contacts, tw, problem, vdtype = fctx.state
        gv, gp, _ = contact_grad(problem.ctx, hier, problem.pairs, problem.eps, poses, contacts,
                                 problem.mass, problem.k_s, float(g.item()))
        gt = twist_grad(problem.ctx, tw, gp)
        return gv.to(vdtype), gt, None


def contact_energy(problem: ContactProblem, verts=None, twist=None):
    """ContactEnergy at the problem's meshes and poses (or the given ones),
    with the inputs returned as leaves that require gradients."""
    info = problem.hier.info()
    d = problem.pairs.device
    if verts is None:
        verts = problem.mesh[1].clone().requires_grad_(True)
    if twist is None:
        twist = torch.zeros((info["n_particles"], 6), dtype=torch.float64, device=d,
                            requires_grad=True)
    return ContactEnergy.apply(verts, twist, problem), verts, twist
