"""FP64 CPU oracle (test infrastructure only).

Loads `mrdem_oracle.cpp` (compiled with g++ into `oracle/_build/`) through
ctypes and exposes numpy-level wrappers.  Only the tests, the smoke check and
the CPU-baseline leg of bench.py use this module; the product path never
imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrdem_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++, OpenMP, no fast-math) unless a build of the
    same source (content hash, stored beside the library) is present."""
    import hashlib
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off"]
    with open(_SRC, "rb") as f:
        digest = hashlib.sha256(" ".join(cmd + [os.uname().machine]).encode() + f.read()).hexdigest()
    try:
        with open(_OUT + ".inputs") as f:
            fresh = os.path.exists(_OUT) and f.read().strip() == digest
    except OSError:
        fresh = False
    if force or not fresh:
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(cmd + [_SRC, "-o", tmp])
        os.replace(tmp, _OUT)
        with open(_OUT + ".inputs", "w") as f:
            f.write(digest + "\n")
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_P = C.c_void_p
_I64 = C.c_int64


def _declare(L):
    L.orc_point_triangle.argtypes = [_I64, _P, _P, _P, _P]
    L.orc_segment_segment.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.orc_tri_tri.argtypes = [_I64, _P, _P, _P, _P, _P, _P]
    L.orc_pose_matrix.argtypes = [_P, _P]
    L.orc_detect.argtypes = [_P, _P, _P, _P, _P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P, _P,
                             _P, C.c_int]
    L.orc_detect.restype = _I64
    L.orc_forces.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_double, _I64, _P, _P, _P,
                             _P, _P, _P, _P]
    L.orc_energy.argtypes = [_P, _P, _P, _P, _P, _P, _I64, _P, _P, C.c_double, C.c_int]
    L.orc_energy.restype = C.c_double
    L.orc_grad.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, C.c_double, _I64, _P, _P, _P, _P,
                           _P, _P]
    L.orc_sweep.argtypes = [_I64, _P, _P, C.c_int, C.c_double, C.c_double, C.c_double, _P, _P,
                            _P, _P, _P]
    L.orc_vertex_surrogate_distance.argtypes = [_I64, _P, _P, _P]
    L.orc_tri_pairs.argtypes = [_P, _P, _P, _P, _P, _I64, _P, _P, _P, _P, _P, C.c_int]


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


# ----------------------------------------------------------------------------
# primitives
# ----------------------------------------------------------------------------
def point_triangle(p, T):
    p = _c(p, np.float64).reshape(-1, 3)
    T = _c(T, np.float64).reshape(-1, 9)
    n = len(p)
    q = np.empty((n, 3))
    d = np.empty(n)
    lib().orc_point_triangle(n, _ptr(p), _ptr(T), _ptr(q), _ptr(d))
    return d, q


def segment_segment(S1, S2):
    S1 = _c(S1, np.float64).reshape(-1, 6)
    S2 = _c(S2, np.float64).reshape(-1, 6)
    n = len(S1)
    c1, c2, d = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
    lib().orc_segment_segment(n, _ptr(S1), _ptr(S2), _ptr(c1), _ptr(c2), _ptr(d))
    return d, c1, c2


def tri_tri(P, Q):
    """Exact triangle-triangle distance (comparison-based); returns d, pa, pb, feature."""
    P = _c(P, np.float64).reshape(-1, 9)
    Q = _c(Q, np.float64).reshape(-1, 9)
    n = len(P)
    d, pa, pb = np.empty(n), np.empty((n, 3)), np.empty((n, 3))
    f = np.empty(n, np.int32)
    lib().orc_tri_tri(n, _ptr(P), _ptr(Q), _ptr(d), _ptr(pa), _ptr(pb), _ptr(f))
    return d, pa, pb, f


def pose_matrix(pose):
    pose = _c(pose, np.float64)
    R = np.empty(9)
    lib().orc_pose_matrix(_ptr(pose), _ptr(R))
    return R.reshape(3, 3)


def sweep(P, Q, eps, n_iter=4, rho_reg=1.0, rho_iter=1e3, conv_c=1.0):
    P = _c(P, np.float64).reshape(-1, 9)
    Q = _c(Q, np.float64).reshape(-1, 9)
    n = len(P)
    eps = _c(np.broadcast_to(eps, (n,)), np.float64)
    x, gap, dist = np.empty((n, 4)), np.empty(n), np.empty(n)
    conv = np.empty(n, np.int32)
    lib().orc_sweep(n, _ptr(P), _ptr(Q), n_iter, rho_reg, rho_iter, conv_c, _ptr(eps), _ptr(x),
                    _ptr(gap), _ptr(conv), _ptr(dist))
    return dict(x=x, gap=gap, converged=conv.astype(bool), dist_iter=dist)


def vertex_surrogate_distance(v, T):
    v = _c(v, np.float64).reshape(-1, 3)
    T = _c(T, np.float64).reshape(-1, 9)
    d = np.empty(len(v))
    lib().orc_vertex_surrogate_distance(len(v), _ptr(v), _ptr(T), _ptr(d))
    return d


# ----------------------------------------------------------------------------
# scene-level
# ----------------------------------------------------------------------------
def _mesh(scene, verts=None):
    v = scene.verts if verts is None else verts
    return (_c(scene.vert_off, np.int64), _c(v, np.float64), _c(scene.tri_off, np.int64),
            _c(scene.tris, np.int32))


def detect(scene, poses=None, pairs=None, eps=None, n_threads=0, verts=None):
    """Brute-force contact set of every pair (sorted by pair, ta, tb)."""
    vo, v, to, t = _mesh(scene, verts)
    poses = _c(scene.poses if poses is None else poses, np.float64)
    pairs = _c(scene.pairs if pairs is None else pairs, np.int32)
    eps = _c(scene.eps if eps is None else eps, np.float64)
    n_pairs = len(pairs)
    cap = 1024
    while True:
        out = dict(pair=np.empty(cap, np.int32), ta=np.empty(cap, np.int32),
                   tb=np.empty(cap, np.int32), d=np.empty(cap), pa=np.empty((cap, 3)),
                   pb=np.empty((cap, 3)), feature=np.empty(cap, np.int32))
        n = lib().orc_detect(_ptr(vo), _ptr(v), _ptr(to), _ptr(t), _ptr(poses), n_pairs,
                             _ptr(pairs), _ptr(eps), cap, _ptr(out["pair"]), _ptr(out["ta"]),
                             _ptr(out["tb"]), _ptr(out["d"]), _ptr(out["pa"]), _ptr(out["pb"]),
                             _ptr(out["feature"]), n_threads)
        if n <= cap:
            return {k: a[:n] for k, a in out.items()}
        cap = int(n)


def tri_pairs(scene, abt, poses=None, n_threads=0):
    """Distances of listed fine triangle pairs: abt [n, 4] = (particle A,
    local triangle of A, particle B, local triangle of B).  The same world
    triangles and exact distance as detect, so a listed pair gets the values
    detect reports for it.  Returns d, pa, pb, feature."""
    vo, v, to, t = _mesh(scene)
    poses = _c(scene.poses if poses is None else poses, np.float64)
    abt = _c(abt, np.int32).reshape(-1, 4)
    n = len(abt)
    d, pa, pb = np.empty(n), np.empty((n, 3)), np.empty((n, 3))
    f = np.empty(n, np.int32)
    lib().orc_tri_pairs(_ptr(vo), _ptr(v), _ptr(to), _ptr(t), _ptr(poses), n, _ptr(abt), _ptr(d),
                        _ptr(pa), _ptr(pb), _ptr(f), n_threads)
    return d, pa, pb, f


def forces(scene, contacts, k_s=1000.0, poses=None):
    vo, v, to, t = _mesh(scene)
    poses = _c(scene.poses if poses is None else poses, np.float64)
    ft = np.zeros((scene.n_particles, 6))
    en = np.zeros(1)
    n = len(contacts["d"])
    lib().orc_forces(_ptr(vo), _ptr(v), _ptr(to), _ptr(t), _ptr(poses),
                     _ptr(_c(scene.mass, np.float64)), _ptr(_c(scene.com, np.float64)),
                     _ptr(_c(scene.pairs, np.int32)), _ptr(_c(scene.eps, np.float64)), k_s, n,
                     _ptr(_c(contacts["pair"], np.int32)), _ptr(_c(contacts["ta"], np.int32)),
                     _ptr(_c(contacts["d"], np.float64)), _ptr(_c(contacts["pa"], np.float64)),
                     _ptr(_c(contacts["pb"], np.float64)), _ptr(ft), _ptr(en))
    return ft, float(en[0])


def energy(scene, poses=None, verts=None, k_s=1000.0, n_threads=0):
    vo, v, to, t = _mesh(scene, verts)
    poses = _c(scene.poses if poses is None else poses, np.float64)
    return lib().orc_energy(_ptr(vo), _ptr(v), _ptr(to), _ptr(t), _ptr(poses),
                            _ptr(_c(scene.mass, np.float64)), scene.n_pairs,
                            _ptr(_c(scene.pairs, np.int32)), _ptr(_c(scene.eps, np.float64)), k_s,
                            n_threads)


def grad(scene, contacts, k_s=1000.0, poses=None, verts=None):
    """Analytic gradient: (dE/dverts [nv,3] body frame, dE/dpose [n,6], jac [P,12,12])."""
    vo, v, to, t = _mesh(scene, verts)
    poses = _c(scene.poses if poses is None else poses, np.float64)
    gv = np.zeros((len(v), 3))
    gp = np.zeros((scene.n_particles, 6))
    jac = np.zeros((scene.n_pairs, 12, 12))
    n = len(contacts["pair"])
    lib().orc_grad(_ptr(vo), _ptr(v), _ptr(to), _ptr(t), _ptr(poses),
                   _ptr(_c(scene.mass, np.float64)), _ptr(_c(scene.pairs, np.int32)),
                   _ptr(_c(scene.eps, np.float64)), k_s, n, _ptr(_c(contacts["pair"], np.int32)),
                   _ptr(_c(contacts["ta"], np.int32)), _ptr(_c(contacts["tb"], np.int32)),
                   _ptr(gv), _ptr(gp), _ptr(jac))
    return gv, gp, jac


def world_triangles(scene, i, poses=None):
    """FP64 world-frame triangles [n, 9] of particle i (for tests)."""
    poses = scene.poses if poses is None else poses
    v, t = scene.particle(i)
    R = pose_matrix(poses[i])
    w = v.astype(np.float64) @ R.T + poses[i][:3]
    return w[t].reshape(-1, 9)


def merge_contacts(contacts, eps):
    """Redundant-contact filter of Sec. 2 (the implementation note on the
    contact set C): close-by contact points of one particle pair are merged
    into one average point.

    Reading: within each pair p, two contacts are linked when their contact
    points x = (pa + pb)/2 are closer than the pair's eps, evaluated in FP64
    as ((dx*dx + dy*dy) + dz*dz) < eps*eps; every connected component of the
    links (the transitive closure, so the result does not depend on the order
    of C) with two or more members becomes one contact with pa and pb the
    means of its members' (its contact point is then the mean contact point
    and its normal the mean normal), d = |pa - pb|, and ta, tb of the member
    with the smallest (ta, tb); a contact with no other closer than eps stays
    as it is (d included).  Returns the merged list sorted by (pair, ta, tb) and, per
    merged contact, the number of members ("members").
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    pair = np.asarray(contacts["pair"], np.int64)
    ta = np.asarray(contacts["ta"], np.int64)
    tb = np.asarray(contacts["tb"], np.int64)
    pa = np.asarray(contacts["pa"], np.float64).reshape(-1, 3)
    pb = np.asarray(contacts["pb"], np.float64).reshape(-1, 3)
    dist = np.asarray(contacts["d"], np.float64)
    eps = np.asarray(eps, np.float64)
    order = np.lexsort((tb, ta, pair))
    starts = np.flatnonzero(np.r_[True, pair[order][1:] != pair[order][:-1]]) if len(order) else []
    ends = list(starts[1:]) + [len(order)]
    out = {k: [] for k in ("pair", "ta", "tb", "d", "pa", "pb", "members")}
    for s, e in zip(starts, ends):
        idx = order[s:e]
        p = int(pair[idx[0]])
        x = (pa[idx] + pb[idx]) * 0.5
        lim = eps[p] * eps[p]
        n = len(idx)
        rows, cols = [], []
        for r0 in range(0, n, 512):  # the squared distances, a block of rows at a time
            xr = x[r0:r0 + 512]
            dx = xr[:, None, 0] - x[None, :, 0]
            dy = xr[:, None, 1] - x[None, :, 1]
            dz = xr[:, None, 2] - x[None, :, 2]
            i, j = np.nonzero((dx * dx + dy * dy) + dz * dz < lim)
            rows.append(i + r0)
            cols.append(j)
        rows, cols = np.concatenate(rows), np.concatenate(cols)
        adj = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
        _, lab = connected_components(adj, directed=False)
        # components in the order of their first (smallest-key) member
        first = {}
        for k, c in enumerate(lab):
            first.setdefault(int(c), k)
        for c, k0 in sorted(first.items(), key=lambda t: t[1]):
            m = idx[lab == c]
            if len(m) == 1:  # nothing close by: the contact stays as detected
                a, b, d = pa[m[0]], pb[m[0]], float(dist[m[0]])
            else:
                a, b = pa[m].mean(axis=0), pb[m].mean(axis=0)
                d = float(np.sqrt(np.sum((a - b) ** 2)))
            out["pair"].append(p)
            out["ta"].append(int(ta[idx[k0]]))
            out["tb"].append(int(tb[idx[k0]]))
            out["pa"].append(a)
            out["pb"].append(b)
            out["d"].append(d)
            out["members"].append(len(m))
    return dict(pair=np.array(out["pair"], np.int32), ta=np.array(out["ta"], np.int32),
                tb=np.array(out["tb"], np.int32), d=np.array(out["d"], np.float64),
                pa=np.array(out["pa"], np.float64).reshape(-1, 3),
                pb=np.array(out["pb"], np.float64).reshape(-1, 3),
                members=np.array(out["members"], np.int64))
