"""Bumped icosphere particles and particle-pair scenes (seeded, synthetic).

The paper's particles are spheres triangulated into |T| triangles whose
vertices are displaced along the surface normal by a noise function (Sec. 6.1,
"Experimental setup").  Its noise model is not specified, so these scenes use
an i.i.d. uniform radial factor per unique vertex, which keeps every mesh
closed and watertight.

Layout produced for a scene with n particles:
  verts      float32 [sum_v, 3]  body-frame vertex coordinates, all particles
  vert_off   int64   [n+1]       vertex range of particle i
  tris       int32   [sum_t, 3]  vertex indices local to the particle, CCW
                                 seen from outside (outward normal)
  tri_off    int64   [n+1]       triangle range of particle i
  poses      float64 [n, 7]      world pose: translation xyz, quaternion wxyz
  mass       float64 [n]         (4/3) pi r^3 (unit density)
  com        float64 [n, 3]      body-frame centre of mass (the origin)
  pairs      int32   [P, 2]      particle indices (A, B)
  eps        float64 [P]         epsilon of the pair (both particles)
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

BASE_SEED = 2105124150


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------
def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
        [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
        [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
    ], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


@functools.lru_cache(maxsize=None)
def icosphere(level: int):
    """Unit icosphere after `level` midpoint subdivisions: 20*4^level faces.

    Returns (vertices float64 [nv,3] on the unit sphere, faces int32 [nf,3]).
    Shared edges get one midpoint vertex, so the mesh stays closed.
    """
    v, f = _icosahedron()
    for _ in range(level):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        key = np.sort(e, axis=1)
        uniq, inv = np.unique(key[:, 0] * (len(v) + 1) + key[:, 1], return_inverse=True)
        a = uniq // (len(v) + 1)
        b = uniq % (len(v) + 1)
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        nf = len(f)
        m = inv.reshape(3, nf).T + len(v)          # midpoint ids of edges 01,12,20
        v = np.concatenate([v, mid], axis=0)
        f = np.concatenate([
            np.stack([f[:, 0], m[:, 0], m[:, 2]], 1),
            np.stack([f[:, 1], m[:, 1], m[:, 0]], 1),
            np.stack([f[:, 2], m[:, 2], m[:, 1]], 1),
            np.stack([m[:, 0], m[:, 1], m[:, 2]], 1),
        ], axis=0)
    v.setflags(write=False)
    f = f.astype(np.int32)
    f.setflags(write=False)
    return v, f


def bumped_icosphere(level: int, radius: float, rng: np.random.Generator, amp: float = 0.05):
    """Icosphere of `radius` with each unique vertex scaled by U[1-amp, 1+amp]."""
    v, f = icosphere(level)
    s = rng.uniform(1.0 - amp, 1.0 + amp, size=len(v)) if amp > 0 else np.ones(len(v))
    return (v * (radius * s)[:, None]).astype(np.float32), f


# ----------------------------------------------------------------------------
# rigid motions
# ----------------------------------------------------------------------------
def random_quaternion(rng: np.random.Generator, n: int | None = None):
    """Uniform random unit quaternion(s) (w, x, y, z), Shoemake's method."""
    shape = () if n is None else (n,)
    u1, u2, u3 = (rng.random(shape) for _ in range(3))
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                  a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=-1)
    return q


def quat_to_matrix_f64(q):
    """Rotation matrix of unit quaternion(s) q = (w, x, y, z); float64."""
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def support(verts_f32, q, u):
    """max over vertices of (R(q) v) . u  (float64)."""
    R = quat_to_matrix_f64(q)
    return float(np.max(verts_f32.astype(np.float64) @ (R.T @ np.asarray(u, np.float64))))


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Scene:
    verts: np.ndarray
    vert_off: np.ndarray
    tris: np.ndarray
    tri_off: np.ndarray
    poses: np.ndarray
    mass: np.ndarray
    com: np.ndarray
    radius: np.ndarray
    pairs: np.ndarray
    eps: np.ndarray
    name: str = ""

    @property
    def n_particles(self):
        return len(self.vert_off) - 1

    @property
    def n_pairs(self):
        return len(self.pairs)

    def particle(self, i):
        v = self.verts[self.vert_off[i]:self.vert_off[i + 1]]
        t = self.tris[self.tri_off[i]:self.tri_off[i + 1]]
        return v, t

    def n_tri(self, i):
        return int(self.tri_off[i + 1] - self.tri_off[i])

    def subset(self, pair_ids, name=None):
        """Scene holding only the given pairs (and their particles, renumbered)."""
        pair_ids = np.asarray(pair_ids, dtype=np.int64)
        used = np.unique(self.pairs[pair_ids].reshape(-1))
        remap = -np.ones(self.n_particles, dtype=np.int64)
        remap[used] = np.arange(len(used))
        vs, ts, vo, to = [], [], [0], [0]
        for i in used:
            v, t = self.particle(i)
            vs.append(v)
            ts.append(t)
            vo.append(vo[-1] + len(v))
            to.append(to[-1] + len(t))
        return Scene(np.concatenate(vs), np.array(vo, np.int64), np.concatenate(ts),
                     np.array(to, np.int64), self.poses[used].copy(), self.mass[used].copy(),
                     self.com[used].copy(), self.radius[used].copy(),
                     remap[self.pairs[pair_ids]].astype(np.int32), self.eps[pair_ids].copy(),
                     name or (self.name + "-subset"))


def _assemble(meshes, poses, radius, pairs, eps, name):
    vs = [m[0] for m in meshes]
    ts = [m[1] for m in meshes]
    vo = np.zeros(len(meshes) + 1, np.int64)
    to = np.zeros(len(meshes) + 1, np.int64)
    vo[1:] = np.cumsum([len(v) for v in vs])
    to[1:] = np.cumsum([len(t) for t in ts])
    radius = np.ascontiguousarray(radius, np.float64)
    return Scene(np.ascontiguousarray(np.concatenate(vs), dtype=np.float32), vo,
                 np.ascontiguousarray(np.concatenate(ts), dtype=np.int32), to,
                 np.asarray(poses, np.float64), (4.0 / 3.0) * np.pi * radius ** 3,
                 np.zeros((len(meshes), 3)), radius,
                 np.asarray(pairs, np.int32).reshape(-1, 2), np.asarray(eps, np.float64), name)


def _place_pair(rng, mA, mB, gap, origin):
    """Pose A at `origin` and B along a random unit u such that A's extreme
    vertex along u and B's extreme vertex along -u lie on one line parallel to
    u, `gap` apart.  The two support planes are then `gap` apart, so for
    gap >= 0 the meshes' distance is exactly `gap` (reached by that vertex
    pair); a negative gap pushes the two vertices into each other."""
    qA, qB = random_quaternion(rng), random_quaternion(rng)
    u = _unit(rng)
    RA, RB = quat_to_matrix_f64(qA), quat_to_matrix_f64(qB)
    wA = mA[0].astype(np.float64) @ RA.T
    wB = mB[0].astype(np.float64) @ RB.T
    vA = wA[np.argmax(wA @ u)]
    vB = wB[np.argmax(wB @ -u)]
    tB = np.asarray(origin) + vA + gap * u - vB
    return np.concatenate([origin, qA]), np.concatenate([tB, qB])


def scene_pairs(levels_a, levels_b, radii_a, radii_b, eps, gaps, seed, name, amp=0.05, spread=50.0):
    """Generic batched scene: pair k uses particles 2k (A) and 2k+1 (B)."""
    rng = np.random.default_rng([BASE_SEED, seed])
    meshes, poses, radius, pairs = [], [], [], []
    for k in range(len(eps)):
        mA = bumped_icosphere(int(levels_a[k]), float(radii_a[k]), rng, amp)
        mB = bumped_icosphere(int(levels_b[k]), float(radii_b[k]), rng, amp)
        origin = rng.uniform(-spread, spread, size=3)
        pA, pB = _place_pair(rng, mA, mB, float(gaps[k]), origin)
        meshes += [mA, mB]
        poses += [pA, pB]
        radius += [radii_a[k], radii_b[k]]
        pairs.append((2 * k, 2 * k + 1))
    return _assemble(meshes, poses, radius, pairs, eps, name)


# Gap for the single-pair workload.  For two spheres of radius R at surface
# gap g (negative: interpenetration), the points of A within 2*eps of B form a
# cap of half-angle theta with R*theta^2 ~ 2*eps - g, whose area fraction is
# ~theta^2/4: a 5% patch needs 2*eps - g ~ 0.2 R by this estimate; on the
# seeded bumped meshes 0.25 R gives 5% of A's triangles in contact.
C1_EPS = 0.02
C1_GAP = 2 * C1_EPS - 0.25


def scene_c1(seed: int = 1):
    """One pair of bumped subdivision-3 icospheres (1280 triangles), R = 1,
    eps = 0.02, overlapping so that ~5% of A's triangles are in contact."""
    return scene_pairs([3], [3], [1.0], [1.0], [C1_EPS], [C1_GAP], seed, "c1-one-pair-1280")


def scene_c2(n_pairs: int = 4096, seed: int = 2):
    """Batched workload: subdivision U{1..5} per particle (80..20480 triangles),
    radius log-uniform in [0.1, 1], eps = 0.01 min(rA, rB), gap
    U[-0.5 eps, 3 eps] between the two closest (aligned extreme) vertices."""
    rng = np.random.default_rng([BASE_SEED, seed, 7])
    la = rng.integers(1, 6, size=n_pairs)
    lb = rng.integers(1, 6, size=n_pairs)
    ra = np.exp(rng.uniform(np.log(0.1), np.log(1.0), size=n_pairs))
    rb = np.exp(rng.uniform(np.log(0.1), np.log(1.0), size=n_pairs))
    eps = 0.01 * np.minimum(ra, rb)
    gaps = rng.uniform(-0.5, 3.0, size=n_pairs) * eps
    return scene_pairs(la, lb, ra, rb, eps, gaps, seed, f"c2-batched-{n_pairs}-pairs")


def scene_c3(n_pairs: int = 1024, seed: int = 3):
    """Differentiation workload: subdivision-4 icospheres (5120 triangles),
    R = 1, eps = 0.02, eps-environments overlapping by 0.3 eps: the meshes'
    distance is exactly 1.7 eps (no intersecting triangles)."""
    eps = np.full(n_pairs, 0.02)
    return scene_pairs(np.full(n_pairs, 4), np.full(n_pairs, 4), np.ones(n_pairs), np.ones(n_pairs),
                       eps, 1.7 * eps, seed, f"c3-grad-{n_pairs}-pairs")


def scene_tiny(n_pairs: int = 8, seed: int = 4, levels=(0, 1), amp=0.05):
    """Small meshes (icosahedron, 80-triangle sphere) for exhaustive checks."""
    rng = np.random.default_rng([BASE_SEED, seed, 11])
    la = rng.choice(levels, size=n_pairs)
    lb = rng.choice(levels, size=n_pairs)
    ra = rng.uniform(0.5, 1.0, size=n_pairs)
    rb = rng.uniform(0.5, 1.0, size=n_pairs)
    eps = 0.02 * np.minimum(ra, rb)
    gaps = rng.uniform(-2.0, 3.0, size=n_pairs) * eps
    return scene_pairs(la, lb, ra, rb, eps, gaps, seed, f"tiny-{n_pairs}", amp=amp)


def scene_regular_pair(level: int, radius: float, centre_dist: float, qA, qB, eps: float):
    """Two unbumped icospheres at a given centre distance along +x with given
    orientations; used for the closed-form mesh-distance checks."""
    v, f = icosphere(level)
    m = ((v * radius).astype(np.float32), f)
    pA = np.concatenate([[0.0, 0.0, 0.0], qA])
    pB = np.concatenate([[centre_dist, 0.0, 0.0], qB])
    return _assemble([m, m], [pA, pB], [radius, radius], [(0, 1)], [eps], "regular-pair")


def scene_particle_on_plane(levels=(3, 3, 4, 5), gaps=(-0.5, 0.3, 1.5, 2.5), eps: float = 0.01,
                            radius: float = 1.0, plane_inradius: float = 3.0, seed: int = 6,
                            amp: float = 0.05, spread: float = 50.0):
    """The particle-on-plane setup of Sec. 6: a bumped sphere-like particle
    over a tilted plane made of one large triangle (the paper notes that the
    plane's triangulation does not matter while its triangles are large next
    to the particle).  Pair k: particle 2k (subdivision levels[k], radius
    `radius`, random rotation) and plane 2k+1, an equilateral triangle of
    inradius `plane_inradius` (a body-frame triangle in the z = 0 plane,
    counter-clockwise seen from +z) with a random orientation whose +z side
    faces the particle.  The plane is placed gaps[k] * eps below the
    particle's lowest vertex along its normal, so for gaps >= 0 the meshes'
    distance is gaps[k] * eps; the particle's centre projects onto the
    triangle's centre.  eps is per pair (the paper uses 1e-2 relative to the
    particle diameter)."""
    rng = np.random.default_rng([BASE_SEED, seed, 13])
    a = 2.0 * plane_inradius  # circumradius
    tri_v = np.array([[a * np.cos(t), a * np.sin(t), 0.0]
                      for t in (np.pi / 2, np.pi / 2 + 2 * np.pi / 3, np.pi / 2 + 4 * np.pi / 3)])
    plane = (tri_v.astype(np.float32), np.array([[0, 1, 2]], np.int32))
    meshes, poses, radii, pairs, eps_l = [], [], [], [], []
    for k, (lv, g) in enumerate(zip(levels, gaps)):
        m = bumped_icosphere(int(lv), radius, rng, amp)
        qA = random_quaternion(rng)
        qP = random_quaternion(rng)
        RA, RP = quat_to_matrix_f64(qA), quat_to_matrix_f64(qP)
        n = RP[:, 2]  # the plane's normal in the world frame
        c = rng.uniform(-spread, spread, size=3)
        w = m[0].astype(np.float64) @ RA.T  # particle vertices relative to its centre
        h_min = float((w @ n).min())
        t_plane = c + (h_min - float(g) * eps) * n
        meshes += [m, plane]
        poses += [np.concatenate([c, qA]), np.concatenate([t_plane, qP])]
        radii += [radius, plane_inradius]
        pairs.append((2 * k, 2 * k + 1))
        eps_l.append(eps)
    return _assemble(meshes, poses, radii, pairs, eps_l, "particle-on-plane")


class _OverlapEnergy:
    """Soft-sphere overlap energy of spheres (centres c, radii R) in the cube
    [0, side]^3: E = 1/2 sum over overlapping pairs (R_i + R_j - |c_i - c_j|)^2
    plus 1/2 sum over wall penetrations (R_i - c_ik)^2 and (c_ik + R_i - side)^2,
    with its gradient.  Candidate pairs come from a neighbour list within
    R_i + R_j + skin, rebuilt when a centre has moved by half the skin.  Once
    every overlap is at most `slack` times its pair's radius sum (and every
    wall penetration `slack` times the radius) the energy reports zero with
    a zero gradient, which ends the minimisation there."""

    def __init__(self, R, side, skin, slack=0.0):
        self.R, self.side, self.skin, self.slack, self.ref = R, side, skin, slack, None

    def _neighbours(self, c):
        from scipy.spatial import cKDTree
        p = cKDTree(c).query_pairs(2.0 * self.R.max() + self.skin, output_type="ndarray")
        d = np.linalg.norm(c[p[:, 1]] - c[p[:, 0]], axis=1)
        p = p[d < self.R[p[:, 0]] + self.R[p[:, 1]] + self.skin]
        self.i0, self.i1 = p[:, 0], p[:, 1]
        self.S = self.R[self.i0] + self.R[self.i1]
        self.ref = c.copy()

    def __call__(self, x):
        c = x.reshape(-1, 3)
        n = len(c)
        if self.ref is None or np.abs(c - self.ref).max() > 0.5 * self.skin:
            self._neighbours(c)
        v = c[self.i1] - c[self.i0]
        d = np.sqrt((v * v).sum(1))
        ov = self.S - d
        lo = np.maximum(self.R[:, None] - c, 0.0)
        hi = np.maximum(c + self.R[:, None] - self.side, 0.0)
        lim = self.slack * self.R[:, None]
        if (ov <= self.slack * self.S).all() and (lo <= lim).all() and (hi <= lim).all():
            return 0.0, np.zeros(x.shape)
        m = ov > 0
        e = 0.5 * float((ov[m] ** 2).sum())
        f = (ov[m] / np.maximum(d[m], 1e-300))[:, None] * v[m]
        g = np.empty_like(c)
        for k in range(3):
            g[:, k] = (np.bincount(self.i0[m], f[:, k], n)
                       - np.bincount(self.i1[m], f[:, k], n))
        e += 0.5 * float((lo ** 2).sum() + (hi ** 2).sum())
        g += hi - lo
        return e, g.ravel()


def _spheres_disjoint(c, R, side):
    """True when no two spheres overlap and every sphere lies in the cube."""
    from scipy.spatial import cKDTree
    p = cKDTree(c).query_pairs(2.0 * R.max(), output_type="ndarray")
    d = np.linalg.norm(c[p[:, 1]] - c[p[:, 0]], axis=1)
    return bool((d >= R[p[:, 0]] + R[p[:, 1]]).all() and (c >= R[:, None]).all()
                and (c <= side - R[:, None]).all())


def _compress_packing(R, vol, fraction, rng, start=0.3, step=0.1, margin=1e-3):
    """Dense random packing of spheres of radii R (nominal volume `vol`) by
    compression with soft-sphere energy minimisation, the jamming protocol of
    O'Hern, Silbert, Liu and Nagel (Phys. Rev. E 68, 011306, 2003): uniform
    random centres in a cube sized for the volume fraction `start`, the
    overlap energy of the spheres inflated by (1 + margin) minimised
    (L-BFGS) until no inflated overlap exceeds half the margin; then the cube
    shrinks (centres mapped affinely) to the next fraction, `step` higher,
    up to `fraction`, minimising again each time.  Below the jamming fraction
    the minimum is zero and the true spheres end disjoint; the first stage
    that leaves them overlapping stops the compression.  Returns (centres,
    side) of the last disjoint stage."""
    from scipy.optimize import minimize
    fr = [f for f in np.arange(start, fraction - 1e-9, step)] + [fraction]
    sides = [(vol / f) ** (1.0 / 3.0) for f in fr]
    side = sides[0]
    c = rng.uniform(R[:, None], side - R[:, None], size=(len(R), 3))
    good = None
    for s_new in sides:
        span_old = np.maximum(side - 2.0 * R[:, None], 1e-12)
        c = R[:, None] + (c - R[:, None]) * (s_new - 2.0 * R[:, None]) / span_old
        side = s_new
        energy = _OverlapEnergy(R * (1.0 + margin), side, 0.3 * float(R.min()),
                                0.5 * margin / (1.0 + margin))
        res = minimize(energy, c.ravel(), jac=True, method="L-BFGS-B",
                       options=dict(maxiter=20000, maxfun=40000, ftol=0.0, gtol=1e-12,
                                    maxcor=20))
        c = res.x.reshape(-1, 3).copy()
        if not _spheres_disjoint(c, R, side):
            break
        good = (c, side)
    if good is None:
        raise ValueError(f"no disjoint packing of {len(R)} spheres at volume fraction {start}")
    return good


def scene_packing(n: int = 64, fraction: float = 0.3, levels=(2, 3, 4), r_min: float = 1.0,
                  r_max: float = 10.0, eps_rel: float = 0.01, overlap: float = 0.3,
                  seed: int = 10, amp: float = 0.05, tries_per_particle: int = 200,
                  method: str = "rsa"):
    """Many-particle packing (the implicit-step workload): n bumped
    sphere-like particles, subdivision uniform in `levels`, radius log-uniform
    in [r_min, r_max], in a cube sized for the requested volume fraction of
    the nominal spheres; a particle's bounding radius 1.05 r (its vertices lie
    within [0.95 r, 1.05 r]) may not overlap another particle's nor leave the
    cube.  method "rsa": random sequential addition, largest first; it jams
    well below dense packings, so when a particle finds no place in
    `tries_per_particle` attempts the cube grows by 1 % and the placement goes
    on.  method "compress": compression by soft-sphere energy minimisation
    (`_compress_packing`), which reaches dense random packings (0.55 of
    nominal spheres, 0.64 of bounding spheres, for 10 000 particles) and
    stops at the last disjoint stage below a jam.  Either way the achieved
    fraction is returned.  A share `overlap` of the particles is then moved
    towards its nearest neighbour until their bounding spheres overlap by
    eps / 2, so that contacts exist.  eps of a pair = eps_rel *
    min(diameters).  The scene's pair list is empty (pairs come from a broad
    phase).  Returns (scene, achieved fraction, velocities [n, 6] = (v,
    omega), zero)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng([BASE_SEED, seed, 17])
    radius = np.sort(np.exp(rng.uniform(np.log(r_min), np.log(r_max), size=n)))[::-1]
    R = 1.05 * radius
    vol = (4.0 / 3.0) * np.pi * (radius ** 3).sum()
    side = (vol / fraction) ** (1.0 / 3.0)
    if method == "compress":
        centres, side = _compress_packing(R, vol, fraction, rng)
        i = n
    elif method == "rsa":
        centres = np.zeros((n, 3))
        i = 0
    else:
        raise ValueError(f"unknown packing method {method!r}")
    tree, in_tree = None, 0
    while i < n:
        ok = False
        for _ in range(tries_per_particle):
            c = rng.uniform(R[i], side - R[i], size=3)
            near = list(range(in_tree, i))
            if tree is not None:
                near += tree.query_ball_point(c, R[i] + R[0])
            if not near or (np.linalg.norm(centres[near] - c, axis=1) >= R[near] + R[i]).all():
                ok = True
                break
        if not ok:
            side *= 1.01
            continue
        centres[i] = c
        i += 1
        if i - in_tree >= 64:
            tree, in_tree = cKDTree(centres[:i]), i
    meshes, poses = [], []
    for k in range(n):
        meshes.append(bumped_icosphere(int(rng.choice(levels)), float(radius[k]), rng, amp))
        poses.append(np.concatenate([centres[k], random_quaternion(rng)]))
    poses = np.array(poses)
    # bring some particles into contact with their nearest neighbour
    movers = rng.choice(n, size=int(overlap * n), replace=False) if n > 1 else []
    for k in movers:
        d = np.linalg.norm(poses[:, :3] - poses[k, :3], axis=1)
        d[k] = np.inf
        j = int(np.argmin(d))
        e = eps_rel * 2.0 * min(radius[k], radius[j])
        shift = d[j] - (R[k] + R[j] - 0.5 * e)
        if shift > 0:
            poses[k, :3] += shift * (poses[j, :3] - poses[k, :3]) / d[j]
    achieved = vol / side ** 3
    s = _assemble(meshes, poses, radius, np.zeros((0, 2), np.int32), np.zeros(0), "packing")
    return s, float(achieved), np.zeros((n, 6))


def scene_disparity(n_pairs: int = 64, level_big: int = 6, level_small: int = 3,
                    ratio: float = 20.0, eps_rel: float = 0.01, seed: int = 12, amp: float = 0.05):
    """Size-disparity pairs (the scale study of Sec. 6 and the many-particle
    scale workload): pair k holds a big particle (subdivision level_big,
    radius `ratio`) and a small one (subdivision level_small, radius 1), both
    bumped, random orientations, eps = eps_rel times the small diameter, gap
    U[-0.5 eps, 3 eps] between the two closest aligned extreme vertices."""
    rng = np.random.default_rng([BASE_SEED, seed, 19])
    eps = np.full(n_pairs, eps_rel * 2.0)
    gaps = rng.uniform(-0.5, 3.0, size=n_pairs) * eps
    return scene_pairs(np.full(n_pairs, level_big), np.full(n_pairs, level_small),
                       np.full(n_pairs, ratio), np.ones(n_pairs), eps, gaps, seed,
                       f"disparity-{n_pairs}-pairs-x{ratio:g}", amp=amp)


def scene_regular_disparate_pair(level_a: int, radius_a: float, level_b: int, radius_b: float,
                                 centre_dist: float, qA, qB, eps: float):
    """Two unbumped icospheres of different sizes and subdivisions at a given
    centre distance along +x; for closed-form distances."""
    va, fa = icosphere(level_a)
    vb, fb = icosphere(level_b)
    mA = ((va * radius_a).astype(np.float32), fa)
    mB = ((vb * radius_b).astype(np.float32), fb)
    pA = np.concatenate([[0.0, 0.0, 0.0], qA])
    pB = np.concatenate([[centre_dist, 0.0, 0.0], qB])
    return _assemble([mA, mB], [pA, pB], [radius_a, radius_b], [(0, 1)], [eps], "regular-disparate")


def scene_chain(k: int = 4, seed: int = 41, level: int = 2):
    """k bumped icospheres (radius U[1, 1.5]) in a chain: particle i sits
    along a random direction from particle i - 1 so that their extreme
    vertices along it are 0.5 eps apart (eps = 0.02 times the smaller largest
    coordinate), so every consecutive pair touches; the direction is drawn
    again while the new particle's bounding sphere comes within 4 eps of a
    particle other than its predecessor, so the consecutive pairs are the
    only contacts and no two meshes intersect.  No pairs listed (a broad
    phase supplies them)."""
    rng = np.random.default_rng([BASE_SEED, seed])
    meshes = [bumped_icosphere(level, float(rng.uniform(1.0, 1.5)), rng) for _ in range(k)]
    bound = [float(np.sqrt((m[0].astype(np.float64) ** 2).sum(1)).max()) for m in meshes]
    poses = [np.concatenate([[0.0, 0.0, 0.0], random_quaternion(rng)])]
    for i in range(1, k):
        e = 0.02 * min(np.abs(meshes[i - 1][0]).max(), np.abs(meshes[i][0]).max())
        wp = meshes[i - 1][0].astype(np.float64) @ quat_to_matrix_f64(poses[-1][3:]).T + poses[-1][:3]
        while True:
            u = _unit(rng)
            q = random_quaternion(rng)
            wc = meshes[i][0].astype(np.float64) @ quat_to_matrix_f64(q).T
            t = wp[np.argmax(wp @ u)] + 0.5 * e * u - wc[np.argmax(wc @ -u)]
            if all(np.linalg.norm(t - poses[j][:3]) > bound[i] + bound[j] + 4 * e for j in range(i - 1)):
                break
        poses.append(np.concatenate([t, q]))
    radius = [float(np.linalg.norm(m[0], axis=1).mean()) for m in meshes]
    return _assemble(meshes, poses, radius, np.zeros((0, 2), np.int32), np.zeros(0), "chain")



def scene_scale(n_small: int = 100000, n_big: int = 100, level_small: int = 3,
                level_big: int = 6, ratio: float = 20.0, fraction: float = 0.3,
                eps_rel: float = 0.01, overlap: float = 0.3, seed: int = 23,
                amp: float = 0.05, tries_per_particle: int = 200):
    """Scale workload (the many-particle scale study of Sec. 6): n_big bumped
    icospheres of subdivision level_big and radius `ratio` among n_small of
    subdivision level_small and radius 1, random orientations, placed by
    random sequential addition (the big ones first) in a cube sized for the
    requested volume fraction, growing by 1 % when a particle finds no place
    (bounding radius 1.05 r); then a share `overlap` of the particles moves
    towards its nearest neighbour until their bounding spheres overlap by
    eps / 2, eps = eps_rel * min(diameters).  No pairs listed (a broad phase
    supplies them).  Returns (scene, achieved fraction)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng([BASE_SEED, seed, 29])
    n = n_big + n_small
    radius = np.concatenate([np.full(n_big, float(ratio)), np.ones(n_small)])
    R = 1.05 * radius
    side = ((4.0 / 3.0) * np.pi * (radius ** 3).sum() / fraction) ** (1.0 / 3.0)
    centres = np.zeros((n, 3))

    def place(lo, hi, reach):
        """Places particles lo..hi-1 (equal radius) avoiding the ones before."""
        nonlocal side
        big_tree = cKDTree(centres[:n_big]) if lo >= n_big and n_big else None
        tree, in_tree = None, lo
        i = lo
        while i < hi:
            ok = False
            for _ in range(tries_per_particle):
                c = rng.uniform(R[i], side - R[i], size=3)
                near = list(range(in_tree, i))
                if tree is not None:
                    near += [lo + k for k in tree.query_ball_point(c, 2 * R[i])]
                if big_tree is not None:
                    near += big_tree.query_ball_point(c, R[i] + R[0])
                if lo < n_big:
                    near = list(range(lo, i))
                if not near or (np.linalg.norm(centres[near] - c, axis=1) >= R[near] + R[i]).all():
                    ok = True
                    break
            if not ok:
                side *= 1.01
                continue
            centres[i] = c
            i += 1
            if i - in_tree >= 256:
                tree, in_tree = cKDTree(centres[lo:i]), i
        return reach

    place(0, n_big, R[0])
    place(n_big, n, R[n_big])
    meshes = [bumped_icosphere(level_big if k < n_big else level_small, float(radius[k]), rng, amp)
              for k in range(n)]
    quats = random_quaternion(rng, n)
    poses = np.concatenate([centres, quats], 1)
    # bring some particles into contact with their nearest neighbour
    tree = cKDTree(centres)
    movers = rng.choice(n, size=int(overlap * n), replace=False) if n > 1 else []
    for k in movers:
        dist, idx = tree.query(poses[k, :3], k=2)
        j = int(idx[1])
        d = float(np.linalg.norm(poses[j, :3] - poses[k, :3]))
        e = eps_rel * 2.0 * min(radius[k], radius[j])
        shift = d - (R[k] + R[j] - 0.5 * e)
        if shift > 0 and d > 0:
            poses[k, :3] += shift * (poses[j, :3] - poses[k, :3]) / d
    achieved = (4.0 / 3.0) * np.pi * (radius ** 3).sum() / side ** 3
    s = _assemble(meshes, list(poses), list(radius), np.zeros((0, 2), np.int32), np.zeros(0),
                  "scale")
    return s, float(achieved)
