"""Pins of the oracle's contact set (Algorithm 2 with the contact criterion
d <= 2 eps of Definition "contact point") against closed-form mesh distances,
an exhaustive KKT brute force on tiny meshes and invariants."""
import numpy as np
import pytest

from gen import icosphere, quat_to_matrix_f64, random_quaternion, scene_regular_pair, scene_tiny
from tests.kkt_reference import kkt_distance


def _quat_from_matrix(R):
    # Shepperd's method; good enough for building test poses
    w = np.sqrt(max(0.0, 1 + R[0, 0] + R[1, 1] + R[2, 2])) / 2
    x = np.sqrt(max(0.0, 1 + R[0, 0] - R[1, 1] - R[2, 2])) / 2
    y = np.sqrt(max(0.0, 1 - R[0, 0] + R[1, 1] - R[2, 2])) / 2
    z = np.sqrt(max(0.0, 1 - R[0, 0] - R[1, 1] + R[2, 2])) / 2
    x = np.copysign(x, R[2, 1] - R[1, 2])
    y = np.copysign(y, R[0, 2] - R[2, 0])
    z = np.copysign(z, R[1, 0] - R[0, 1])
    q = np.array([w, x, y, z])
    return q / np.linalg.norm(q)


def _rotation_taking(a, b):
    """A rotation matrix mapping unit vector a onto unit vector b."""
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    v = np.cross(a, b)
    c = float(a @ b)
    if np.linalg.norm(v) < 1e-12:
        if c > 0:
            return np.eye(3)
        p = np.array([1.0, 0, 0]) if abs(a[0]) < 0.9 else np.array([0, 1.0, 0])
        v = np.cross(a, p)
        v /= np.linalg.norm(v)
        return 2 * np.outer(v, v) - np.eye(3)
    K = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + K + K @ K / (1 + c)


def _min_distance(orc, scene, eps_big):
    c = orc.detect(scene, eps=np.array([eps_big]))
    assert len(c["d"]) > 0
    return c["d"].min()


@pytest.mark.parametrize("level", [0, 1, 2])
def test_regular_icospheres_vertex_aligned(orc, level):
    """Vertex of A on +x, vertex of B on -x: distance D - |vA| - |vB|."""
    v, f = icosphere(level)
    R = 1.0
    vf = (v * R).astype(np.float32).astype(np.float64)
    ia, ib = 0, 5
    qA = _quat_from_matrix(_rotation_taking(vf[ia], np.array([1.0, 0, 0])))
    qB = _quat_from_matrix(_rotation_taking(vf[ib], np.array([-1.0, 0, 0])))
    D = 2.3
    s = scene_regular_pair(level, R, D, qA, qB, eps=0.5)
    # the axis vertices after the (FP64) pose rotation
    RA, RB = quat_to_matrix_f64(qA), quat_to_matrix_f64(qB)
    xa = RA @ vf[ia]
    xb = RB @ vf[ib] + np.array([D, 0, 0])
    expected = np.linalg.norm(xb - xa)
    assert abs(_min_distance(orc, s, 0.5) - expected) < 1e-12


@pytest.mark.parametrize("level", [0, 1, 2])
def test_regular_icospheres_face_aligned(orc, level):
    """Face of A facing +x, face of B facing -x, both centred on the axis:
    D - rf_A - rf_B with rf the face-plane distance (FP64 from the stored
    float32 vertices)."""
    v, f = icosphere(level)
    vf = v.astype(np.float32).astype(np.float64)
    fa, fb = 0, len(f) // 2

    def setup(fi, target):
        T = vf[f[fi]]
        n = np.cross(T[1] - T[0], T[2] - T[0])
        n /= np.linalg.norm(n)
        rf = float(n @ T[0])
        Rm = _rotation_taking(n, target)
        return _quat_from_matrix(Rm), rf

    qA, rfA = setup(fa, np.array([1.0, 0, 0]))
    qB, rfB = setup(fb, np.array([-1.0, 0, 0]))
    # the foot of the perpendicular from each centre onto its face plane is
    # the face's circumcentre (vertices lie on the sphere), which is on the x
    # axis after the rotations and inside the (acute) face
    D = 2.2
    s = scene_regular_pair(level, 1.0, D, qA, qB, eps=0.5)
    expected = D - rfA - rfB
    got = _min_distance(orc, s, 0.5)
    assert abs(got - expected) < 1e-12, (got, expected)


@pytest.mark.parametrize("level", [0, 1])
def test_regular_icospheres_vertex_to_face(orc, level):
    v, f = icosphere(level)
    vf = v.astype(np.float32).astype(np.float64)
    T = vf[f[3]]
    n = np.cross(T[1] - T[0], T[2] - T[0])
    n /= np.linalg.norm(n)
    rf = float(n @ T[0])
    qA = _quat_from_matrix(_rotation_taking(vf[7], np.array([1.0, 0, 0])))
    qB = _quat_from_matrix(_rotation_taking(n, np.array([-1.0, 0, 0])))
    D = 2.1
    s = scene_regular_pair(level, 1.0, D, qA, qB, eps=0.5)
    xa = quat_to_matrix_f64(qA) @ vf[7]
    expected = D - rf - np.linalg.norm(xa)
    assert abs(_min_distance(orc, s, 0.5) - expected) < 1e-12


def test_tiny_meshes_exhaustive(orc):
    """Every triangle pair of tiny meshes: the oracle's contact set equals the
    set of pairs whose KKT-enumerated distance is <= 2 eps (outside a 1e-9
    band around the threshold)."""
    s = scene_tiny(n_pairs=6, levels=(0, 1))
    c = orc.detect(s)
    for p in range(s.n_pairs):
        A, B = s.pairs[p]
        TA = orc.world_triangles(s, A)
        TB = orc.world_triangles(s, B)
        I, J = np.meshgrid(np.arange(len(TA)), np.arange(len(TB)), indexing="ij")
        dk = kkt_distance(TA[I.ravel()], TB[J.ravel()])
        tau = 2 * s.eps[p]
        sel = c["pair"] == p
        got = set(zip(c["ta"][sel].tolist(), c["tb"][sel].tolist()))
        band = np.abs(dk - tau) <= 1e-9
        exp = set(zip(I.ravel()[(dk <= tau) & ~band].tolist(), J.ravel()[(dk <= tau) & ~band].tolist()))
        amb = set(zip(I.ravel()[band].tolist(), J.ravel()[band].tolist()))
        assert exp <= got and got <= exp | amb
        # distances agree with the enumeration
        lut = dict(zip(zip(I.ravel().tolist(), J.ravel().tolist()), dk.tolist()))
        for ta, tb, d in zip(c["ta"][sel], c["tb"][sel], c["d"][sel]):
            assert abs(lut[(int(ta), int(tb))] - d) < 1e-9


def test_swap_and_rigid_motion_invariance(orc):
    s = scene_tiny(n_pairs=8, levels=(1, 2), seed=9)
    c = orc.detect(s)
    # swapping A and B gives the same set with roles swapped
    c2 = orc.detect(s, pairs=s.pairs[:, ::-1].copy())
    a = sorted(zip(c["pair"], c["ta"], c["tb"]))
    b = sorted(zip(c2["pair"], c2["tb"], c2["ta"]))
    assert a == b
    m1 = {(p, i, j): d for p, i, j, d in zip(c["pair"], c["ta"], c["tb"], c["d"])}
    for p, i, j, d in zip(c2["pair"], c2["tb"], c2["ta"], c2["d"]):
        assert abs(m1[(p, i, j)] - d) < 1e-12
    # a common rigid motion of all particles changes nothing
    rng = np.random.default_rng(0)
    qm = random_quaternion(rng)
    Rm = quat_to_matrix_f64(qm)
    tm = rng.normal(size=3) * 5
    poses = s.poses.copy()
    for i in range(s.n_particles):
        poses[i, :3] = Rm @ s.poses[i, :3] + tm
        w1, v1 = qm[0], qm[1:]
        w2, v2 = s.poses[i, 3], s.poses[i, 4:]
        poses[i, 3] = w1 * w2 - v1 @ v2
        poses[i, 4:] = w1 * v2 + w2 * v1 + np.cross(v1, v2)
    c3 = orc.detect(s, poses=poses)
    assert sorted(zip(c3["pair"], c3["ta"], c3["tb"])) == sorted(zip(c["pair"], c["ta"], c["tb"]))
    for p, i, j, d in zip(c3["pair"], c3["ta"], c3["tb"], c3["d"]):
        assert abs(m1[(p, i, j)] - d) < 1e-11


def test_particle_on_plane_closed_form(orc):
    """Particle-on-plane (Sec. 6): against one large plane triangle, a
    particle triangle's distance is a closed form of its vertices' heights h
    over the plane: 0 if they change sign, else min |h| (the nearest vertex
    projects inside the plane triangle).  The contact set and distances of
    the oracle match it; the gap-2.5 eps pair has no contacts."""
    from gen import scene_particle_on_plane
    s = scene_particle_on_plane()
    c = orc.detect(s)
    for k in range(s.n_pairs):
        A, B = s.pairs[k]
        WA = orc.world_triangles(s, A).reshape(-1, 3, 3)
        WP = orc.world_triangles(s, B).reshape(3, 3)
        nrm = np.cross(WP[1] - WP[0], WP[2] - WP[0])
        nrm /= np.linalg.norm(nrm)
        h = (WA - WP[0]) @ nrm
        d = np.where((h.min(1) <= 0) & (h.max(1) >= 0), 0.0, np.abs(h).min(1))
        want = np.flatnonzero(d <= 2 * s.eps[k])
        sel = c["pair"] == k
        got = np.sort(c["ta"][sel])
        band = np.flatnonzero(np.abs(d - 2 * s.eps[k]) <= 1e-9)
        assert set(got) ^ set(want) <= set(band), k
        dd = dict(zip(c["ta"][sel].tolist(), c["d"][sel].tolist()))
        for t in set(got) & set(want):
            assert abs(dd[t] - d[t]) <= 1e-12 * (1 + np.abs(WA).max()), (k, t, dd[t], d[t])
        assert (c["tb"][sel] == 0).all()
    counts = np.bincount(c["pair"], minlength=s.n_pairs)
    assert counts[3] == 0 and counts[:3].min() > 0


@pytest.mark.parametrize("la,ra,lb,rb", [(4, 20.0, 1, 1.0), (3, 8.0, 0, 1.0), (1, 1.0, 3, 4.0)])
def test_size_disparity_vertex_aligned(orc, la, ra, lb, rb):
    """Size disparity (Sec. 6, Tables 7 and 8): a vertex of a large regular
    icosphere facing a vertex of a small one along x: the distance is the
    distance of the two vertices; the brute force finds exactly that."""
    from gen import scene_regular_disparate_pair
    va, _ = icosphere(la)
    vb, _ = icosphere(lb)
    xa0 = (va[0] * ra).astype(np.float32).astype(np.float64)
    xb0 = (vb[5] * rb).astype(np.float32).astype(np.float64)
    qA = _quat_from_matrix(_rotation_taking(xa0, np.array([1.0, 0, 0])))
    qB = _quat_from_matrix(_rotation_taking(xb0, np.array([-1.0, 0, 0])))
    D = ra + rb + 0.3
    s = scene_regular_disparate_pair(la, ra, lb, rb, D, qA, qB, eps=0.5)
    xa = quat_to_matrix_f64(qA) @ xa0
    xb = quat_to_matrix_f64(qB) @ xb0 + np.array([D, 0, 0])
    expected = np.linalg.norm(xb - xa)
    c = orc.detect(s)
    assert len(c["d"]) > 0
    assert abs(c["d"].min() - expected) < 1e-12 * max(1.0, ra)
    # a vertex against a vertex: the minimum is attained by the triangle
    # pairs around the two axis vertices only
    fa = icosphere(la)[1]
    fb = icosphere(lb)[1]
    at_min = np.abs(c["d"] - expected) < 1e-9
    assert set(c["ta"][at_min]) <= set(np.flatnonzero((fa == 0).any(1)))
    assert set(c["tb"][at_min]) <= set(np.flatnonzero((fb == 5).any(1)))
