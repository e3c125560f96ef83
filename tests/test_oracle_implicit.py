"""Pins of the implicit-step oracle (Algorithm 3 with the force law of
Sec. 2) and of its broad phase, against closed forms, an independent
library search and invariants."""
import numpy as np
import pytest

from gen import quat_to_matrix_f64, scene_packing


@pytest.fixture(scope="module")
def imp():
    import oracle
    oracle.build()
    from oracle import implicit
    return implicit


def test_broad_phase_matches_kdtree(imp):
    from scipy.spatial import cKDTree
    s, _, _ = scene_packing(300, 0.3, seed=21)
    c = s.poses[:, :3]
    bound = imp.bounding_radius(s)
    got = imp.broad_phase(c, bound, s.radius)
    lim_max = 2 * bound.max() + 2 * 0.02 * s.radius.max()
    cand = np.array(sorted(cKDTree(c).query_pairs(lim_max)))
    i, j = cand[:, 0], cand[:, 1]
    d = np.linalg.norm(c[i] - c[j], axis=1)
    keep = d <= bound[i] + bound[j] + 2 * imp.pair_eps(s.radius, i, j)
    want = cand[keep]
    assert len(got) > 0
    np.testing.assert_array_equal(got, want[np.lexsort((want[:, 1], want[:, 0]))])


def test_broad_phase_lattice_closed_form(imp):
    """Unit spheres on a k x k x k cubic lattice of spacing 2 + eps: each
    pair of face neighbours touches within 2 eps, diagonal neighbours do not;
    3 k^2 (k - 1) pairs."""
    k = 5
    g = np.arange(k) * 2.015
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ones = np.ones(len(c))
    got = imp.broad_phase(c, ones, ones)   # eps = 0.02 per pair
    assert len(got) == 3 * k * k * (k - 1)
    assert np.allclose(np.linalg.norm(c[got[:, 0]] - c[got[:, 1]], axis=1), 2.015)


def _single(levels=2, radius=1.0):
    s, _, _ = scene_packing(1, 0.1, levels=(levels,), r_min=radius, r_max=radius, seed=3)
    return s


def test_free_flight_closed_form(imp):
    """No contacts: v' = v + dt g, c' = c + dt v', q' = exp(dt omega) q; the
    first update is the fixed point (the second iteration only confirms
    it)."""
    s = _single()
    vel = np.array([[0.3, -0.2, 1.0, 0.5, -1.5, 2.0]])
    dt = 1e-3
    poses, v, it, _ = imp.implicit_euler_step(s, vel, np.zeros((0, 2)), np.zeros(0), dt)
    assert it == 2
    v_want = vel[0, :3] + dt * imp.G_DEFAULT
    np.testing.assert_allclose(v[0, :3], v_want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(v[0, 3:], vel[0, 3:], rtol=0, atol=0)
    np.testing.assert_allclose(poses[0, :3], s.poses[0, :3] + dt * v_want, rtol=0, atol=1e-13)
    # orientation: rotation by dt omega about the world axis omega/|omega|
    w = vel[0, 3:]
    th = dt * np.linalg.norm(w)
    ax = w / np.linalg.norm(w)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rw = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    R0 = quat_to_matrix_f64(s.poses[0, 3:])
    np.testing.assert_allclose(quat_to_matrix_f64(poses[0, 3:]), Rw @ R0, rtol=0, atol=1e-14)


def _colliding_pair(imp, seed=4):
    """Two particles whose meshes are within 2 eps of each other (placed by
    the pair generator at gap 0.5 eps), approaching each other."""
    from gen import scene_pairs
    e = 0.02 * 1.0
    s = scene_pairs([2], [2], [1.0], [1.2], [e], [0.5 * e], seed, "colliding", spread=5.0)
    bound = imp.bounding_radius(s)
    pairs = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    assert pairs.tolist() == [[0, 1]]
    eps = imp.pair_eps(s.radius, pairs[:, 0], pairs[:, 1])
    assert np.allclose(eps, e)
    u = s.poses[1, :3] - s.poses[0, :3]
    u /= np.linalg.norm(u)
    vel = np.zeros((2, 6))
    vel[0, :3] = 0.2 * u
    vel[1, :3] = -0.1 * u
    vel[:, 3:] = [[0.0, 0.3, -0.2], [0.1, 0.0, 0.4]]
    return s, vel, pairs, eps


def test_momentum_balance_and_convergence(imp):
    """Contact forces are equal and opposite: the total momentum changes by
    dt * sum(m) g exactly (rounding aside), and the Picard iteration
    contracts to a fixed point."""
    s, vel, pairs, eps = _colliding_pair(imp)
    import oracle
    c = oracle.detect(s.__class__(**{**s.__dict__, "pairs": pairs, "eps": eps}))
    assert len(c["d"]) > 0   # the pair is in contact at the start
    dt = 2e-4
    _, v, it, hist = imp.implicit_euler_step(s, vel, pairs, eps, dt)
    assert 1 < it < 200 and hist[-1] <= 1e-13
    m = s.mass
    p0 = (m[:, None] * vel[:, :3]).sum(0) + dt * m.sum() * imp.G_DEFAULT
    p1 = (m[:, None] * v[:, :3]).sum(0)
    assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(m[:, None] * vel[:, :3]).sum()
    # the contact pushed them apart: the approach speed dropped
    u = s.poses[1, :3] - s.poses[0, :3]
    assert (v[0, :3] - v[1, :3]) @ u < (vel[0, :3] - vel[1, :3]) @ u


def test_galilean_and_rotation_invariance(imp):
    """A uniform extra velocity adds to every result velocity; rotating the
    scene, its velocities and gravity rotates the result."""
    s, vel, pairs, eps = _colliding_pair(imp, seed=6)
    dt = 2e-4
    P, V, _, _ = imp.implicit_euler_step(s, vel, pairs, eps, dt)
    w = np.array([0.05, -0.02, 0.01])
    vel2 = vel.copy()
    vel2[:, :3] += w
    P2, V2, _, _ = imp.implicit_euler_step(s, vel2, pairs, eps, dt)
    np.testing.assert_allclose(V2[:, :3] - w, V[:, :3], rtol=0, atol=1e-9)
    np.testing.assert_allclose(V2[:, 3:], V[:, 3:], rtol=0, atol=1e-9)
    # rotation of everything
    th = 0.7
    Q = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    Q = Q @ quat_to_matrix_f64(np.array([0.9, 0.1, -0.3, 0.2]) / np.linalg.norm([0.9, 0.1, -0.3, 0.2]))
    qQ = _quat_of(Q)
    s3 = s.__class__(**s.__dict__)
    s3.poses = s.poses.copy()
    for i in range(s.n_particles):
        s3.poses[i, :3] = Q @ s.poses[i, :3]
        s3.poses[i, 3:] = _qmul(qQ, s.poses[i, 3:])
    vel3 = np.concatenate([vel[:, :3] @ Q.T, vel[:, 3:] @ Q.T], 1)
    P3, V3, _, _ = imp.implicit_euler_step(s3, vel3, pairs, eps, dt, g=Q @ imp.G_DEFAULT)
    np.testing.assert_allclose(V3[:, :3], V[:, :3] @ Q.T, rtol=0, atol=1e-9)
    np.testing.assert_allclose(V3[:, 3:], V[:, 3:] @ Q.T, rtol=0, atol=1e-9)
    np.testing.assert_allclose(P3[:, :3], P[:, :3] @ Q.T, rtol=0, atol=1e-9)


def _quat_of(R):
    w = np.sqrt(max(0.0, 1 + R[0, 0] + R[1, 1] + R[2, 2])) / 2
    x = np.copysign(np.sqrt(max(0.0, 1 + R[0, 0] - R[1, 1] - R[2, 2])) / 2, R[2, 1] - R[1, 2])
    y = np.copysign(np.sqrt(max(0.0, 1 - R[0, 0] + R[1, 1] - R[2, 2])) / 2, R[0, 2] - R[2, 0])
    z = np.copysign(np.sqrt(max(0.0, 1 - R[0, 0] - R[1, 1] + R[2, 2])) / 2, R[1, 0] - R[0, 1])
    q = np.array([w, x, y, z])
    return q / np.linalg.norm(q)


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_angular_momentum_identity(imp):
    """Each contact applies +F and -F at one point, so over an implicit Euler
    step the total angular momentum about the origin,
    L = sum c_i x m_i v_i + I_i omega_i, obeys
    L' = L + dt sum c_i x m_i g - dt^2 sum v'_i x F_i
    (F_i the total contact force on i at the end of the step): exact up to
    rounding, so it pins the torques, the inertia and the rotation update."""
    import dataclasses

    import oracle
    s, vel, pairs, eps = _colliding_pair(imp, seed=8)
    dt = 5e-4
    P, V, it, _ = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=1e-15)
    m = s.mass
    inertia = 0.4 * m * s.radius ** 2
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((2, 3)))
    c = oracle.detect(base, poses=P)
    assert len(c["d"]) > 0
    ft, _ = oracle.forces(base, c, poses=P)
    F = ft[:, :3]
    c0 = s.poses[:, :3]
    L0 = (np.cross(c0, m[:, None] * vel[:, :3]) + inertia[:, None] * vel[:, 3:]).sum(0)
    L1 = (np.cross(P[:, :3], m[:, None] * V[:, :3]) + inertia[:, None] * V[:, 3:]).sum(0)
    want = L0 + dt * np.cross(c0, m[:, None] * imp.G_DEFAULT).sum(0) - dt ** 2 * np.cross(V[:, :3], F).sum(0)
    scale = np.abs(np.cross(c0, m[:, None] * vel[:, :3])).sum() + np.abs(inertia[:, None] * vel[:, 3:]).sum()
    assert np.abs(L1 - want).max() <= 1e-11 * scale, (L1 - want, scale)
    # a wrong inertia would break it
    L1_bad = (np.cross(P[:, :3], m[:, None] * V[:, :3]) + 1.1 * inertia[:, None] * V[:, 3:]).sum(0)
    assert np.abs(L1_bad - want).max() > 1e-6 * scale


@pytest.mark.parametrize("seed", [4, 6, 8])
def test_newton_and_picard_reach_the_same_step(imp, seed):
    """Two different solvers of the implicit Euler equations, the paper's
    Picard iteration and Newton's method with the Gauss-Newton contact
    stiffness, converge to the same velocities and poses.  (Both converge
    linearly here: the Gauss-Newton blocks leave out the negative tangential
    stiffness e'(d) Hess(d) of vertex and edge contacts.)"""
    s, vel, pairs, eps = _colliding_pair(imp, seed=seed)
    dt = 5e-4
    # Picard stops at its rounding floor (about 5e-14 change per iteration)
    P1, V1, it1, hist = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=2e-13, max_iter=1000)
    P2, V2, it2 = imp.implicit_euler_step_newton(s, vel, pairs, eps, dt, tol=1e-12, max_iter=1000)
    assert it1 < 1000 and it2 < 1000, (it1, it2)
    scale = np.abs(V1).max()
    assert np.abs(V1 - V2).max() <= 1e-10 * scale, (np.abs(V1 - V2).max(), scale, it1, it2)
    np.testing.assert_allclose(P2[:, :3], P1[:, :3], rtol=0, atol=1e-12)


def test_pose_hessian_vertex_against_vertex_closed_form(imp):
    """Two regular icosahedra tip to tip (every contact between the triangles
    around the two tips has the tips as closest points): the translation
    block of the energy's Hessian is 25 (e'' u u^T + e' (I - u u^T) / d),
    e' = -K_s sqrt(mu) (1 - d/(2 eps)), e'' = K_s sqrt(mu) / (2 eps); the
    Gauss-Newton block has only the first term."""
    import oracle
    from gen import icosphere, scene_regular_pair
    from tests.test_oracle_contacts import _quat_from_matrix, _rotation_taking
    v, f = icosphere(0)
    qA = _quat_from_matrix(_rotation_taking(v[0], np.array([1.0, 0, 0])))
    qB = _quat_from_matrix(_rotation_taking(v[3], np.array([-1.0, 0, 0])))
    s = scene_regular_pair(0, 1.0, 2.06, qA, qB, 0.05)
    c = oracle.detect(s)
    assert len(c["d"]) == 25
    H = imp.pose_hessian(s, s.poses, s.pairs, s.eps)
    d = float(c["d"][0])
    u = (c["pa"][0] - c["pb"][0]) / d
    ks = 1000.0 * np.sqrt(1 / (1 / s.mass[0] + 1 / s.mass[1]))
    e1 = -ks * (1 - d / (2 * s.eps[0]))
    e2 = ks / (2 * s.eps[0])
    want = 25 * (e2 * np.outer(u, u) + e1 * (np.eye(3) - np.outer(u, u)) / d)
    np.testing.assert_allclose(H[0:3, 0:3], want, rtol=0, atol=1e-5 * np.abs(want).max())
    np.testing.assert_allclose(H[6:9, 6:9], want, rtol=0, atol=1e-5 * np.abs(want).max())
    np.testing.assert_allclose(H[0:3, 6:9], -want, rtol=0, atol=1e-5 * np.abs(want).max())
    _, _, jac = oracle.grad(s, c)
    np.testing.assert_allclose(jac[0][0:3, 0:3], 25 * e2 * np.outer(u, u), rtol=1e-9, atol=1e-9)


def test_newton_with_the_full_hessian_converges_fast(imp):
    """With the full pose Hessian as stiffness, Newton's method converges in
    a handful of iterations to the Picard fixed point."""
    s, vel, pairs, eps = _colliding_pair(imp, seed=8)
    dt = 5e-4
    _, V1, it1, _ = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=2e-13, max_iter=1000)
    _, V2, it2 = imp.implicit_euler_step_newton(s, vel, pairs, eps, dt, tol=1e-12, max_iter=50,
                                                stiffness="hessian")
    assert it2 <= 8, it2
    assert np.abs(V1 - V2).max() <= 1e-9 * np.abs(V1).max()


def test_packing_generator():
    """Every requested particle is placed; the achieved volume fraction is
    stated (random sequential addition jams below dense packings); the
    particles moved towards a neighbour give overlapping bounding spheres;
    the same seed gives the same scene."""
    s, frac, vel = scene_packing(400, 0.5, seed=31)
    assert s.n_particles == 400 and vel.shape == (400, 6)
    r = s.radius
    vol = (4.0 / 3.0) * np.pi * (r ** 3).sum()
    c = s.poses[:, :3]
    side_est = (vol / frac) ** (1 / 3)
    assert 0 < frac <= 0.5 and np.ptp(c, axis=0).max() <= side_est * 1.0001
    d = np.linalg.norm(c[:, None] - c[None], axis=-1) + np.eye(400) * 1e9
    overlap = (d < 1.05 * (r[:, None] + r[None])).any(1)
    assert overlap.sum() >= 0.2 * 400 * 0.5
    s2, frac2, _ = scene_packing(400, 0.5, seed=31)
    assert frac2 == frac and np.array_equal(s2.poses, s.poses) and np.array_equal(s2.verts, s.verts)


def test_packing_generator_compressed():
    """The compressed packing (soft-sphere energy minimisation) reaches a
    denser packing than random sequential addition on the same particles,
    with every bounding sphere (1.05 r, which holds every vertex) disjoint
    from the others and inside the cube, and the stated fraction equal to the
    nominal spheres' volume over the cube's."""
    n = 400
    s, frac, _ = scene_packing(n, 0.55, seed=31, overlap=0.0, method="compress")
    _, frac_rsa, _ = scene_packing(n, 0.55, seed=31, overlap=0.0)
    assert frac >= frac_rsa + 0.1 and frac <= 0.55 + 1e-12, (frac, frac_rsa)
    r, c = s.radius, s.poses[:, :3]
    vmax = np.array([np.linalg.norm(s.particle(i)[0].astype(np.float64), axis=1).max()
                     for i in range(n)])
    assert (vmax <= 1.05 * r * (1 + 1e-6)).all()
    side = ((4.0 / 3.0) * np.pi * (r ** 3).sum() / frac) ** (1 / 3)
    R = 1.05 * r
    d = np.linalg.norm(c[:, None] - c[None], axis=-1) + np.eye(n) * 1e9
    assert (d >= R[:, None] + R[None]).all()
    assert (c >= R[:, None] * (1 - 1e-12)).all() and (c <= side - R[:, None] * (1 - 1e-12)).all()
    with pytest.raises(ValueError):
        scene_packing(8, 0.3, method="lattice")


def test_packing_overlap_energy_gradient():
    """The compression's soft-sphere energy (gen.icosphere._OverlapEnergy)
    returns its own gradient: central differences agree on a small
    overlapping configuration with wall contacts, and the energy reports zero
    once every overlap is within the slack."""
    from gen.icosphere import _OverlapEnergy
    rng = np.random.default_rng(3)
    R = rng.uniform(0.5, 2.0, size=12)
    x = rng.uniform(0.0, 6.0, size=(12, 3)).ravel()
    en = _OverlapEnergy(R, 6.0, 0.5)
    e0, g = en(x)
    assert e0 > 0
    h = 1e-6
    fd = np.array([(en(x + h * np.eye(len(x))[i])[0] - en(x - h * np.eye(len(x))[i])[0]) / (2 * h)
                   for i in range(len(x))])
    assert np.abs(fd - g).max() <= 1e-6 * max(1.0, np.abs(g).max())
    far = np.array([[10.0 * i + 3.0, 3.0, 3.0] for i in range(3)]).ravel()
    e1, g1 = _OverlapEnergy(np.full(3, 1.0), 40.0, 0.5, slack=1e-3)(far)
    assert e1 == 0.0 and not g1.any()


def test_disparity_generator():
    from gen import scene_disparity
    s = scene_disparity(3)
    nt = np.diff(s.tri_off)
    assert list(nt) == [81920, 1280] * 3
    assert np.allclose(s.radius, [20.0, 1.0] * 3) and np.allclose(s.eps, 0.02)


def test_many_particles_momentum_identities(imp):
    """A small packing with several contacting pairs (one particle may touch
    several others): the momentum balance and the angular-momentum identity
    of the implicit Euler step hold for the whole system."""
    import dataclasses

    import oracle
    from gen import scene_chain
    s = scene_chain(4, seed=41)
    bound = imp.bounding_radius(s)
    pairs = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    eps = imp.pair_eps(s.radius, pairs[:, 0], pairs[:, 1])
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((s.n_particles, 3)))
    c0 = oracle.detect(base)
    assert len(np.unique(c0["pair"])) >= 3   # the chain's pairs are in contact
    rng = np.random.default_rng(2)
    vel = rng.normal(scale=0.1, size=(s.n_particles, 6))
    dt = 2e-4
    P, V, it, hist = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=2e-13, max_iter=2000)
    assert it < 2000
    m = s.mass
    inertia = 0.4 * m * s.radius ** 2
    p0 = (m[:, None] * vel[:, :3]).sum(0) + dt * m.sum() * imp.G_DEFAULT
    p1 = (m[:, None] * V[:, :3]).sum(0)
    assert np.abs(p1 - p0).max() <= 1e-11 * (np.abs(m[:, None] * vel[:, :3]).sum() + dt * m.sum() * 9.81)
    c = oracle.detect(base, poses=P)
    ft, _ = oracle.forces(base, c, poses=P)
    x0 = s.poses[:, :3]
    L0 = (np.cross(x0, m[:, None] * vel[:, :3]) + inertia[:, None] * vel[:, 3:]).sum(0)
    L1 = (np.cross(P[:, :3], m[:, None] * V[:, :3]) + inertia[:, None] * V[:, 3:]).sum(0)
    want = L0 + dt * np.cross(x0, m[:, None] * imp.G_DEFAULT).sum(0) - dt ** 2 * np.cross(V[:, :3], ft[:, :3]).sum(0)
    scale = np.abs(np.cross(x0, m[:, None] * vel[:, :3])).sum() + np.abs(inertia[:, None] * vel[:, 3:]).sum() \
        + dt * np.abs(np.cross(x0, m[:, None] * imp.G_DEFAULT)).sum()
    assert np.abs(L1 - want).max() <= 1e-10 * scale, (np.abs(L1 - want).max(), scale)


def _one_contact(c, k):
    return {key: v[k:k + 1] for key, v in c.items()}


def _icosahedra_facing(kind_a, kind_b, angle=0.7, gap=1.0, eps=0.05):
    """Two regular icosahedra along x, A's vertex / edge / face ('v', 'e',
    'f') facing B's, B turned by `angle` about x (so facing edges cross), the
    facing features gap * eps apart."""
    from gen import icosphere, scene_regular_pair
    from tests.test_oracle_contacts import _quat_from_matrix, _rotation_taking
    v, f = icosphere(0)

    def direction(kind):
        return {"v": v[0], "e": v[f[0][0]] + v[f[0][1]], "f": v[f[0]].sum(0)}[kind]

    ca, sa = np.cos(angle), np.sin(angle)
    Rx = np.array([[1.0, 0, 0], [0, ca, -sa], [0, sa, ca]])
    RA = _rotation_taking(direction(kind_a), np.array([1.0, 0, 0]))
    RB = Rx @ _rotation_taking(direction(kind_b), np.array([-1.0, 0, 0]))
    w = v.astype(np.float32).astype(np.float64)
    D = (w @ RA.T)[:, 0].max() - (w @ RB.T)[:, 0].min() + gap * eps
    return scene_regular_pair(0, 1.0, D, _quat_from_matrix(RA), _quat_from_matrix(RB), eps)


FACING = [("v", "f"), ("f", "v"), ("e", "e"), ("v", "e"), ("e", "v"), ("v", "v")]


@pytest.mark.parametrize("case", [4, 8] + FACING)
def test_contact_hessian_matches_finite_differences(imp, case):
    """The closed-form contact Hessian equals the central differences of the
    analytic pose gradient (closest points free to move), once the
    commutator of two rotations, -1/2 [dE/dtheta]x, is added to each
    rotation block; the antisymmetric part of the differences is exactly
    that term."""
    import dataclasses

    import oracle
    if isinstance(case, int):
        s, _, pairs, eps = _colliding_pair(imp, seed=case)
    else:
        s = _icosahedra_facing(*case)
        pairs, eps = s.pairs, s.eps
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((2, 3)))
    c = oracle.detect(base)
    assert len(c["d"]) >= 1 and (c["d"] > 0).all()
    Ha = imp.contact_hessian(base, c)
    Hf = imp.pose_hessian(s, s.poses, pairs, eps)
    _, gp, _ = oracle.grad(base, c)
    scale = np.abs(Hf).max()
    assert np.abs(Ha - Ha.T).max() <= 1e-12 * scale
    assert np.abs(imp.twist_hessian_fd_form(Ha, gp) - Hf).max() <= 1e-6 * scale
    anti = 0.5 * (Hf - Hf.T)
    for i in range(2):
        want = -0.5 * imp._skew(gp[i, 3:])
        assert np.abs(anti[6 * i + 3:6 * i + 6, 6 * i + 3:6 * i + 6] - want).max() <= 1e-6 * scale
        if isinstance(case, int):   # off-centre contacts: the term is far above the tolerance
            assert np.abs(gp[i, 3:]).max() >= 1e-4 * scale


def test_contact_hessian_translation_block_closed_form(imp):
    """Per contact, translating B moves the closest points along with it, so
    the distance's translation Hessian is (I - u u^T - Pi) / d, Pi the
    projector onto the directions of the active features (the span of the
    edges of a closest edge or face of either triangle): zero for a vertex
    against a face or two crossing edges, (I - u u^T - f f^T)/d for a vertex
    against an edge f, (I - u u^T)/d for two vertices.  The block is then
    e'' u u^T + e' (I - u u^T - Pi)/d, the same for A and B, and minus it
    between them."""
    import dataclasses

    import oracle
    kinds = set()
    scenes = [_icosahedra_facing(a, b) for a, b in FACING]
    for seed in (4, 8):
        s, _, pairs, eps = _colliding_pair(imp, seed=seed)
        scenes.append(dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((2, 3))))
    for base in scenes:
        s, eps = base, base.eps
        c = oracle.detect(base)
        assert len(c["d"]) > 0
        TA = oracle.world_triangles(base, 0)
        TB = oracle.world_triangles(base, 1)
        ks = 1000.0 * np.sqrt(1 / (1 / s.mass[0] + 1 / s.mass[1]))
        for k in range(len(c["d"])):
            d = float(c["d"][k])
            u = (c["pa"][k] - c["pb"][k]) / d
            dirs, kind = [], []
            for T, pt in ((TA[c["ta"][k]].reshape(3, 3), c["pa"][k]), (TB[c["tb"][k]].reshape(3, 3), c["pb"][k])):
                w = imp._barycentric(pt, T)
                S = [i for i in range(3) if w[i] > 1e-9]
                dirs += [T[j] - T[S[0]] for j in S[1:]]
                kind.append(len(S))
            kinds.add(tuple(kind))
            Pi = np.zeros((3, 3))
            if dirs:
                Q, sv, _ = np.linalg.svd(np.array(dirs).T)
                for col in range(int((sv > 1e-12 * sv.max()).sum())):
                    q = Q[:, col] - (Q[:, col] @ u) * u
                    Pi += np.outer(q, q) / (q @ q)
            e1 = -ks * (1 - d / (2 * eps[0]))
            e2 = ks / (2 * eps[0])
            want = e2 * np.outer(u, u) + e1 * (np.eye(3) - np.outer(u, u) - Pi) / d
            H = imp.contact_hessian(base, _one_contact(c, k))
            tol = 1e-9 * (abs(e2) + abs(e1) / d)
            assert np.abs(H[0:3, 0:3] - want).max() <= tol, (k, H[0:3, 0:3], want)
            assert np.abs(H[6:9, 6:9] - want).max() <= tol
            assert np.abs(H[0:3, 6:9] + want).max() <= tol
    assert kinds == {(1, 3), (3, 1), (2, 2), (1, 2), (2, 1), (1, 1)}   # every generic feature pair


def test_contact_hessian_vertex_against_vertex_closed_form(imp):
    """The tip-to-tip icosahedra of the finite-difference pin: the closed form
    gives 25 (e'' u u^T + e' (I - u u^T) / d) directly."""
    import oracle
    from gen import icosphere, scene_regular_pair
    from tests.test_oracle_contacts import _quat_from_matrix, _rotation_taking
    v, f = icosphere(0)
    qA = _quat_from_matrix(_rotation_taking(v[0], np.array([1.0, 0, 0])))
    qB = _quat_from_matrix(_rotation_taking(v[3], np.array([-1.0, 0, 0])))
    s = scene_regular_pair(0, 1.0, 2.06, qA, qB, 0.05)
    c = oracle.detect(s)
    H = imp.contact_hessian(s, c)
    d = float(c["d"][0])
    u = (c["pa"][0] - c["pb"][0]) / d
    ks = 1000.0 * np.sqrt(1 / (1 / s.mass[0] + 1 / s.mass[1]))
    e1 = -ks * (1 - d / (2 * s.eps[0]))
    e2 = ks / (2 * s.eps[0])
    want = 25 * (e2 * np.outer(u, u) + e1 * (np.eye(3) - np.outer(u, u)) / d)
    np.testing.assert_allclose(H[0:3, 0:3], want, rtol=0, atol=1e-9 * np.abs(want).max())
    np.testing.assert_allclose(H[0:3, 6:9], -want, rtol=0, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("case", [4, 8, "chain"])
@pytest.mark.parametrize("stiffness", ["analytic", "analytic-sym"])
def test_newton_with_the_analytic_hessian(imp, case, stiffness):
    """Newton's method with the closed-form Hessian as stiffness (as the
    differences see it, or its symmetric form, which a conjugate-gradient
    solve needs) and a backtracking line search converges in a handful of
    iterations to the Picard fixed point; Picard takes 18 to 149 here."""
    if case == "chain":
        from gen import scene_chain
        s = scene_chain(4, seed=41)
        pairs = imp.broad_phase(s.poses[:, :3], imp.bounding_radius(s), s.radius)
        eps = imp.pair_eps(s.radius, pairs[:, 0], pairs[:, 1])
        vel = np.random.default_rng(2).normal(scale=0.1, size=(s.n_particles, 6))
        dt = 2e-4
    else:
        s, vel, pairs, eps = _colliding_pair(imp, seed=case)
        dt = 5e-4
    _, V1, _, _ = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=2e-13, max_iter=1000)
    _, V2, it2 = imp.implicit_euler_step_newton(s, vel, pairs, eps, dt, tol=1e-12, max_iter=50,
                                                stiffness=stiffness)
    assert it2 <= 12, it2
    assert np.abs(V1 - V2).max() <= 1e-9 * np.abs(V1).max()


def test_scale_generator():
    """The scale workload's generator at a reduced size: the big particles
    first with their subdivision and radius, then the small ones; the same
    seed gives the same scene; some particles overlap a neighbour's bounding
    sphere (so the broad phase finds pairs), the rest keep apart."""
    from gen.icosphere import scene_scale
    s, frac = scene_scale(n_small=1500, n_big=3, fraction=0.2)
    nt = np.diff(s.tri_off)
    assert s.n_particles == 1503 and list(nt[:3]) == [81920] * 3 and (nt[3:] == 1280).all()
    assert np.allclose(s.radius[:3], 20.0) and np.allclose(s.radius[3:], 1.0)
    assert 0 < frac <= 0.2
    c = s.poses[:, :3]
    from scipy.spatial import cKDTree
    d, _ = cKDTree(c).query(c, k=2)
    near = d[:, 1] < 1.05 * 2.0 * 1.0
    assert near.sum() >= 100
    s2, frac2 = scene_scale(n_small=1500, n_big=3, fraction=0.2)
    assert frac2 == frac and np.array_equal(s2.poses, s.poses)


def test_kept_candidates_premise(orc, imp):
    """The premise of keeping candidates across iterations: when every point
    of A moves by at most m_A (centre shift plus rotation angle times the
    bounding radius) and of B by at most m_B, every triangle distance
    changes by at most m_A + m_B; so the pairs within 2 eps at the moved
    poses are among those within 2 (eps + w) at the reference poses when
    m_A + m_B <= 2 w.  Checked on the chain's triangle pairs under random
    rigid motions."""
    import dataclasses
    from gen import scene_chain
    s = scene_chain(4, seed=41)
    pairs = imp.broad_phase(s.poses[:, :3], imp.bounding_radius(s), s.radius)
    eps = imp.pair_eps(s.radius, pairs[:, 0], pairs[:, 1])
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((4, 3)))
    bound = imp.bounding_radius(s)
    rng = np.random.default_rng(31)
    w = 0.25 * eps.min()
    wide = orc.detect(dataclasses.replace(base, eps=eps + w))
    keys_wide = set(zip(wide["pair"].tolist(), wide["ta"].tolist(), wide["tb"].tolist()))
    for _ in range(5):
        vel = rng.normal(size=(4, 6))
        motion = np.abs(vel[:, :3]).sum(1) + np.linalg.norm(vel[:, 3:], axis=1) * bound
        dt = w / motion.max()       # every point moves by at most w
        moved = imp.moved_poses(s.poses, vel, dt)
        c = orc.detect(base, poses=moved)
        keys = set(zip(c["pair"].tolist(), c["ta"].tolist(), c["tb"].tolist()))
        assert keys <= keys_wide
        # distances of the kept pairs move by at most the two motions
        P0 = [orc.world_triangles(base, i) for i in range(4)]
        P1 = [orc.world_triangles(base, i, poses=moved) for i in range(4)]
        for p, ta, tb in list(keys_wide)[:200]:
            a, b = pairs[p]
            d0 = orc.tri_tri(P0[a][ta], P0[b][tb])[0][0]
            d1 = orc.tri_tri(P1[a][ta], P1[b][tb])[0][0]
            assert abs(d1 - d0) <= dt * (motion[a] + motion[b]) * (1 + 1e-9) + 1e-12
