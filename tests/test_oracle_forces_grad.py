"""Pins of the oracle's penalty forces (Sec. 2, F(c)), contact energy and its
analytic gradient / Gauss-Newton blocks: single-contact closed form,
equal-and-opposite forces, torque balance, F = -dE/dt and central finite
differences."""
import numpy as np
import pytest

from gen import Scene, quat_to_matrix_f64, scene_pairs


def _two_triangle_scene(P, Q, eps, mass=(2.0, 3.0)):
    """Two one-triangle 'particles' at identity poses."""
    verts = np.concatenate([P.reshape(3, 3), Q.reshape(3, 3)]).astype(np.float32)
    return Scene(verts, np.array([0, 3, 6]), np.array([[0, 1, 2], [0, 1, 2]], np.int32),
                 np.array([0, 1, 2]), np.array([[0, 0, 0, 1, 0, 0, 0.0]] * 2),
                 np.array(mass, float), np.array([[0.1, 0.2, 0.3], [0.0, -0.5, 0.2]]),
                 np.ones(2), np.array([[0, 1]], np.int32), np.array([eps]), "two-triangles")


def test_single_contact_closed_form(orc):
    P = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], float)
    eps = 0.05
    for h in (1 / 128, 1 / 64, 3 / 64, 5 / 64):        # exact in float32
        Q = P.reshape(3, 3) + [0.125, 0.125, -h]        # below P, parallel
        Q = Q[[0, 2, 1]]                                 # opposite orientation
        s = _two_triangle_scene(P, Q, eps)
        c = orc.detect(s)
        assert len(c["d"]) == 1 and abs(c["d"][0] - h) < 1e-15
        ft, E = orc.forces(s, c)
        mu = 1 / (1 / 2.0 + 1 / 3.0)
        mag = 1000 * np.sqrt(mu) * (1 - h / (2 * eps))
        assert np.allclose(ft[0, :3], [0, 0, mag], rtol=1e-14)       # pushes A up (+z)
        assert np.allclose(ft[1, :3], [0, 0, -mag], rtol=1e-14)
        assert abs(E - 1000 * np.sqrt(mu) * eps * (1 - h / (2 * eps)) ** 2) < 1e-12
    # no contact beyond 2 eps
    Q = P.reshape(3, 3) + [0.1, 0.1, -2 * eps - 1e-6]
    assert len(orc.detect(_two_triangle_scene(P, Q, eps))["d"]) == 0


def _c3_like(n_pairs=3, level=2, seed=5):
    eps = np.full(n_pairs, 0.02)
    return scene_pairs(np.full(n_pairs, level), np.full(n_pairs, level), np.full(n_pairs, 0.7),
                       np.full(n_pairs, 1.0), eps, 1.7 * eps, seed, "grad-test", spread=3.0)


def test_forces_balance_and_torque(orc):
    s = scene_pairs([2, 1, 2], [1, 2, 2], [1.0, 0.5, 0.8], [0.6, 1.0, 0.8], [0.02, 0.01, 0.015],
                    [-0.08, 0.0, 0.005], 17, "balance", spread=5.0)
    c = orc.detect(s)
    assert len(c["d"]) > 0 and (c["d"] == 0).any()
    ft, _ = orc.forces(s, c)
    for p in range(s.n_pairs):
        A, B = s.pairs[p]
        assert np.allclose(ft[A, :3] + ft[B, :3], 0, atol=1e-9)
        # torques about the common world origin cancel
        cA = quat_to_matrix_f64(s.poses[A, 3:]) @ s.com[A] + s.poses[A, :3]
        cB = quat_to_matrix_f64(s.poses[B, 3:]) @ s.com[B] + s.poses[B, :3]
        tot = ft[A, 3:] + np.cross(cA, ft[A, :3]) + ft[B, 3:] + np.cross(cB, ft[B, :3])
        scale = np.abs(ft[A, :3]).sum() * (1 + np.abs(s.poses[A, :3]).max())
        assert np.abs(tot).max() <= 1e-11 * scale


def test_force_is_minus_translation_gradient(orc):
    s = _c3_like()
    c = orc.detect(s)
    ft, _ = orc.forces(s, c)
    _, gp, _ = orc.grad(s, c)
    assert np.allclose(ft[:, :3], -gp[:, :3], rtol=1e-12, atol=1e-9)


def _apply_twist(pose, k, h):
    """Pose with a world translation (k < 3) or a left rotation about the
    particle origin (k >= 3) of size h along axis k mod 3."""
    p = pose.copy()
    if k < 3:
        p[k] += h
        return p
    ax = np.zeros(3)
    ax[k - 3] = 1.0
    dq = np.r_[np.cos(h / 2), np.sin(h / 2) * ax]
    w1, v1, w2, v2 = dq[0], dq[1:], p[3], p[4:]
    p[3] = w1 * w2 - v1 @ v2
    p[4:] = w1 * v2 + w2 * v1 + np.cross(v1, v2)
    return p


def test_pose_gradient_finite_differences(orc):
    s = _c3_like()
    c = orc.detect(s)
    assert len(c["d"]) > 0 and c["d"].min() >= 1.7 * 0.02 - 1e-9
    _, gp, _ = orc.grad(s, c)
    h = 1e-6
    for i in range(s.n_particles):
        for k in range(6):
            pp, pm = s.poses.copy(), s.poses.copy()
            pp[i] = _apply_twist(s.poses[i], k, h)
            pm[i] = _apply_twist(s.poses[i], k, -h)
            fd = (orc.energy(s, poses=pp) - orc.energy(s, poses=pm)) / (2 * h)
            assert abs(fd - gp[i, k]) <= 1e-5 * max(1.0, np.abs(gp).max()), (i, k, fd, gp[i, k])


def test_vertex_gradient_finite_differences(orc):
    s = _c3_like(n_pairs=2)
    c = orc.detect(s)
    gv, _, _ = orc.grad(s, c)
    V = s.verts.astype(np.float64)
    rng = np.random.default_rng(0)
    active = np.unique(np.abs(gv).sum(1).nonzero()[0])
    idx = np.concatenate([rng.choice(active, size=min(12, len(active)), replace=False),
                          rng.choice(len(V), size=4, replace=False)])
    h = 1e-6
    scale = max(1.0, np.abs(gv).max())
    for vi in idx:
        for k in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[vi, k] += h
            Vm[vi, k] -= h
            fd = (orc.energy(s, verts=Vp) - orc.energy(s, verts=Vm)) / (2 * h)
            assert abs(fd - gv[vi, k]) <= 1e-5 * scale, (vi, k, fd, gv[vi, k])


def test_gauss_newton_block_translation_part(orc):
    """Vertex-face contact: d is affine in the translations, so the exact
    Hessian of E over (t_A, t_B) equals the Gauss-Newton block; compare with
    central differences of the analytic translation gradient."""
    P = np.array([0.3, 0.3, 0.0, 1.0, 0.2, 0.8, 0.1, 1.0, 0.9], float)   # P0 is the closest
    Q = np.array([0, 0, -0.03, 1, 0, -0.03, 0, 1, -0.03], float)[[0, 1, 2, 6, 7, 8, 3, 4, 5]]
    s = _two_triangle_scene(P, Q, eps=0.05)
    c = orc.detect(s)
    assert len(c["d"]) == 1
    _, _, jac = orc.grad(s, c)
    J = jac[0]
    assert np.allclose(J, J.T)
    assert np.linalg.eigvalsh(J).min() > -1e-9
    h = 1e-7
    H = np.zeros((6, 6))
    cols = [(0, k) for k in range(3)] + [(1, k) for k in range(3)]
    for a, (i, k) in enumerate(cols):
        pp, pm = s.poses.copy(), s.poses.copy()
        pp[i, k] += h
        pm[i, k] -= h
        _, gpp, _ = orc.grad(s, orc.detect(s, poses=pp), poses=pp)
        _, gpm, _ = orc.grad(s, orc.detect(s, poses=pm), poses=pm)
        g = (gpp - gpm) / (2 * h)
        H[:, a] = np.r_[g[0, :3], g[1, :3]]
    sub = J[np.ix_([0, 1, 2, 6, 7, 8], [0, 1, 2, 6, 7, 8])]
    assert np.allclose(H, sub, rtol=1e-6, atol=1e-6 * np.abs(sub).max())


@pytest.mark.parametrize("k_s", [1000.0, 10.0])
def test_energy_scales_with_spring_constant(orc, k_s):
    s = _c3_like(n_pairs=1)
    assert abs(orc.energy(s, k_s=k_s) - orc.energy(s) * k_s / 1000.0) < 1e-9
