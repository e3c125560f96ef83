"""Pins of the oracle's FP64 penalty sweep (Sec. 3, Eq. 3 functional, Eq. 4
alternating modified Newton; Algorithm 4 fixed iteration count)."""
import numpy as np


def test_one_iteration_by_hand(orc):
    """P: unit right triangle at z = 1; Q: the same shifted by (0.5, 0.5, -1).
    From x = 0: r = P0 - Q0 = (-0.5, -0.5, 1), grad J^ = (r.e1, r.e2, -r.f1,
    -r.f2) = (-0.5, -0.5, 0.5, 0.5), diag H^ = 1, s = 1, alpha_reg = 1, so the
    first half-step gives (0.25, 0.25, -0.25, -0.25).  P's unknowns are
    feasible; Q's violate a >= 0 and b >= 0 once each, so each moves by
    alpha_it * 0.25 / (alpha_it + alpha_reg) towards 0: -0.25/(1 + 100)."""
    P = np.array([0, 0, 1, 1, 0, 1, 0, 1, 1], float)
    Q = np.array([0.5, 0.5, 0, 1.5, 0.5, 0, 0.5, 1.5, 0], float)
    r = orc.sweep(P, Q, eps=0.1, n_iter=1, rho_reg=1.0, rho_iter=100.0)
    exp = np.array([0.25, 0.25, -0.25 / 101.0, -0.25 / 101.0])
    assert np.allclose(r["x"][0], exp, rtol=0, atol=1e-15)
    # the a+b<=1 constraint: push P's unknowns beyond the hypotenuse
    P2 = np.array([0, 0, 1, 1, 0, 1, 0, 1, 1], float)
    Q2 = np.array([2.0, 2.0, 0, 3.0, 2.0, 0, 2.0, 3.0, 0], float)
    r2 = orc.sweep(P2, Q2, eps=0.1, n_iter=1, rho_reg=1.0, rho_iter=100.0)
    # half-step: r = (-2,-2,1): grad (-2,-2,2,2) -> x = (1, 1, -1, -1)
    # P: a+b-1 = 1 active, a,b <= 1 not violated (a = 1 is not > 1):
    #    a <- 1 - 100*1/(100+1)
    # Q: a,b < 0 active: a <- -1 + 100/101
    a = 1 - 100.0 / 101.0
    b = -1 + 100.0 / 101.0
    assert np.allclose(r2["x"][0], [a, a, b, b], rtol=0, atol=1e-15)


def _near_pairs(rng, n):
    P = rng.normal(size=(n, 3, 3))
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    Q = P + rng.uniform(-0.1, 0.2, size=(n, 1)) [:, :, None] * nrm[:, None, :] \
        + rng.normal(scale=0.3, size=(n, 1, 3)) + rng.normal(scale=0.05, size=(n, 3, 3))
    return P.reshape(n, 9), Q.reshape(n, 9)


def test_certificate_is_a_lower_bound(orc):
    """gap = min u.P - max u.Q along any unit u bounds the distance from below."""
    rng = np.random.default_rng(21)
    P1 = rng.normal(size=(20000, 9))
    Q1 = rng.normal(size=(20000, 9)) + np.tile(rng.normal(size=(20000, 3)), 3)
    P2, Q2 = _near_pairs(rng, 20000)
    P, Q = np.concatenate([P1, P2]), np.concatenate([Q1, Q2])
    d, _, _, _ = orc.tri_tri(P, Q)
    for n_iter in (1, 4, 16):
        r = orc.sweep(P, Q, eps=0.01, n_iter=n_iter)
        assert np.all(r["gap"] <= d + 1e-12)
        # the certificate prunes well-separated pairs
        far = d > 1.0
        assert np.mean(r["gap"][far] > 0.5 * d[far]) > 0.8


def test_vertex_face_converges_to_exact_distance(orc):
    """Closest feature = vertex P0 (the start point a1 = b1 = 0) over Q's
    interior: the Q unknowns follow a damped Jacobi iteration on the 2x2
    normal equations of the projection, P's stay at 0 by the penalty, so the
    iterate distance tends to the point-plane distance."""
    rng = np.random.default_rng(2)
    Ps, Qs = [], []
    for _ in range(400):
        Q = np.c_[rng.normal(size=(3, 2)), np.zeros(3)]
        foot = rng.dirichlet([3, 3, 3]) @ Q
        P0 = foot + [0, 0, rng.uniform(0.05, 1.0)]
        P1 = P0 + np.r_[rng.normal(size=2), rng.uniform(0.2, 1.0)]
        P2 = P0 + np.r_[rng.normal(size=2), rng.uniform(0.2, 1.0)]
        Ps.append(np.r_[P0, P1, P2])
        Qs.append(Q.ravel())
    P, Q = np.array(Ps), np.array(Qs)
    d, _, _, f = orc.tri_tri(P, Q)
    assert np.all(f == 0)
    r = orc.sweep(P, Q, eps=0.01, n_iter=5000, rho_reg=1.0, rho_iter=1e6)
    rel = np.abs(r["dist_iter"] - d) / d
    assert np.median(rel) < 1e-5 and np.percentile(rel, 95) < 1e-3
    assert r["converged"].all()
