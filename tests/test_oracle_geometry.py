"""Pins of the oracle's exact triangle-triangle distance (Sec. 3, comparison-based
method) against closed forms, an independent KKT enumeration and brute-force
sampling."""
import numpy as np
import pytest

from tests.kkt_reference import grid_distance, kkt_distance


def _rand_tris(rng, n, spread=1.0, size=1.0):
    c = rng.uniform(-spread, spread, size=(n, 1, 3))
    return (c + rng.normal(scale=size, size=(n, 3, 3))).reshape(n, 9)


def _rot(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


# ---------------------------------------------------------------------------
# point-triangle and segment-segment closed forms
def test_point_triangle_regions(orc):
    T = np.array([0, 0, 0, 2, 0, 0, 0, 2, 0], float)
    cases = [
        ((0.5, 0.5, 3.0), 3.0, (0.5, 0.5, 0)),             # above the interior
        ((-1.0, -1.0, 0.0), np.sqrt(2), (0, 0, 0)),        # vertex region of v0
        ((1.0, -2.0, 1.0), np.sqrt(5), (1, 0, 0)),         # edge v0v1 region
        ((2.0, 2.0, 0.0), np.sqrt(2), (1, 1, 0)),          # edge v1v2 region (hypotenuse)
        ((3.0, -1.0, 0.0), np.sqrt(2), (2, 0, 0)),         # vertex v1
    ]
    for p, d_exp, q_exp in cases:
        d, q = orc.point_triangle(np.array(p, float), T)
        assert abs(d[0] - d_exp) < 1e-14
        assert np.allclose(q[0], q_exp, atol=1e-14)


def test_segment_segment_closed_forms(orc):
    # skew segments with the common perpendicular along z
    S1 = np.array([-1, 0, 0, 1, 0, 0], float)
    S2 = np.array([0, -1, 0.7, 0, 1, 0.7], float)
    d, c1, c2 = orc.segment_segment(S1, S2)
    assert abs(d[0] - 0.7) < 1e-15
    assert np.allclose(c1[0], [0, 0, 0]) and np.allclose(c2[0], [0, 0, 0.7])
    # the perpendicular foot outside one segment: clamp to its endpoint
    S2 = np.array([2, -1, 0.7, 2, 1, 0.7], float)
    d, _, _ = orc.segment_segment(S1, S2)
    assert abs(d[0] - np.hypot(1.0, 0.7)) < 1e-14
    # parallel overlapping segments
    S2 = np.array([0.5, 0.3, 0, 3, 0.3, 0], float)
    d, _, _ = orc.segment_segment(S1, S2)
    assert abs(d[0] - 0.3) < 1e-15


# ---------------------------------------------------------------------------
# triangle-triangle closed forms
@pytest.mark.parametrize("seed", range(5))
def test_parallel_offset_copy(orc, seed):
    """A triangle against its copy translated by h along its unit normal, plus
    an in-plane shift that keeps the projections overlapping: d = h."""
    rng = np.random.default_rng(seed)
    for _ in range(50):
        P = rng.normal(size=(3, 3))
        n = np.cross(P[1] - P[0], P[2] - P[0])
        n /= np.linalg.norm(n)
        h = rng.uniform(1e-4, 2.0)
        w = rng.dirichlet([1, 1, 1])
        shift = 0.3 * (w @ P - P.mean(0))          # small in-plane shift
        shift -= (shift @ n) * n
        Q = P + h * n + shift
        d, pa, pb, _ = orc.tri_tri(P.ravel(), Q.ravel())
        assert abs(d[0] - h) <= 1e-12 * max(1.0, h)
        assert abs(np.linalg.norm(pa[0] - pb[0]) - d[0]) < 1e-12


def test_crossing_triangles_distance_zero(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        R = _rot(rng)
        P = np.array([[-1, -1, 0], [2, -1, 0], [-1, 2, 0]], float)
        Q = np.array([[0, 0, -1], [0.2, 0.1, 1], [0.5, -0.3, 1]], float)   # pierces P
        off = rng.normal(size=3)
        d, pa, pb, f = orc.tri_tri((P @ R.T + off).ravel(), (Q @ R.T + off).ravel())
        assert d[0] == 0.0 and f[0] >= 100
        assert np.allclose(pa[0], pb[0])


def test_kkt_enumeration_random(orc):
    """Random pairs (separated, touching, crossing, near-parallel): the oracle
    equals the independent KKT enumeration."""
    rng = np.random.default_rng(11)
    n = 20000
    P = _rand_tris(rng, n, spread=1.5)
    Q = _rand_tris(rng, n, spread=1.5)
    # near-parallel family: Q = P rotated by a tiny angle and offset
    m = 4000
    for k in range(m):
        Pk = P[k].reshape(3, 3)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        ang = rng.uniform(0, 1e-3)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        Rk = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
        nrm = np.cross(Pk[1] - Pk[0], Pk[2] - Pk[0])
        nrm /= np.linalg.norm(nrm)
        Q[k] = ((Pk - Pk.mean(0)) @ Rk.T + Pk.mean(0) + rng.uniform(-0.1, 0.3) * nrm
                + rng.normal(scale=0.3, size=3)).ravel()
    d, pa, pb, _ = orc.tri_tri(P, Q)
    dk = kkt_distance(P, Q)
    err = np.abs(d - dk)
    assert np.all(err <= 1e-9 * np.maximum(1.0, dk)), err.max()
    # the returned points realise the distance and lie on their triangles
    assert np.allclose(np.linalg.norm(pa - pb, axis=1), d, atol=1e-12)
    dpa, _ = orc.point_triangle(pa, P)
    dpb, _ = orc.point_triangle(pb, Q)
    assert dpa.max() < 1e-12 and dpb.max() < 1e-12


def test_grid_sampling_upper_bound(orc):
    rng = np.random.default_rng(3)
    P = _rand_tris(rng, 30)
    Q = _rand_tris(rng, 30)
    d, _, _, _ = orc.tri_tri(P, Q)
    for k in range(30):
        g = grid_distance(P[k], Q[k], m=30)
        # sampling never beats the exact minimum and approaches it
        assert g >= d[k] - 1e-12
        size = max(np.ptp(P[k].reshape(3, 3), 0).max(), np.ptp(Q[k].reshape(3, 3), 0).max())
        assert g - d[k] <= size / 30 * 2.5


def test_symmetry_and_rigid_motion(orc):
    rng = np.random.default_rng(5)
    P = _rand_tris(rng, 3000, spread=1.0)
    Q = _rand_tris(rng, 3000, spread=1.0)
    d, _, _, _ = orc.tri_tri(P, Q)
    d2, _, _, _ = orc.tri_tri(Q, P)
    assert np.allclose(d, d2, rtol=0, atol=1e-12)
    R = _rot(rng)
    t = rng.normal(size=3) * 10
    Pm = (P.reshape(-1, 3, 3) @ R.T + t).reshape(-1, 9)
    Qm = (Q.reshape(-1, 3, 3) @ R.T + t).reshape(-1, 9)
    d3, _, _, _ = orc.tri_tri(Pm, Qm)
    assert np.allclose(d, d3, rtol=0, atol=1e-11)
    # scale covariance
    d4, _, _, _ = orc.tri_tri(2.5 * P, 2.5 * Q)
    assert np.allclose(d4, 2.5 * d, rtol=1e-13, atol=1e-13)


def _near_parallel(rng, P):
    """Q = P turned by a tiny angle about its centroid, moved along P's normal
    by U[-0.1, 0.3] and sideways (vectorised form of the family above)."""
    n = len(P)
    T = P.reshape(n, 3, 3)
    ax = rng.normal(size=(n, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    ang = rng.uniform(0, 1e-3, n)
    K = np.zeros((n, 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -ax[:, 2], ax[:, 1], -ax[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = ax[:, 2], -ax[:, 1], ax[:, 0]
    R = np.eye(3) + np.sin(ang)[:, None, None] * K + (1 - np.cos(ang))[:, None, None] * (K @ K)
    c = T.mean(1, keepdims=True)
    nrm = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    off = rng.uniform(-0.1, 0.3, (n, 1)) * nrm + rng.normal(scale=0.3, size=(n, 3))
    return (np.einsum("nij,nkj->nki", R, T - c) + c + off[:, None, :]).reshape(n, 9)


def test_kkt_enumeration_million(orc):
    """One million seeded random triangle pairs (15 chunks of separated,
    touching and crossing pairs, 5 of near-parallel ones) against the
    independent KKT enumeration, in chunks of 50 000."""
    rng = np.random.default_rng(2105)
    worst = 0.0
    for chunk in range(20):
        n = 50_000
        P = _rand_tris(rng, n, spread=1.5)
        Q = _near_parallel(rng, P) if chunk >= 15 else _rand_tris(rng, n, spread=1.5)
        d = orc.tri_tri(P, Q)[0]
        dk = kkt_distance(P, Q)
        err = np.abs(d - dk) / np.maximum(1.0, dk)
        worst = max(worst, float(err.max()))
        assert err.max() <= 1e-9, (chunk, err.max())
    assert worst < 1e-9
