"""Pins of the oracle's redundant-contact merge (Sec. 2, the implementation
note on the contact set: contact points of one pair closer than eps are merged
into one average point).  The merge is read as connected components of the
relation |x_i - x_j| < eps between contact points x = (pa + pb)/2 of one pair;
each component becomes one contact at the members' mean pa and pb."""
import numpy as np
import pytest

from gen import icosphere, scene_regular_pair
from tests.test_oracle_contacts import _quat_from_matrix, _rotation_taking


def _contacts(pair, ta, tb, pa, pb):
    pa = np.asarray(pa, np.float64).reshape(-1, 3)
    pb = np.asarray(pb, np.float64).reshape(-1, 3)
    return dict(pair=np.asarray(pair, np.int32), ta=np.asarray(ta, np.int32),
                tb=np.asarray(tb, np.int32), pa=pa, pb=pb,
                d=np.sqrt(((pa - pb) ** 2).sum(1)))


def _python_components(x, eps):
    """Independent check: breadth-first search over the links, plain Python
    floats (IEEE double, no fused operations), same predicate."""
    n = len(x)
    lab = [-1] * n
    lim = eps * eps
    c = 0
    for s in range(n):
        if lab[s] >= 0:
            continue
        lab[s] = c
        todo = [s]
        while todo:
            i = todo.pop()
            for j in range(n):
                if lab[j] < 0:
                    dx = x[i][0] - x[j][0]
                    dy = x[i][1] - x[j][1]
                    dz = x[i][2] - x[j][2]
                    if (dx * dx + dy * dy) + dz * dz < lim:
                        lab[j] = c
                        todo.append(j)
        c += 1
    return lab


def _partition(m, c):
    """Merged output -> {representative key: member count}; input keys."""
    return {(int(p), int(a), int(b)): int(k)
            for p, a, b, k in zip(m["pair"], m["ta"], m["tb"], m["members"])}


def test_duplicates_merge_to_their_common_point(orc):
    rng = np.random.default_rng(11)
    a, b = rng.normal(size=3), rng.normal(size=3)
    n = 7
    c = _contacts([3] * n, rng.permutation(n) + 10, [5] * n, [a] * n, [b] * n)
    m = orc.merge_contacts(c, np.full(4, 1e-3))
    assert len(m["d"]) == 1 and m["members"][0] == n
    assert (m["pair"][0], m["ta"][0], m["tb"][0]) == (3, 10, 5)
    # the mean of n equal values: within an ulp or two of that value
    np.testing.assert_allclose(m["pa"][0], a, rtol=5e-16, atol=0)
    np.testing.assert_allclose(m["pb"][0], b, rtol=5e-16, atol=0)
    assert m["d"][0] == pytest.approx(np.linalg.norm(a - b), rel=1e-15)


def test_closer_than_eps_is_strict():
    import oracle as orc
    eps = 0.25  # powers of two: every coordinate and difference below is exact
    for gap, merged in [(eps, False), (eps - 2.0 ** -30, True), (eps + 2.0 ** -30, False)]:
        pa = [[0.0, 0.0, 0.0], [gap, 0.0, 0.0]]
        pb = [[0.0, 0.0, 0.125], [gap, 0.0, 0.125]]
        m = orc.merge_contacts(_contacts([0, 0], [0, 1], [0, 0], pa, pb), [eps])
        assert len(m["d"]) == (1 if merged else 2), gap


def test_chain_is_one_component_with_mean_point(orc):
    # contact points 0.75 eps apart along a line: neighbours linked, the ends
    # are 6.75 eps apart; the transitive closure is one contact at the middle
    eps, n = 1.0, 10
    xs = 0.75 * np.arange(n)
    pa = np.stack([xs, np.zeros(n), np.zeros(n)], 1)
    pb = pa + [0.0, 0.0, 0.5]
    m = orc.merge_contacts(_contacts([0] * n, np.arange(n), np.zeros(n), pa, pb), [eps])
    assert len(m["d"]) == 1 and m["members"][0] == n
    np.testing.assert_allclose(m["pa"][0], [xs.mean(), 0.0, 0.0], rtol=0, atol=1e-15)
    assert m["d"][0] == pytest.approx(0.5, rel=1e-15)
    # spacing equal to eps: nothing links
    pa = np.stack([np.arange(n) * eps, np.zeros(n), np.zeros(n)], 1)
    m = orc.merge_contacts(_contacts([0] * n, np.arange(n), np.zeros(n), pa, pa + [0.0, 0.0, 0.5]),
                           [eps])
    assert len(m["d"]) == n and (m["members"] == 1).all()


def test_pairs_never_merge_with_each_other(orc):
    a, b = [1.0, 2.0, 3.0], [1.0, 2.0, 3.01]
    c = _contacts([0, 1, 1, 2], [0, 0, 1, 0], [0, 0, 0, 0], [a] * 4, [b] * 4)
    m = orc.merge_contacts(c, [1.0, 1.0, 1.0])
    assert list(m["pair"]) == [0, 1, 2] and list(m["members"]) == [1, 2, 1]


def test_mean_of_two(orc):
    pa = [[1.0, 0.0, 0.0], [1.5, 0.5, 0.0]]
    pb = [[1.0, 0.0, 1.0], [1.5, 0.5, 0.5]]
    m = orc.merge_contacts(_contacts([0, 0], [4, 2], [9, 9], pa, pb), [1.0])
    np.testing.assert_array_equal(m["pa"][0], [1.25, 0.25, 0.0])
    np.testing.assert_array_equal(m["pb"][0], [1.25, 0.25, 0.75])
    assert m["d"][0] == 0.75 and (m["ta"][0], m["tb"][0]) == (2, 9)


@pytest.mark.parametrize("seed", range(4))
def test_components_match_breadth_first_search(orc, seed):
    """Clustered random contact points in several pairs against the plain
    Python search; the result does not depend on the input order."""
    rng = np.random.default_rng(100 + seed)
    n_pairs = 5
    eps = rng.uniform(0.05, 0.2, n_pairs)
    rows = []
    for p in range(n_pairs):
        n = int(rng.integers(1, 60))
        centres = rng.uniform(-1, 1, (int(rng.integers(1, 8)), 3))
        x = centres[rng.integers(0, len(centres), n)] + rng.normal(scale=eps[p], size=(n, 3))
        keys = rng.choice(10_000, size=n, replace=False)
        for k in range(n):
            rows.append((p, int(keys[k]) // 100, int(keys[k]) % 100, x[k]))
    pair = np.array([r[0] for r in rows])
    ta = np.array([r[1] for r in rows])
    tb = np.array([r[2] for r in rows])
    x = np.array([r[3] for r in rows])
    # half-segments comparable to eps: linking pa or pb instead of the
    # midpoint would change the partition
    half = rng.normal(scale=0.1, size=x.shape)
    pa, pb = x - half, x + half
    c = _contacts(pair, ta, tb, pa, pb)
    m = orc.merge_contacts(c, eps)
    # expected partition by the plain search (on the same FP64 contact points)
    xs = (c["pa"] + c["pb"]) * 0.5
    want = {}
    for p in range(n_pairs):
        sel = np.flatnonzero(pair == p)
        lab = _python_components([tuple(v) for v in xs[sel]], float(eps[p]))
        for g in set(lab):
            mem = sel[[i for i, l in enumerate(lab) if l == g]]
            key = min((int(ta[i]), int(tb[i])) for i in mem)
            want[(p,) + key] = len(mem)
            k = np.flatnonzero((m["pair"] == p) & (m["ta"] == key[0]) & (m["tb"] == key[1]))
            assert len(k) == 1
            np.testing.assert_allclose(m["pa"][k[0]], c["pa"][mem].mean(0), rtol=0, atol=1e-14)
            np.testing.assert_allclose(m["pb"][k[0]], c["pb"][mem].mean(0), rtol=0, atol=1e-14)
    assert _partition(m, c) == want
    # order of C does not matter
    perm = rng.permutation(len(pair))
    m2 = orc.merge_contacts({k: v[perm] for k, v in c.items()}, eps)
    for k in ("pair", "ta", "tb", "members"):
        np.testing.assert_array_equal(m[k], m2[k])
    np.testing.assert_allclose(m2["pa"], m["pa"], rtol=0, atol=1e-14)
    # output sorted by (pair, ta, tb)
    keys = list(zip(m["pair"], m["ta"], m["tb"]))
    assert keys == sorted(keys)


def test_paper_example_vertex_against_vertex(orc):
    """Sec. 2's example of redundancy: when the closest distance of two
    objects is spanned by two vertices, every pair of triangles adjacent to
    them finds the same contact.  Two regular icosahedra (valence 5) tip to
    tip at gap g < 2 eps give 5 x 5 contacts at the two tips, which merge
    into one contact whose points are the tips and whose distance is g."""
    v, f = icosphere(0)
    ia, ib = 0, 3
    qA = _quat_from_matrix(_rotation_taking(v[ia], np.array([1.0, 0, 0])))
    qB = _quat_from_matrix(_rotation_taking(v[ib], np.array([-1.0, 0, 0])))
    eps, g = 0.05, 0.06
    s = scene_regular_pair(0, 1.0, 2.0 + g, qA, qB, eps)
    c = orc.detect(s)
    assert len(c["d"]) == 25
    assert set(c["ta"]) == set(np.flatnonzero((f == ia).any(1)))
    assert set(c["tb"]) == set(np.flatnonzero((f == ib).any(1)))
    tipA = orc.pose_matrix(s.poses[0]) @ s.verts[ia].astype(np.float64) + s.poses[0][:3]
    tipB = (orc.pose_matrix(s.poses[1]) @ s.verts[s.vert_off[1] + ib].astype(np.float64)
            + s.poses[1][:3])
    m = orc.merge_contacts(c, s.eps)
    assert len(m["d"]) == 1 and m["members"][0] == 25
    np.testing.assert_allclose(m["pa"][0], tipA, rtol=0, atol=1e-14)
    np.testing.assert_allclose(m["pb"][0], tipB, rtol=0, atol=1e-14)
    assert m["d"][0] == pytest.approx(np.linalg.norm(tipA - tipB), rel=1e-12)
    # the tips are float32 vertices of a unit icosahedron: g up to their rounding
    assert m["d"][0] == pytest.approx(g, abs=1e-6)
    assert (m["ta"][0], m["tb"][0]) == (min(c["ta"]), min(c["tb"]))


def test_empty(orc):
    m = orc.merge_contacts(_contacts([], [], [], np.zeros((0, 3)), np.zeros((0, 3))), [])
    assert all(len(v) == 0 for v in m.values())


def test_a_dropped_link_would_split(orc):
    """Guard against an off-by-one in the link predicate or a missing
    transitive step: removing the middle point of a three-point chain splits
    it, keeping it joins all three."""
    eps = 1.0
    x = np.array([[0.0, 0, 0], [0.9, 0, 0], [1.8, 0, 0]])
    for keep, want in [((0, 1, 2), 1), ((0, 2), 2)]:
        sel = list(keep)
        c = _contacts([0] * len(sel), sel, [0] * len(sel), x[sel], x[sel])
        assert len(orc.merge_contacts(c, [eps])["d"]) == want


def test_lone_contact_stays_as_detected(orc):
    """A contact with no other contact of its pair closer than eps is not
    averaged with anything: it comes out as it went in, its distance included
    (a crossing pair keeps d = 0 even where the two closest points differ in
    the last bits)."""
    pa = [[0.0, 0.0, 0.0], [5.0, 0.0, 0.0]]
    pb = [[0.0, 0.0, 1e-17], [5.0, 0.0, 0.25]]
    c = _contacts([0, 0], [1, 2], [3, 4], pa, pb)
    c["d"] = np.array([0.0, 0.25])
    m = orc.merge_contacts(c, [0.5])
    assert list(m["members"]) == [1, 1]
    np.testing.assert_array_equal(m["d"], [0.0, 0.25])
    np.testing.assert_array_equal(m["pa"], np.asarray(pa))
    np.testing.assert_array_equal(m["pb"], np.asarray(pb))
