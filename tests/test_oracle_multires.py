"""Pins of the multiresolution implicit-Euler oracle (Algorithm 6): the
active-set update on hand-built trees against hand-worked lists, the cut
property of the active sets, Lemma 1 on the unfolded sets (their fine
contacts equal the brute force), narrowing back to the roots, the force law
of surrogate contacts against the derivative of its energy, and the
paper's correctness lemma for Algorithm 6 (its fixed point is the plain
Picard fixed point)."""
import dataclasses

import numpy as np
import pytest

from gen import scene_chain


@pytest.fixture(scope="module")
def mr():
    import oracle
    oracle.build()
    from oracle import multires
    return multires


@pytest.fixture(scope="module")
def imp():
    from oracle import implicit
    return implicit


def _toy(mr):
    """Particle 0: root 0 over leaves 1, 2; particle 1: root 3 over leaves
    4, 5; particle 2: root 6, a leaf."""
    ex = dict(node_tri=np.zeros((7, 9), np.float32), node_delta=np.zeros(7, np.float32),
              node_child=np.array([[1, 2], [0, -1], [1, -1], [4, 2], [2, -1], [3, -1], [4, -1]]),
              node_level=np.array([1, 2, 2, 1, 2, 2, 1]), root=np.array([0, 3, 6]),
              slot_tri=np.array([0, 0, 0, 0, 0]))
    return mr.Trees(ex)


def test_update_rules_on_hand_built_trees(mr):
    T = _toy(mr)
    B, L, W = mr.BOT, mr.LEAF, mr.WIDEN
    N, V = mr.N_BIT, mr.V_BIT
    kids = [(0, 1, 4, 0), (0, 1, 5, 0), (0, 2, 4, 0), (0, 2, 5, 0)]
    # widening the root pair lists its four children, A's index major
    assert mr.frontier_update(T, [(0, 0, 3, 0)], [W]) == (kids, 1, 0)
    # a complete all-bottom group narrows to its parent, which carries N
    assert mr.frontier_update(T, kids, [B] * 4) == ([(0, 0, 3, N)], 0, 1)
    # widening an N item re-adds the children with the veto flag ...
    vk = [(p, a, b, V) for p, a, b, _ in kids]
    assert mr.frontier_update(T, [(0, 0, 3, N)], [W]) == (vk, 1, 0)
    # ... and they are not removed again
    assert mr.frontier_update(T, vk, [B] * 4) == (vk, 0, 0)
    # one member in contact keeps the group
    assert mr.frontier_update(T, kids, [B, L, B, B]) == (kids, 0, 0)
    # a leaf side stays while the other unfolds; its group narrows alike
    assert mr.frontier_update(T, [(1, 6, 3, 0)], [W]) == ([(1, 6, 4, 0), (1, 6, 5, 0)], 1, 0)
    assert T.parent_pair(6, 5) == (6, 3) and T.child_index(6, 5, (6, 3)) == (1, 2)
    # groups of several pairs side by side; an incomplete group stays
    both = kids + [(1, 6, 4, 0), (1, 6, 5, 0)]
    assert mr.frontier_update(T, both, [B] * 6) == ([(0, 0, 3, N), (1, 6, 3, N)], 0, 2)
    part = kids[:2] + [(1, 6, 4, 0), (1, 6, 5, 0)]
    assert mr.frontier_update(T, part, [B] * 4) == (kids[:2] + [(1, 6, 3, N)], 0, 1)
    # the root pair has no parent
    assert mr.frontier_update(T, [(0, 0, 3, 0)], [B]) == ([(0, 0, 3, 0)], 0, 0)


def _leaves(T, v):
    if T.leaf(v):
        return [int(v)]
    b, c = T.child[v]
    return [x for ch in range(b, b + c) for x in _leaves(T, ch)]


def _check_cut(T, frontier, pairs):
    """Every pair of leaves of every particle pair below exactly one item."""
    for p, (A, B) in enumerate(pairs):
        want = sorted((x, y) for x in _leaves(T, T.root[A]) for y in _leaves(T, T.root[B]))
        got = sorted((x, y) for q, a, b, _ in frontier if q == p
                     for x in _leaves(T, a) for y in _leaves(T, b))
        assert got == want, p


def _chain(imp):
    import paper_2105_12415_gb300 as m
    s = scene_chain(4, seed=41)
    v, t = s.particle(0)
    bound = imp.bounding_radius(s)
    pairs = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    eps = imp.pair_eps(s.radius, pairs[:, 0], pairs[:, 1])
    h = m.Hierarchy.build_host(s.vert_off, s.verts, s.tri_off, s.tris)
    return s, pairs, eps, h.export()


def _unfold(mr, s, T, poses, pairs, eps, frontier, check=None):
    """Test and update at fixed poses until nothing widens or narrows."""
    for _ in range(20):
        st, fine, sur = mr.frontier_test(s, T, poses, pairs, eps, frontier)
        frontier, w, n = mr.frontier_update(T, frontier, st)
        if check:
            check(frontier)
        if w == 0 and n == 0:
            return frontier, st, fine, sur
    raise AssertionError("active sets did not settle")


def test_unfolded_sets_are_cuts_and_find_every_contact(mr, imp, orc):
    s, pairs, eps, ex = _chain(imp)
    T = mr.Trees(ex)
    assert T.level[T.root].min() >= 0 and (T.child[:, 1] > 0).sum() > len(pairs)
    F0 = mr.initial_frontier(T, pairs)
    _check_cut(T, F0, pairs)
    F, st, fine, sur = _unfold(mr, s, T, s.poses, pairs, eps, F0,
                               check=lambda f: _check_cut(T, f, pairs))
    assert len(sur["d"]) == 0 and mr.WIDEN not in st
    base = dataclasses.replace(s, pairs=pairs, eps=eps)
    want = orc.detect(base)
    assert len(want["d"]) > 0
    for k in ("pair", "ta", "tb"):
        np.testing.assert_array_equal(fine[k], want[k])
    np.testing.assert_array_equal(fine["d"], want["d"])
    # the unfolded sets are far smaller than the leaf products
    full = sum(len(_leaves(T, T.root[A])) * len(_leaves(T, T.root[B])) for A, B in pairs)
    assert len(F) < full


def _last_member_rule(T, frontier, seen):
    """In a cut listed in depth-first order, a first child's sibling group is
    listed in full (the parent's children side by side, in child order) if
    and only if the item size - 1 places after it is the same parent's last
    child: the items between are then the other children themselves.  The
    GPU's narrowing checks completeness this way; `seen` counts the groups
    found complete and incomplete."""
    n = len(frontier)

    def is_child(i, p, par, k):
        q, a, b, _ = frontier[i]
        return (q == p and T.parent_pair(a, b) == par
                and T.child_index(a, b, par)[0] == k)

    for i, (p, a, b, _) in enumerate(frontier):
        par = T.parent_pair(a, b)
        if par is None:
            continue
        c, size = T.child_index(a, b, par)
        if c != 0:
            continue
        full = i + size <= n and all(is_child(i + k, p, par, k) for k in range(size))
        last = i + size <= n and is_child(i + size - 1, p, par, size - 1)
        assert full == last, (i, p, par, size)
        seen[full] += 1


def test_group_completeness_from_its_last_member(mr, imp):
    """The completeness shortcut holds on every active set the unfolding and
    the narrowing back to the roots produce, with both outcomes occurring."""
    s, pairs, eps, ex = _chain(imp)
    T = mr.Trees(ex)
    seen = {True: 0, False: 0}
    F, _, _, _ = _unfold(mr, s, T, s.poses, pairs, eps, mr.initial_frontier(T, pairs),
                         check=lambda f: _last_member_rule(T, f, seen))
    far = s.poses.copy()
    far[:, :3] *= 20.0
    G = [(p, a, b, 0) for p, a, b, _ in F]
    for _ in range(10):
        st, _, _ = mr.frontier_test(s, T, far, pairs, eps, G)
        G, _, n = mr.frontier_update(T, G, st)
        _last_member_rule(T, G, seen)
        if n == 0:
            break
    assert seen[True] > 0 and seen[False] > 0, seen


def test_separated_pairs_narrow_to_their_roots(mr, imp):
    """Unfold at the contact poses, then move the particles far apart: with
    the flags cleared every group narrows, one level per iteration, back to
    the root pairs; with the flags of the unfolding kept, the groups that
    were narrowed and re-added (V) stay."""
    s, pairs, eps, ex = _chain(imp)
    T = mr.Trees(ex)
    F, _, _, _ = _unfold(mr, s, T, s.poses, pairs, eps, mr.initial_frontier(T, pairs))
    assert len(F) > len(pairs)
    far = s.poses.copy()
    far[:, :3] *= 20.0

    def settle(G):
        narrowed = []
        for _ in range(10):
            st, fine, sur = mr.frontier_test(s, T, far, pairs, eps, G)
            assert len(fine["d"]) == 0 and len(sur["d"]) == 0 and set(st) == {mr.BOT}
            G, w, n = mr.frontier_update(T, G, st)
            assert w == 0
            _check_cut(T, G, pairs)
            narrowed.append(n)
            if n == 0:
                return G, narrowed
        raise AssertionError("did not settle")

    G, narrowed = settle([(p, a, b, 0) for p, a, b, _ in F])
    assert [(p, a, b) for p, a, b, _ in G] == [(p, int(T.root[A]), int(T.root[B]))
                                               for p, (A, B) in enumerate(pairs)]
    assert all(f == mr.N_BIT for *_, f in G)
    assert len(narrowed) - 1 <= int(T.level.max() - T.level.min())
    vetoed = [x for x in F if x[3] & mr.V_BIT]
    assert vetoed, "the unfolding narrowed and re-added no group"
    H, _ = settle(F)
    assert all(x in H for x in vetoed)


def test_surrogate_force_is_minus_the_energy_derivative(mr, imp):
    s, pairs, eps, _ = _chain(imp)
    p = 0
    A, B = pairs[p]
    u = np.array([0.36, -0.48, 0.8])
    pb = np.array([0.1, 0.2, 0.3])
    tau, d = 0.05, 0.02

    def sur(dd):
        return dict(pair=np.array([p]), d=np.array([dd]), pa=np.array([pb + dd * u]),
                    pb=np.array([pb]), tau=np.array([tau]), n=np.array([[0.0, 0.0, 1.0]]))
    ft, _ = mr.surrogate_forces(s, pairs, eps, s.poses, sur(d), weight=0.3)
    h = 1e-6
    _, ep = mr.surrogate_forces(s, pairs, eps, s.poses, sur(d + h), weight=0.3)
    _, em = mr.surrogate_forces(s, pairs, eps, s.poses, sur(d - h), weight=0.3)
    dE = (ep - em) / (2 * h)
    np.testing.assert_allclose(ft[A, :3], -dE * u, rtol=1e-8)
    np.testing.assert_allclose(ft[B, :3], dE * u, rtol=1e-8)
    # torques: about each body origin, at the midpoint of the two points
    xc = pb + 0.5 * d * u
    np.testing.assert_allclose(ft[A, 3:], np.cross(xc - s.poses[A, :3], ft[A, :3]), rtol=1e-12)
    # crossing surrogates push along minus A's surrogate normal
    ft0, _ = mr.surrogate_forces(s, pairs, eps, s.poses, sur(0.0), weight=0.3)
    assert ft0[A, 2] < 0 and np.allclose(ft0[A, :2], 0.0)


def test_multires_step_reaches_the_plain_fixed_point(mr, imp):
    s, pairs, eps, ex = _chain(imp)
    T = mr.Trees(ex)
    rng = np.random.default_rng(2)
    vel = rng.normal(scale=0.1, size=(s.n_particles, 6))
    dt = 2e-4
    P, V, it, hist = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=2e-13, max_iter=2000)
    Pm, Vm, itm, histm, rec = mr.multires_implicit_euler_step(s, T, vel, pairs, eps, dt,
                                                              tol=2e-13, max_iter=2000)
    assert itm < 2000
    # the trees unfold over several iterations, with surrogate contacts on the way
    assert sum(r["widened"] > 0 for r in rec) >= int(T.level.max() - T.level.min())
    assert any(r["surrogate"] > 0 for r in rec)
    assert rec[-1]["widened"] == 0 and rec[-1]["narrowed"] == 0 and rec[-1]["surrogate"] == 0
    # the same fixed point: both stop within 2e-13 relative of it and the
    # map contracts, so they agree to a small multiple of that
    scale = np.abs(V).max()
    assert np.abs(Vm - V).max() <= 1e-10 * scale
    assert np.abs(Pm - P).max() <= dt * 1e-10 * scale + 1e-14 * (1 + np.abs(P).max())
