"""The multiresolution implicit step on the GPU (Algorithm 6) against the
FP64 oracle: the active sets stay cuts of the product trees through every
widening and narrowing, their fine contacts at rest equal the brute force
(Lemma 1), separated pairs narrow back to their roots (and re-added groups
stay, the memory set U), the surrogate contact forces follow the oracle's
law on the same list, overflowing buffers grow, and a whole step reaches
the plain Picard fixed point of the oracle.

Tolerances are those of the Picard tests of the implicit step: the fixed
points differ by at most about tol_F dt sum_c |F_c| max(1/m, R/I) / (1 - rho)
(tol_F the force parity bound of the form); the tests allow ten times
tol_F dt sum_c |F_c| max(1/m, R/I).  Surrogate forces: FP64 sums of the same
formula, 1e-12 relative."""
import dataclasses

import numpy as np
import pytest

from gen import scene_chain
from gpu_common import compare_contacts

pytestmark = pytest.mark.gpu

TOL_F = {"fp64": 1e-9, "fp32": 1e-5}


@pytest.fixture(scope="module")
def m():
    import paper_2105_12415_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def ctx(m):
    return m.Context(0)


@pytest.fixture(scope="module")
def mr(orc):
    from oracle import multires
    return multires


@pytest.fixture(scope="module")
def imp(orc):
    import oracle.implicit as imp
    return imp


def _t(a, dtype="float64"):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=getattr(torch, dtype), device="cuda:0")


@pytest.fixture(scope="module")
def chain(m, ctx, imp):
    s = scene_chain(4, seed=41)
    bound = imp.bounding_radius(s)
    pairs = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    eps = imp.pair_eps(s.radius, pairs[:, 0], pairs[:, 1])
    hier = m.Hierarchy.from_scene(ctx, s)
    return s, pairs, eps, hier, hier.export()


def _leaves(T, v):
    if T.leaf(v):
        return [int(v)]
    b, c = T.child[v]
    return [x for ch in range(b, b + c) for x in _leaves(T, ch)]


def _check_cut(T, items, pairs):
    for p, (A, B) in enumerate(pairs):
        want = sorted((x, y) for x in _leaves(T, T.root[A]) for y in _leaves(T, T.root[B]))
        got = sorted((x, y) for q, a, b, _ in items.tolist() if q == p
                     for x in _leaves(T, a) for y in _leaves(T, b))
        assert got == want, p


def _settle(m, ctx, hier, tp, te, poses, sets, precision, T=None, pairs=None, limit=20):
    """Steps at fixed poses until nothing widens or narrows; checks the cut
    property after each step when T is given.  Returns the last step's
    (sets, contacts, surrogate, counts) and the steps' counts."""
    other = None
    hist = []
    for _ in range(limit):
        out, con, sur, cnt = m.active_sets_step(ctx, hier, tp, te, poses, sets, other, precision)
        c = cnt.tolist()
        hist.append(c)
        if T is not None:
            _check_cut(T, out.to_numpy(), pairs)
        other, sets = sets, out
        if c[0] == 0 and c[1] == 0:
            return sets, con, sur, c, hist
    raise AssertionError(f"active sets did not settle: {hist}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_active_sets_are_cuts_and_find_every_contact(m, ctx, mr, orc, chain, precision):
    s, pairs, eps, hier, ex = chain
    T = mr.Trees(ex)
    tp, te, poses = _t(pairs, "int32"), _t(eps), _t(s.poses)
    sets = m.active_sets_init(ctx, hier, tp)
    assert sets.to_numpy().tolist() == [[p, int(T.root[A]), int(T.root[B]), 0]
                                        for p, (A, B) in enumerate(pairs)]
    sets, con, sur, c, hist = _settle(m, ctx, hier, tp, te, poses, sets, precision, T, pairs)
    assert hist[0][0] == len(pairs) and hist[0][3] >= 0   # the roots widen first
    assert c[3] == 0 and sur.n() == 0
    base = dataclasses.replace(s, pairs=pairs, eps=eps)
    ref = orc.detect(base)
    assert len(ref["d"]) > 0
    compare_contacts(con.to_numpy(), ref, base, precision)
    assert c[2] > 0 and sets.n() < sum(len(_leaves(T, T.root[A])) * len(_leaves(T, T.root[B]))
                                       for A, B in pairs)


def test_surrogate_contacts_and_forces(m, ctx, mr, chain):
    """The first step from the roots lists surrogate contacts (the implicit
    guess): nodes of the pair's own particles within delta_a + delta_b +
    2 eps; their forces equal the oracle's law on the same list."""
    import torch
    s, pairs, eps, hier, ex = chain
    T = mr.Trees(ex)
    tp, te, poses = _t(pairs, "int32"), _t(eps), _t(s.poses)
    sets = m.active_sets_init(ctx, hier, tp)
    sur = None
    for _ in range(4):
        sets, _, sur, cnt = m.active_sets_step(ctx, hier, tp, te, poses, sets, None, "fp64")
        if sur.n():
            break
    n = sur.n()
    assert n > 0
    sp = sur.pair[:n].cpu().numpy()
    a, b = sur.tri_a[:n].cpu().numpy(), sur.tri_b[:n].cpu().numpy()
    d = sur.dist[:n].cpu().numpy()
    assert np.array_equal(T.particle[a], pairs[sp, 0]) and np.array_equal(T.particle[b], pairs[sp, 1])
    tau = T.delta[a] + T.delta[b] + 2 * eps[sp]
    assert np.all(d >= 0) and np.all(d <= tau * (1 + 1e-6))
    pa, pb = sur.point_a[:n].cpu().numpy(), sur.point_b[:n].cpu().numpy()
    np.testing.assert_allclose(np.linalg.norm(pa - pb, axis=1), d, rtol=1e-12, atol=1e-15)
    mass, com = _t(s.mass), _t(np.zeros((s.n_particles, 3)))
    ft = torch.zeros((s.n_particles, 6), dtype=torch.float64, device="cuda:0")
    en = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    m.surrogate_forces(ctx, hier, tp, te, poses, sur, mass, com, 1000.0, 0.3, ft, en)
    nrm = np.zeros((n, 3))
    for k in range(n):
        W = T.tri[a[k]] @ orc_rot(s.poses[pairs[sp[k], 0]]).T
        nrm[k] = np.cross(W[1] - W[0], W[2] - W[0])
    want, e_want = mr.surrogate_forces(s, pairs, eps, s.poses,
                                       dict(pair=sp, d=d, pa=pa, pb=pb, tau=tau, n=nrm), 0.3)
    got = ft.cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    assert abs(en.item() - e_want) <= 1e-12 * e_want


def orc_rot(pose):
    import oracle
    return oracle.pose_matrix(pose)


def test_separated_pairs_narrow_to_their_roots(m, ctx, mr, chain):
    import torch
    s, pairs, eps, hier, ex = chain
    T = mr.Trees(ex)
    tp, te = _t(pairs, "int32"), _t(eps)
    sets = m.active_sets_init(ctx, hier, tp)
    sets, _, _, _, _ = _settle(m, ctx, hier, tp, te, _t(s.poses), sets, "fp64")
    flagged = sets.to_numpy()
    assert len(flagged) > len(pairs)
    far = s.poses.copy()
    far[:, :3] *= 20.0
    far = _t(far)
    # flags cleared: every group narrows back, one level per step
    clean = m.ActiveSets(sets.capacity, "cuda:0")
    clean.item[:len(flagged)] = torch.as_tensor(flagged * np.array([1, 1, 1, 0]), dtype=torch.int32,
                                                device="cuda:0")
    clean.count.fill_(len(flagged))
    got, _, _, c, hist = _settle(m, ctx, hier, tp, te, far, clean, "fp64", T, pairs)
    assert all(h[0] == 0 for h in hist) and sum(h[1] for h in hist) > 0
    assert got.to_numpy().tolist() == [[p, int(T.root[A]), int(T.root[B]), 2]
                                       for p, (A, B) in enumerate(pairs)]
    # flags kept: the items re-added after a narrowing (bit 0) stay
    vetoed = [tuple(x) for x in flagged.tolist() if x[3] & 1]
    kept, _, _, _, _ = _settle(m, ctx, hier, tp, te, far, sets, "fp64", T, pairs)
    have = set(map(tuple, kept.to_numpy().tolist()))
    assert all(v in have for v in vetoed)


def test_buffers_grow_and_the_step_repeats(m, ctx, chain):
    s, pairs, eps, hier, _ = chain
    tp, te, poses = _t(pairs, "int32"), _t(eps), _t(s.poses)
    big = m.active_sets_init(ctx, hier, tp)
    small = m.active_sets_init(ctx, hier, tp, out=m.ActiveSets(len(pairs), "cuda:0"))
    res = []
    for sets, cap in ((big, None), (small, 1)):
        out = m.ActiveSets(cap or 4096, "cuda:0")
        con = m.Contacts(cap or 4096, "cuda:0")
        sur = m.Contacts(cap or 4096, "cuda:0")
        for _ in range(3):
            out, con, sur, cnt = m.active_sets_step(ctx, hier, tp, te, poses, sets, out, "fp64",
                                                    con, sur)
            sets, out = out, sets
        res.append((sets.to_numpy(), con.to_numpy(), cnt.tolist()))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][2] == res[1][2]
    for k in ("pair", "ta", "tb", "d"):
        assert np.array_equal(res[0][1][k], res[1][1][k])


def _fixed_point_bound(orc, s, pairs, eps, P, dt, precision):
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((s.n_particles, 3)))
    c = orc.detect(base, poses=P)
    mu = 1 / (1 / s.mass[pairs[:, 0]] + 1 / s.mass[pairs[:, 1]])
    mag = 1000.0 * np.sqrt(mu[c["pair"]]) * (1 - c["d"] / (2 * eps[c["pair"]]))
    tot = np.zeros(s.n_particles)
    for col in (0, 1):
        np.add.at(tot, pairs[c["pair"], col], mag)
    inertia = 0.4 * s.mass * s.radius ** 2
    lever = np.array([np.sqrt((s.particle(i)[0].astype(np.float64) ** 2).sum(1)).max()
                      for i in range(s.n_particles)])
    return 10.0 * TOL_F[precision] * dt * (tot * np.maximum(1 / s.mass, lever / inertia)).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_multires_step_reaches_the_oracle_fixed_point(m, ctx, orc, imp, chain, precision, tol):
    s, pairs, eps, hier, _ = chain
    rng = np.random.default_rng(2)
    vel = rng.normal(scale=0.1, size=(s.n_particles, 6))
    dt = 2e-4
    P, V, it_ref, _ = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=2e-13, max_iter=2000)
    inertia = 0.4 * s.mass * s.radius ** 2
    poses, Vg, it, hist, rec = m.implicit_euler_step_multires(
        ctx, hier, _t(s.poses), _t(vel), _t(s.mass), _t(inertia), _t(pairs, "int32"), _t(eps), dt,
        precision=precision, tol=tol, max_iter=200)
    assert it < 200, hist[-5:]
    assert rec[0]["widened"] == len(pairs) and any(r["surrogate"] > 0 for r in rec)
    assert rec[-1]["widened"] == 0 and rec[-1]["narrowed"] == 0 and rec[-1]["surrogate"] == 0
    lim = _fixed_point_bound(orc, s, pairs, eps, P, dt, precision) + tol * np.abs(V).max() * 10
    assert np.abs(Vg.cpu().numpy() - V).max() <= lim
    assert np.abs(poses.cpu().numpy() - P).max() <= dt * lim + 1e-14 * (1.0 + np.abs(P).max())
