"""The implicit time step on the GPU (Algorithm 3) against the FP64 oracle:
the uniform-grid broad phase (bit-exact pair list and eps), the rigid-body
pose update, the Picard velocity update, and whole Picard steps whose fixed
point is compared with the oracle's.

Tolerances.  The broad phase takes the same FP64 decisions as the oracle, so
its list must be identical.  Pose updates agree to a few ulps (sin / cos of
the rotation angle).  A Picard step's fixed point V solves
V = v0 + dt M^-1 F(V); the contact forces of the two sides differ by at most
tol_F sum_c |F_c| per particle (tol_F = 1e-9 for the FP64 form, 1e-5 for
FP32, the bounds of the force parity tests), so the fixed points differ by
at most about tol_F dt sum_c |F_c| max(1/m, R/I) times 1 / (1 - rho), rho the
contraction of the iteration (about 0.2 on the chain); the tests allow ten
times tol_F dt sum_c |F_c| max(1/m, R/I), taken over particles.  The chain
has no crossing triangles (d > 0.5 eps throughout the step), where the
force direction would be a convention.
"""
import dataclasses

import numpy as np
import pytest

from gen import scene_chain, scene_packing

pytestmark = pytest.mark.gpu

TOL_F = {"fp64": 1e-9, "fp32": 1e-5}


@pytest.fixture(scope="module")
def m():
    import paper_2105_12415_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def imp(orc):
    import oracle.implicit as imp
    return imp


@pytest.fixture(scope="module")
def ctx(m):
    return m.Context(0)


def _t(a, dtype="float64"):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=getattr(torch, dtype), device="cuda:0")


def _bound(scene):
    """Largest vertex distance from the body origin, per particle (FP64 of
    the float vertices)."""
    return np.array([np.sqrt((scene.particle(i)[0].astype(np.float64) ** 2).sum(1)).max()
                     for i in range(scene.n_particles)])


@pytest.mark.parametrize("n,fraction,levels,seed", [(300, 0.35, (1, 2), 1), (2000, 0.5, (1,), 2),
                                                    (50, 0.55, (1, 2), 3)])
def test_broad_phase_equals_oracle(m, ctx, imp, n, fraction, levels, seed):
    s, _, _ = scene_packing(n, fraction, levels=levels, r_min=1.0, r_max=10.0, seed=seed)
    bound = _bound(s)
    ref = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    ref_eps = imp.pair_eps(s.radius, ref[:, 0], ref[:, 1])
    assert len(ref) > n // 10
    pairs, eps = m.broad_phase(ctx, _t(s.poses), _t(bound), _t(s.radius))
    assert np.array_equal(pairs.cpu().numpy(), ref)
    assert np.array_equal(eps.cpu().numpy(), ref_eps)


def test_broad_phase_grows_and_repeats(m, ctx, imp):
    s, _, _ = scene_packing(300, 0.35, levels=(1, 2), r_min=1.0, r_max=10.0, seed=1)
    bound = _bound(s)
    ref = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    pairs, _ = m.broad_phase(ctx, _t(s.poses), _t(bound), _t(s.radius), cap=3)
    assert np.array_equal(pairs.cpu().numpy(), ref)


def test_broad_phase_edge_cases(m, ctx, imp):
    # no particle, one particle
    for n in (0, 1):
        P = np.zeros((n, 7))
        P[:, 3] = 1.0
        pairs, eps = m.broad_phase(ctx, _t(P), _t(np.ones(n)), _t(np.ones(n)))
        assert pairs.shape == (0, 2) and eps.shape == (0,)
    # coincident points of zero size: every pair, in (i, j) order
    P = np.zeros((5, 7))
    P[:, 3] = 1.0
    pairs, eps = m.broad_phase(ctx, _t(P), _t(np.zeros(5)), _t(np.zeros(5)))
    assert pairs.cpu().numpy().tolist() == [[i, j] for i in range(5) for j in range(i + 1, 5)]
    assert (eps.cpu().numpy() == 0).all()
    # two clusters 1e12 apart (cell coordinates clamped) and touching spheres
    # exactly at the limit distance
    rng = np.random.default_rng(0)
    P = np.zeros((42, 7))
    P[:, 3] = 1.0
    P[:20, :3] = rng.normal(size=(20, 3))
    P[20:40, :3] = 1e12 + rng.normal(size=(20, 3))
    P[40, :3] = (5.0, 5.0, 5.0)
    P[41, :3] = (5.0, 5.0, 6.02)  # at the limit 0.5 + 0.5 + 2 * 0.01, up to rounding
    b = np.full(42, 0.5)
    r = np.full(42, 0.5)
    ref = imp.broad_phase(P[:, :3], b, r)
    pairs, _ = m.broad_phase(ctx, _t(P), _t(b), _t(r))
    assert np.array_equal(pairs.cpu().numpy(), ref)


def test_broad_phase_rejects_nonfinite(m, ctx, imp):
    P = np.zeros((4, 7))
    P[:, 3] = 1.0
    P[:, 0] = np.arange(4)
    P[2, 1] = np.nan
    with pytest.raises(m.MrdemError):
        m.broad_phase(ctx, _t(P), _t(np.ones(4)), _t(np.ones(4)))
    # the context stays usable
    P[2, 1] = 0.0
    pairs, _ = m.broad_phase(ctx, _t(P), _t(np.ones(4)), _t(np.ones(4)))
    # unit spheres at x = 0..3: five pairs lie within 2 + 2 eps, (0, 3) does not
    ref = imp.broad_phase(P[:, :3], np.ones(4), np.ones(4))
    assert len(ref) == 5
    assert np.array_equal(pairs.cpu().numpy(), ref)


def test_move_poses_equals_oracle(m, ctx, imp):
    s, _, _ = scene_packing(200, 0.3, levels=(1,), seed=5)
    rng = np.random.default_rng(7)
    V = rng.normal(size=(200, 6)) * 3.0
    V[0, 3:] = 0.0  # no rotation
    for dt in (1e-3, 0.5):
        got = m.move_poses(ctx, _t(s.poses), _t(V), dt).cpu().numpy()
        ref = imp.moved_poses(s.poses, V, dt)
        assert np.abs(got - ref).max() <= 1e-14 * (1.0 + np.abs(ref).max())
        assert np.abs(np.linalg.norm(got[:, 3:], axis=1) - 1.0).max() <= 1e-15
    # in place
    P = _t(s.poses)
    m.move_poses(ctx, P, _t(V), 1e-3, out=P)
    assert np.abs(P.cpu().numpy() - imp.moved_poses(s.poses, V, 1e-3)).max() <= 1e-14 * (1.0 + np.abs(s.poses).max())


def test_picard_update_closed_form(m, ctx):
    rng = np.random.default_rng(8)
    n = 1000
    v0 = rng.normal(size=(n, 6))
    guess = rng.normal(size=(n, 6))
    ft = rng.normal(size=(n, 6)) * 100.0
    mass = rng.uniform(0.5, 2.0, n)
    inertia = rng.uniform(0.1, 1.0, n)
    g = (0.5, -1.0, -9.81)
    dt = 1e-3
    vel = _t(guess)
    norms = m.picard_update(ctx, _t(v0), _t(ft), _t(mass), _t(inertia), dt, vel, gravity=g)
    want = np.empty((n, 6))
    want[:, :3] = v0[:, :3] + dt * (ft[:, :3] / mass[:, None] + np.array(g))
    want[:, 3:] = v0[:, 3:] + dt * ft[:, 3:] / inertia[:, None]
    # the kernel rounds operation by operation in the formula's order
    assert np.array_equal(vel.cpu().numpy(), want)
    c, sc = norms.cpu().numpy()
    assert c == np.abs(want - guess).max()
    assert sc == np.abs(want).max()


def _chain_problem(imp):
    s = scene_chain(4, seed=41)
    bound = _bound(s)
    pairs = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    eps = imp.pair_eps(s.radius, pairs[:, 0], pairs[:, 1])
    rng = np.random.default_rng(2)
    vel = rng.normal(scale=0.1, size=(s.n_particles, 6))
    return s, bound, pairs, eps, vel


_ORACLE_STEPS = {}


def _oracle_step(imp, key, s, vel, pairs, eps, dt):
    """The oracle's Picard fixed point of a test case, computed once per
    module (several tests compare with it)."""
    if key not in _ORACLE_STEPS:
        _ORACLE_STEPS[key] = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=2e-13,
                                                     max_iter=2000)
    return _ORACLE_STEPS[key]


def _fixed_point_bound(orc, s, pairs, eps, P, dt, precision):
    """ten times tol_F dt sum_c |F_c| max(1/m, R/I), the largest over
    particles, at the oracle's final geometry"""
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((s.n_particles, 3)))
    c = orc.detect(base, poses=P)
    mu = 1 / (1 / s.mass[pairs[:, 0]] + 1 / s.mass[pairs[:, 1]])
    mag = 1000.0 * np.sqrt(mu[c["pair"]]) * (1 - c["d"] / (2 * eps[c["pair"]]))
    tot = np.zeros(s.n_particles)
    for col in (0, 1):
        np.add.at(tot, pairs[c["pair"], col], mag)
    inertia = 0.4 * s.mass * s.radius ** 2
    lever = _bound(s)
    return 10.0 * TOL_F[precision] * dt * (tot * np.maximum(1 / s.mass, lever / inertia)).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_picard_map_at_oracle_fixed_point(m, ctx, orc, imp, precision):
    """One GPU Picard iteration started from the oracle's fixed point returns
    it, within the force tolerance."""
    s, _, pairs, eps, vel = _chain_problem(imp)
    dt = 2e-4
    P, V, it, _ = _oracle_step(imp, "chain", s, vel, pairs, eps, dt)
    assert it < 2000
    hier = m.Hierarchy.from_scene(ctx, s)
    inertia = 0.4 * s.mass * s.radius ** 2
    poses = m.move_poses(ctx, _t(s.poses), _t(V), dt)
    assert np.abs(poses.cpu().numpy() - P).max() <= 1e-14 * (1.0 + np.abs(P).max())
    tp, te = _t(pairs, "int32"), _t(eps)
    contacts, _ = m.detect(ctx, hier, tp, te, poses, precision)
    ft, _ = m.contact_forces(ctx, hier, tp, te, poses, contacts, _t(s.mass),
                             _t(np.zeros((s.n_particles, 3))))
    V1 = _t(V)
    m.picard_update(ctx, _t(vel), ft, _t(s.mass), _t(inertia), dt, V1)
    bound = _fixed_point_bound(orc, s, pairs, eps, P, dt, precision) / 10.0
    assert np.abs(V1.cpu().numpy() - V).max() <= bound + 1e-12 * np.abs(V).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_implicit_step_equals_oracle(m, ctx, orc, imp, precision, tol):
    s, bound, pairs, eps, vel = _chain_problem(imp)
    dt = 2e-4
    P, V, it_ref, _ = _oracle_step(imp, "chain", s, vel, pairs, eps, dt)
    hier = m.Hierarchy.from_scene(ctx, s)
    inertia = 0.4 * s.mass * s.radius ** 2
    # pairs from the GPU broad phase, as a user would run it
    gp, ge = m.broad_phase(ctx, _t(s.poses), _t(bound), _t(s.radius))
    assert np.array_equal(gp.cpu().numpy(), pairs)
    poses, Vg, it, hist = m.implicit_euler_step(ctx, hier, _t(s.poses), _t(vel), _t(s.mass),
                                                _t(inertia), gp, ge, dt, precision=precision,
                                                tol=tol, max_iter=200)
    assert it < 200, hist[-5:]
    lim = _fixed_point_bound(orc, s, pairs, eps, P, dt, precision) + tol * np.abs(V).max() * 10
    assert np.abs(Vg.cpu().numpy() - V).max() <= lim
    assert np.abs(poses.cpu().numpy() - P).max() <= dt * lim + 1e-14 * (1.0 + np.abs(P).max())
    if precision == "fp64":
        assert it <= it_ref + 2  # a looser tolerance than the oracle's stops no later


def test_free_flight_is_exact(m, ctx, imp):
    """No candidate pairs: one iteration gives v0 + dt g exactly."""
    s, _, _ = scene_packing(30, 0.05, levels=(1,), seed=9)
    rng = np.random.default_rng(3)
    vel = rng.normal(size=(s.n_particles, 6))
    dt = 1e-3
    hier = m.Hierarchy.from_scene(ctx, s)
    inertia = 0.4 * s.mass * s.radius ** 2
    empty_p = _t(np.zeros((0, 2)), "int32")
    empty_e = _t(np.zeros(0))
    poses, V, it, _ = m.implicit_euler_step(ctx, hier, _t(s.poses), _t(vel), _t(s.mass),
                                            _t(inertia), empty_p, empty_e, dt)
    Pr, Vr, _, _ = imp.implicit_euler_step(s, vel, np.zeros((0, 2), np.int32), np.zeros(0), dt)
    assert it == 2
    assert np.array_equal(V.cpu().numpy(), Vr)
    assert np.abs(poses.cpu().numpy() - Pr).max() <= 1e-14 * (1.0 + np.abs(Pr).max())


def _hessian_scenes(imp):
    from tests.test_oracle_implicit import FACING, _colliding_pair, _icosahedra_facing
    out = [_icosahedra_facing(a, b) for a, b in FACING]
    for seed in (4, 8):
        s, _, pairs, eps = _colliding_pair(imp, seed=seed)
        out.append(dataclasses.replace(s, pairs=pairs, eps=eps))
    s, _, pairs, eps, _ = _chain_problem(imp)
    out.append(dataclasses.replace(s, pairs=pairs, eps=eps))
    return [dataclasses.replace(s, com=np.zeros((s.n_particles, 3))) for s in out]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_contact_hessian_equals_oracle(m, ctx, orc, imp, precision):
    """The per-pair 12x12 contact Hessian blocks, assembled, equal the
    oracle's closed-form Hessian (an independent implementation: the general
    elimination over the six corners) to 1e-10 of its largest entry; every
    feature pair occurs (vertex-face, crossing edges, vertex-edge,
    vertex-vertex).  The closest points are recomputed in FP64, so the
    FP32-form detection gives the same blocks (no contact lies within 1e-3
    eps of the threshold 2 eps, where the contact sets may differ)."""
    for s in _hessian_scenes(imp):
        ref_c = orc.detect(s)
        assert (np.abs(ref_c["d"] - 2 * s.eps[ref_c["pair"]]) > 1e-3 * s.eps[ref_c["pair"]]).all()
        Href = imp.contact_hessian(s, ref_c)
        hier = m.Hierarchy.from_scene(ctx, s)
        tp, te, tposes, tmass = _t(s.pairs, "int32"), _t(s.eps), _t(s.poses), _t(s.mass)
        contacts, _ = m.detect(ctx, hier, tp, te, tposes, precision)
        if precision == "fp64":
            assert contacts.n() == len(ref_c["d"])
        # (the FP32 form may list a pair just beyond 2 eps; the blocks
        # recompute distances in FP64 and skip it)
        blocks, skipped = m.contact_hessian(ctx, hier, tp, te, tposes, contacts, tmass)
        assert int(skipped.item()) == 0
        H = np.zeros_like(Href)
        for p, (a, b) in enumerate(s.pairs):
            idx = np.r_[6 * a:6 * a + 6, 6 * b:6 * b + 6]
            H[np.ix_(idx, idx)] += blocks[p].cpu().numpy()
        assert np.abs(H - Href).max() <= 1e-10 * np.abs(Href).max()


def test_newton_residual_closed_form(m, ctx):
    rng = np.random.default_rng(11)
    n = 500
    v0, v, ft = rng.normal(size=(n, 6)), rng.normal(size=(n, 6)), rng.normal(size=(n, 6)) * 50
    mass, inertia = rng.uniform(0.5, 2.0, n), rng.uniform(0.1, 1.0, n)
    dt, g = 1e-3, (0.3, 0.0, -9.81)
    res, norms = m.newton_residual(ctx, _t(v0), _t(v), _t(ft), _t(mass), _t(inertia), dt, gravity=g)
    Md = np.concatenate([np.repeat(mass[:, None], 3, 1), np.repeat(inertia[:, None], 3, 1)], 1)
    gext = np.zeros((n, 6))
    gext[:, :3] = mass[:, None] * np.array(g)
    want = (Md * (v - v0)) / dt - ft - gext
    assert np.array_equal(res.cpu().numpy(), want)
    rn, sc = norms.cpu().numpy()
    assert rn == np.abs(want).max() and sc == np.abs(Md * v).max() / dt


def _system(rng, n, pairs, spd=True):
    P = len(pairs)
    Q = rng.normal(size=(P, 12, 12))
    blocks = Q @ Q.transpose(0, 2, 1) if spd else -50.0 * np.repeat(np.eye(12)[None], P, 0)
    mass, inertia = rng.uniform(0.5, 2.0, n), rng.uniform(0.1, 1.0, n)
    return blocks, mass, inertia


def _assemble(n, pairs, blocks, mass, inertia, dt):
    Md = np.concatenate([np.repeat(mass[:, None], 3, 1), np.repeat(inertia[:, None], 3, 1)], 1).ravel()
    A = np.diag(Md / dt)
    for p, (a, b) in enumerate(pairs):
        idx = np.r_[6 * a:6 * a + 6, 6 * b:6 * b + 6]
        A[np.ix_(idx, idx)] += dt * blocks[p]
    return A, Md


def test_newton_solve_conjugate_gradients(m, ctx):
    """The preconditioned conjugate-gradient solve of (M/dt + dt K) x = b
    equals a dense solve of the assembled matrix (K positive semi-definite
    pair blocks on a random pair graph, particles sharing several pairs)."""
    rng = np.random.default_rng(12)
    n = 40
    pairs = np.array(sorted({tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(90)}),
                     np.int32)
    blocks, mass, inertia = _system(rng, n, pairs)
    dt = 0.05
    A, _ = _assemble(n, pairs, blocks, mass, inertia, dt)
    b = rng.normal(size=(n, 6))
    x, info = m.newton_solve(ctx, _t(pairs, "int32"), _t(blocks), _t(mass), _t(inertia), dt, _t(b),
                             max_iter=400, rel_tol=1e-13)
    want = np.linalg.solve(A, b.ravel()).reshape(n, 6)
    it, rel, brk, bn = info.cpu().numpy()
    assert brk == 0 and 0 < it < 400 and rel <= 1e-13
    assert abs(bn - np.linalg.norm(b)) <= 1e-12 * bn
    assert np.abs(x.cpu().numpy() - want).max() <= 1e-10 * np.abs(want).max()
    # the same solve, stopped from the host every 4 iterations
    x4, info4 = m.newton_solve(ctx, _t(pairs, "int32"), _t(blocks), _t(mass), _t(inertia), dt,
                               _t(b), max_iter=400, rel_tol=1e-13, check_every=4)
    assert info4.cpu().numpy()[2] == 0 and info4.cpu().numpy()[1] <= 1e-13
    assert np.abs(x4.cpu().numpy() - want).max() <= 1e-10 * np.abs(want).max()
    # no pairs: x = b dt / M exactly up to rounding, in one iteration
    x0, info0 = m.newton_solve(ctx, _t(np.zeros((0, 2)), "int32"), _t(np.zeros((0, 12, 12))),
                               _t(mass), _t(inertia), dt, _t(b), max_iter=10, rel_tol=1e-14)
    Md = np.concatenate([np.repeat(mass[:, None], 3, 1), np.repeat(inertia[:, None], 3, 1)], 1)
    assert np.abs(x0.cpu().numpy() - b * dt / Md).max() <= 1e-14 * np.abs(b * dt / Md).max()
    assert info0.cpu().numpy()[0] == 1
    # zero right-hand side: x = 0, no iteration
    xz, infoz = m.newton_solve(ctx, _t(pairs, "int32"), _t(blocks), _t(mass), _t(inertia), dt,
                               _t(np.zeros((n, 6))), max_iter=10)
    assert (xz.cpu().numpy() == 0).all() and infoz.cpu().numpy()[0] == 0


def test_newton_solve_reports_negative_curvature(m, ctx):
    """Blocks that make the matrix indefinite along the first direction stop
    the solve at once with the breakdown flag and a step along that
    direction, (r.z / |p.Ap|) p with p = z = b / diag (an entry of the
    diagonal that is not positive uses M/dt)."""
    rng = np.random.default_rng(13)
    n = 6
    pairs = np.array([[0, 1], [2, 3], [4, 5]], np.int32)
    blocks, mass, inertia = _system(rng, n, pairs, spd=False)
    dt = 0.5
    A, Md = _assemble(n, pairs, blocks, mass, inertia, dt)
    b = rng.normal(size=(n, 6))
    x, info = m.newton_solve(ctx, _t(pairs, "int32"), _t(blocks), _t(mass), _t(inertia), dt, _t(b),
                             max_iter=10)
    d = np.diag(A)
    d = np.where(d > 0, d, Md / dt)
    z = b.ravel() / d
    pap = z @ A @ z
    assert pap < 0
    it, _, brk, _ = info.cpu().numpy()
    assert brk == 1 and it == 0
    want = (b.ravel() @ z) / -pap * z
    assert np.abs(x.cpu().numpy().ravel() - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("case", [4, 8, "chain"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_newton_step_reaches_the_picard_fixed_point(m, ctx, orc, imp, case, precision, tol):
    """Newton's method on the GPU (contact Hessian blocks, conjugate
    gradients, backtracking) reaches the oracle's Picard fixed point in a
    handful of iterations (the oracle's Newton needs 5 to 10 here, Picard
    18 to 149), within the fixed-point bound of the Picard test."""
    from tests.test_oracle_implicit import _colliding_pair
    if case == "chain":
        s, _, pairs, eps, vel = _chain_problem(imp)
        dt = 2e-4
    else:
        s, vel, pairs, eps = _colliding_pair(imp, seed=case)
        dt = 5e-4
    P, V, _, _ = _oracle_step(imp, case, s, vel, pairs, eps, dt)
    hier = m.Hierarchy.from_scene(ctx, s)
    inertia = 0.4 * s.mass * s.radius ** 2
    poses, Vg, it, stats = m.implicit_euler_step_newton(
        ctx, hier, _t(s.poses), _t(vel), _t(s.mass), _t(inertia), _t(pairs, "int32"), _t(eps), dt,
        precision=precision, tol=tol, max_iter=30)
    assert it < (16 if precision == "fp64" else 30), stats
    lim = _fixed_point_bound(orc, s, pairs, eps, P, dt, precision) + 10 * tol * np.abs(V).max()
    assert np.abs(Vg.cpu().numpy() - V).max() <= lim, (np.abs(Vg.cpu().numpy() - V).max(), lim)


def test_picard_iterations_replayed_from_a_cuda_graph(m, ctx, imp):
    """The Picard iteration captured once into a CUDA graph and replayed
    gives the uncaptured loop's result (the force sums' atomics may order
    additions differently, so to 1e-12) in as many iterations, give or take
    one; a context with tiny work lists grows them in the first, checked
    iteration and then replays as well."""
    s, _, pairs, eps, vel = _chain_problem(imp)
    dt = 2e-4
    inertia = 0.4 * s.mass * s.radius ** 2
    hier = m.Hierarchy.from_scene(ctx, s)
    args = (_t(s.poses), _t(vel), _t(s.mass), _t(inertia), _t(pairs, "int32"), _t(eps), dt)
    P1, V1, it1, _ = m.implicit_euler_step(ctx, hier, *args, precision="fp64", tol=1e-11)
    P2, V2, it2, _ = m.implicit_euler_step(ctx, hier, *args, precision="fp64", tol=1e-11,
                                           graph=True)
    assert abs(it1 - it2) <= 1
    scale = V1.abs().max().item()
    assert (V1 - V2).abs().max().item() <= 1e-12 * scale
    assert (P1 - P2).abs().max().item() <= 1e-12 * (1.0 + P1.abs().max().item())
    small = m.Context(0, cap_level=64, cap_tiles=64, cap_candidates=64, cap_sweep=64)
    hs = m.Hierarchy.from_scene(small, s)
    _, V3, it3, _ = m.implicit_euler_step(small, hs, *args, precision="fp64", tol=1e-11,
                                          graph=True)
    assert abs(it1 - it3) <= 1
    assert (V1 - V3).abs().max().item() <= 1e-12 * scale


def test_motion_bound_closed_form(m, ctx):
    """A translation moves every point by its length; a rotation by angle a
    about the origin moves a point at distance R by at most a R; the bound
    is the largest over the particles."""
    def one(t, axis, a, R):
        P0 = np.array([[0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]])
        P1 = P0.copy()
        P1[0, :3] = t
        P1[0, 3:] = np.concatenate([[np.cos(a / 2)], np.sin(a / 2) * np.asarray(axis)])
        return m.motion_bound(ctx, _t(P0), _t(P1), _t(np.array([R]))).item()
    assert abs(one((0.3, -0.4, 0.0), (0, 0, 1), 0.0, 2.0) - 0.5) <= 1e-15
    assert abs(one((0.0, 0.0, 0.0), (0, 0, 1), 0.2, 5.0) - 1.0) <= 1e-14
    assert abs(one((0.0, 0.0, 0.1), (1, 0, 0), 0.1, 3.0) - 0.4) <= 1e-14
    assert abs(one((0.0, 0.0, 0.0), (0, 1, 0), -0.3, 1.0) - 0.3) <= 1e-14
    P0 = np.zeros((3, 7))
    P0[:, 3] = 1.0
    P1 = P0.copy()
    P1[0, :3] = (0.3, -0.4, 0.0)
    P1[1, 3:] = (np.cos(0.1), 0.0, 0.0, np.sin(0.1))
    got = m.motion_bound(ctx, _t(P0), _t(P1), _t(np.array([1.0, 5.0, 3.0]))).item()
    assert abs(got - 1.0) <= 1e-14
    assert m.motion_bound(ctx, _t(P0), _t(P0), _t(np.ones(3))).item() == 0.0


def _perturbed(poses, rng, step):
    """Poses moved by a translation of length step * (1 + |rng|) and a
    rotation by an angle of at most step about a random axis."""
    out = np.array(poses, copy=True)
    for i in range(len(out)):
        u = rng.normal(size=3)
        out[i, :3] += step * u / np.linalg.norm(u)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        a = step * rng.uniform(0.5, 1.0)
        w, v = np.cos(a / 2), np.sin(a / 2) * ax
        q = out[i, 3:]
        qn = np.concatenate([[w * q[0] - v @ q[1:]], w * q[1:] + q[0] * v + np.cross(v, q[1:])])
        out[i, 3:] = qn / np.linalg.norm(qn)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_refined_candidates_equal_detection(m, ctx, orc, imp, precision):
    """Candidates detected at eps + w at reference poses, refined at poses
    whose points moved by at most w, give the contact set of a detection at
    those poses (the oracle's), with FP64 distances."""
    from tests.gpu_common import compare_contacts
    s, bound, pairs, eps, _ = _chain_problem(imp)
    hier = m.Hierarchy.from_scene(ctx, s)
    w = 0.25 * eps.min()
    rng = np.random.default_rng(21)
    moved = _perturbed(s.poses, rng, 0.4 * w / (1.0 + bound.max()))   # points move by < w / 2
    tp, te = _t(pairs, "int32"), _t(eps)
    mb = m.motion_bound(ctx, _t(s.poses), _t(moved), _t(bound)).item()
    assert 0 < mb <= w
    cand, _ = m.detect(ctx, hier, tp, _t(eps + w), _t(s.poses), precision)
    got = m.refine_contacts(ctx, hier, tp, te, _t(moved), cand).to_numpy()
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((s.n_particles, 3)))
    ref = orc.detect(base, poses=moved)
    assert len(ref["d"]) > 50 and cand.n() >= len(ref["d"])
    compare_contacts(got, ref, base, "fp64", poses=moved)


def test_picard_with_kept_candidates(m, ctx, imp):
    """The Picard step taking each iteration's contacts from candidates kept
    across the step (detected once at eps + w) gives the step of the full
    detection (FP64 form) to 1e-12 in as many iterations."""
    s, bound, pairs, eps, vel = _chain_problem(imp)
    dt = 2e-4
    inertia = 0.4 * s.mass * s.radius ** 2
    hier = m.Hierarchy.from_scene(ctx, s)
    args = (_t(s.poses), _t(vel), _t(s.mass), _t(inertia), _t(pairs, "int32"), _t(eps), dt)
    P1, V1, it1, _ = m.implicit_euler_step(ctx, hier, *args, precision="fp64", tol=1e-11)
    P2, V2, it2, _ = m.implicit_euler_step(ctx, hier, *args, precision="fp64", tol=1e-11,
                                           cache_margin=0.25 * eps.min(), bound=_t(bound))
    assert abs(it1 - it2) <= 1
    assert (V1 - V2).abs().max().item() <= 1e-12 * V1.abs().max().item()


def test_kept_candidates_detect_again_only_beyond_the_margin(m, ctx, orc, imp):
    """Poses within w of the last detection reuse its candidates; poses
    beyond w trigger a new detection; every call returns the oracle's
    contact set at its poses."""
    from tests.gpu_common import compare_contacts
    s, bound, pairs, eps, _ = _chain_problem(imp)
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((s.n_particles, 3)))
    hier = m.Hierarchy.from_scene(ctx, s)
    w = 0.25 * eps.min()
    kept = m.KeptCandidates(ctx, hier, _t(pairs, "int32"), _t(eps), w, _t(bound), "fp64")
    rng = np.random.default_rng(22)
    near = _perturbed(s.poses, rng, 0.4 * w / (1.0 + bound.max()))
    far = _perturbed(s.poses, rng, 3.0 * w / (1.0 + bound.max()))
    for poses, detections in ((s.poses, 1), (near, 1), (far, 2), (s.poses, 3)):
        got = kept.contacts(_t(poses)).to_numpy()
        assert kept.detections == detections
        compare_contacts(got, orc.detect(base, poses=poses), base, "fp64", poses=poses)


def test_newton_with_kept_candidates(m, ctx, imp):
    s, bound, pairs, eps, vel = _chain_problem(imp)
    dt = 2e-4
    inertia = 0.4 * s.mass * s.radius ** 2
    hier = m.Hierarchy.from_scene(ctx, s)
    args = (_t(s.poses), _t(vel), _t(s.mass), _t(inertia), _t(pairs, "int32"), _t(eps), dt)
    _, V1, it1, _ = m.implicit_euler_step_newton(ctx, hier, *args, precision="fp64", tol=1e-12)
    _, V2, it2, _ = m.implicit_euler_step_newton(ctx, hier, *args, precision="fp64", tol=1e-12,
                                                 cache_margin=0.25 * eps.min(), bound=_t(bound))
    assert abs(it1 - it2) <= 1
    assert (V1 - V2).abs().max().item() <= 1e-10 * V1.abs().max().item()


def test_newton_with_gauss_newton_blocks(m, ctx, imp):
    """Newton's method with the adjoint's Gauss-Newton blocks (closest points
    frozen) as stiffness reaches the same fixed point as with the contact
    Hessian, in more iterations (it converges linearly)."""
    s, bound, pairs, eps, vel = _chain_problem(imp)
    dt = 2e-4
    inertia = 0.4 * s.mass * s.radius ** 2
    hier = m.Hierarchy.from_scene(ctx, s)
    args = (_t(s.poses), _t(vel), _t(s.mass), _t(inertia), _t(pairs, "int32"), _t(eps), dt)
    _, V1, it1, _ = m.implicit_euler_step_newton(ctx, hier, *args, precision="fp64", tol=1e-12)
    _, V2, it2, st2 = m.implicit_euler_step_newton(ctx, hier, *args, precision="fp64", tol=1e-12,
                                                   max_iter=200, stiffness="gauss-newton")
    assert it2 < 200 and it2 >= it1
    assert not any(st["cg_breakdown"] for st in st2)
    assert (V1 - V2).abs().max().item() <= 1e-10 * V1.abs().max().item()
