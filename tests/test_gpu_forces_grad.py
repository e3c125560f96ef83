"""Penalty forces (Sec. 2) and the adjoint kernel on the GPU through the C ABI
against the FP64 oracle, central finite differences and the autograd wrapper."""
import numpy as np
import pytest

from gen import scene_c1, scene_c3, scene_pairs
from tests.gpu_common import gpu_scene_tensors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    import paper_2105_12415_gb300 as m
    m.build()
    return m.Context(0)


def _problem(gctx, s, precision):
    import torch
    import paper_2105_12415_gb300 as m
    hier = m.Hierarchy.from_scene(gctx, s)
    return m.ContactProblem.from_scene(gctx, hier, s, torch.device("cuda:0"), precision=precision)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_forces_match_oracle(gctx, orc, precision, tol):
    """Per particle |F - F_ref| <= tol sum_c |F_c| + sum_c a_c, where a_c is
    the effect of the rounding floors (tests/gpu_common.py) on contact c's
    force K sqrt(mu) (1 - d/2eps) u: K sqrt(mu) f_d / (2 eps) through the
    magnitude (distance floor f_d = K_U u S), plus |F_c| min(2, 2 f_p / d_c)
    through the direction u = (pa - pb)/d, whose error is at most 2 f_p / d
    (closest-point floor f_p = K_P u S; at d = 0 on either side the
    direction is a convention, hence the cap of 2 |F_c|).  Torques: the
    same times the largest lever.  The largest measured fraction of each
    bound is printed."""
    from tests.gpu_common import K_P, K_U, U, world_scale
    for s in (scene_c1(), scene_pairs([2, 3, 1], [3, 1, 2], [1.0, 0.3, 0.5], [0.4, 1.0, 0.5],
                                      [0.004, 0.003, 0.005], [-0.01, 0.0, 0.002], 13, "forces")):
        prob = _problem(gctx, s, precision)
        prob.detect()
        ft, e = prob.forces()
        ref = orc.detect(s)
        ft_ref, e_ref = orc.forces(s, ref)
        ft = ft.cpu().numpy()
        mu = 1 / (1 / s.mass[s.pairs[:, 0]] + 1 / s.mass[s.pairs[:, 1]])
        ks = 1000 * np.sqrt(mu[ref["pair"]])
        eps = s.eps[ref["pair"]]
        mag = ks * (1 - ref["d"] / (2 * eps))
        uS = U * world_scale(s)[ref["pair"]]
        cond = (ks * K_U * uS / (2 * eps)
                + mag * np.minimum(2.0, 2 * K_P * uS / np.maximum(ref["d"], 1e-300)))
        band = mag * (np.abs(ref["d"] - 2 * eps) <= 1e-6 * eps)
        tot = np.zeros(s.n_particles)
        extra = np.zeros(s.n_particles)
        for col in (0, 1):
            np.add.at(tot, s.pairs[ref["pair"], col], mag)
            np.add.at(extra, s.pairs[ref["pair"], col], cond + band)
        lim = (tol * tot + extra)[:, None]
        lever = 2 * (s.radius.max() + np.abs(s.poses[:, :3]).max())
        ferr = np.abs(ft[:, :3] - ft_ref[:, :3])
        terr = np.abs(ft[:, 3:] - ft_ref[:, 3:])
        print(f"{s.name} {precision}: force error / bound {float((ferr / lim).max()):.3g}, "
              f"torque {float((terr / (lim * lever)).max()):.3g}, "
              f"force error / (tol sum |F_c|) {float((ferr / (tol * tot[:, None] + 1e-300)).max()):.3g}")
        assert np.all(ferr <= lim)
        assert np.all(terr <= lim * lever)
        assert abs(float(e.item()) - e_ref) <= tol * max(e_ref, 1e-30)


def test_gradients_match_oracle_c3_subset(gctx, orc):
    s = scene_c3(n_pairs=1024).subset(np.arange(0, 1024, 128))
    prob = _problem(gctx, s, "fp64")
    c, _ = prob.detect()
    gv, gp, jac = prob.grad(want_jac=True)
    ref = orc.detect(s)
    assert ref["d"].min() >= 1.7 * 0.02 * (1 - 1e-9)
    gv_ref, gp_ref, jac_ref = orc.grad(s, ref)
    gp = gp.cpu().numpy()
    assert np.abs(gp - gp_ref).max() <= 1e-9 * np.abs(gp_ref).max()
    gv = gv.cpu().numpy()
    assert np.abs(gv - gv_ref).max() <= 1e-5 * np.abs(gv_ref).max()
    jac = jac.cpu().numpy()
    assert np.abs(jac - jac_ref).max() <= 1e-9 * np.abs(jac_ref).max()


def _contact_energy(orc, scene, abt, ks_eps, eps, poses=None):
    """FP64 energy sum_c K sqrt(mu) eps (1 - d_c/2eps)^2 over the listed
    triangle pairs, each distance from the oracle (tri_pairs).  Near a
    configuration whose contact set it lists it equals the oracle's total
    energy up to O(h^2): a pair entering or leaving the set contributes
    e(d) = O((2 eps - d)^2), and e'(2 eps) = 0."""
    d, _, _, _ = orc.tri_pairs(scene, abt, poses=poses)
    return float((ks_eps * (1.0 - d / (2 * eps)) ** 2).sum())


def test_gradient_finite_differences(gctx, orc):
    """The adjoint's dE/dpose and dE/dverts on the differentiation workload's
    64-pair subset (ids = 0 mod 16) against FP64 central differences
    (h = 1e-6) of the oracle's energy: every pose twist of every particle,
    and the three coordinates of six vertices per pair (the corners of the
    first contact's two triangles).  The energy is summed over the oracle's
    contact triangle pairs, one particle pair at a time (the pairs share no
    particle): a pair that crosses 2 eps under a step of h changes the
    energy by O(h^2) only, since e'(2 eps) = 0."""
    import dataclasses
    from tests import oracle_filtered
    from tests.test_oracle_forces_grad import _apply_twist
    s = scene_c3(n_pairs=1024).subset(np.arange(0, 1024, 16))
    assert len(np.unique(s.pairs)) == 2 * s.n_pairs
    prob = _problem(gctx, s, "fp64")
    prob.detect()
    gv, gp, _ = prob.grad()
    gp, gv = gp.cpu().numpy(), gv.cpu().numpy().astype(np.float64)
    ref = oracle_filtered.contacts(orc, s)
    assert np.all(ref["d"] <= 2 * s.eps[ref["pair"]] * (1 - 1e-3))
    mu = 1 / (1 / s.mass[s.pairs[:, 0]] + 1 / s.mass[s.pairs[:, 1]])
    h = 1e-6
    worst_p = worst_v = 0.0
    for p in range(s.n_pairs):
        sel = ref["pair"] == p
        assert sel.sum() > 0
        A, B = (int(x) for x in s.pairs[p])
        sp = s.subset([p])  # particles A, B renumbered 0, 1
        sp = dataclasses.replace(sp, verts=sp.verts.astype(np.float64))
        abt = np.stack([np.zeros(sel.sum(), int), ref["ta"][sel], np.ones(sel.sum(), int),
                        ref["tb"][sel]], 1)
        eps = s.eps[p]
        ks_eps = 1000 * np.sqrt(mu[p]) * eps
        energy = lambda sc, poses=None: _contact_energy(orc, sc, abt, ks_eps, eps, poses)  # noqa: E731
        for li, gi in ((0, A), (1, B)):
            for k in range(6):
                pp, pm = sp.poses.copy(), sp.poses.copy()
                pp[li] = _apply_twist(sp.poses[li], k, h)
                pm[li] = _apply_twist(sp.poses[li], k, -h)
                fd = (energy(sp, pp) - energy(sp, pm)) / (2 * h)
                worst_p = max(worst_p, abs(fd - gp[gi, k]) / np.abs(gp).max())
        # vertex gradient: corners of the first contact's triangles (body frame)
        c = np.flatnonzero(sel)[0]
        for li, gi, t in ((0, A, ref["ta"][c]), (1, B, ref["tb"][c])):
            for lv in sp.tris[sp.tri_off[li] + t]:
                for k in range(3):
                    vp, vm = sp.verts.copy(), sp.verts.copy()
                    vp[sp.vert_off[li] + lv, k] += h
                    vm[sp.vert_off[li] + lv, k] -= h
                    fd = (energy(dataclasses.replace(sp, verts=vp))
                          - energy(dataclasses.replace(sp, verts=vm))) / (2 * h)
                    worst_v = max(worst_v, abs(fd - gv[s.vert_off[gi] + lv, k]) / np.abs(gv).max())
    print(f"largest error / largest gradient: pose {worst_p:.3g}, vertex {worst_v:.3g}")
    assert worst_p <= 1e-6
    # the vertex gradient is a float32 output
    assert worst_v <= 1e-5


def test_autograd_function(gctx, orc):
    import torch
    import paper_2105_12415_gb300 as m
    s = scene_c3(n_pairs=1024).subset([5, 9])
    prob = _problem(gctx, s, "fp64")
    E, verts, twist = m.contact_energy(prob)
    (2.0 * E).backward()
    ref = orc.detect(s)
    gv_ref, gp_ref, _ = orc.grad(s, ref)
    assert abs(float(E.detach()) - orc.forces(s, ref)[1]) <= 1e-9 * float(E.detach())
    assert np.abs(twist.grad.cpu().numpy() - 2 * gp_ref).max() <= 1e-9 * np.abs(gp_ref).max() * 2
    assert np.abs(verts.grad.cpu().numpy() - 2 * gv_ref).max() <= 1e-5 * np.abs(gv_ref).max() * 2


def test_autograd_energy_is_a_function_of_its_inputs(gctx, orc):
    """ContactEnergy at moved poses and moved vertices equals the oracle's
    energy there, and torch.autograd.gradcheck passes on a 2-pair FP64 case:
    in the twist (FP64, step 1e-6) and in the vertices (steps of 2^-16,
    exact in the float32 meshes the library stores)."""
    import dataclasses
    import torch
    import paper_2105_12415_gb300 as m
    from tests.test_oracle_forces_grad import _apply_twist
    s = scene_c3(n_pairs=1024).subset([5, 9])
    prob = _problem(gctx, s, "fp64")
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(3)
    tw = np.zeros((s.n_particles, 6))
    tw[:, :3] = rng.normal(scale=2e-3, size=(s.n_particles, 3))
    tw[:, 3:] = rng.normal(scale=2e-3, size=(s.n_particles, 3))
    verts = torch.as_tensor(s.verts, device=dev).double()
    verts[:20] += 2.0 ** -10
    E = m.ContactEnergy.apply(verts, torch.as_tensor(tw, device=dev), prob)
    # the oracle at the same geometry: poses moved by the twist (translation,
    # then the rotation vector's turn on the left), vertices moved
    moved = s.poses.copy()
    for i in range(s.n_particles):
        p = moved[i].copy()
        p[:3] += tw[i, :3]
        th = np.linalg.norm(tw[i, 3:])
        if th > 0:
            ax = tw[i, 3:] / th
            dq = np.r_[np.cos(th / 2), np.sin(th / 2) * ax]
            w1, v1, w2, v2 = dq[0], dq[1:], p[3], p[4:].copy()
            p[3] = w1 * w2 - v1 @ v2
            p[4:] = w1 * v2 + w2 * v1 + np.cross(v1, v2)
        moved[i] = p
    s2 = dataclasses.replace(s, verts=verts.float().cpu().numpy(), poses=moved)
    e_ref = orc.forces(s2, orc.detect(s2))[1]
    assert abs(float(E) - e_ref) <= 1e-9 * e_ref
    # gradcheck in the twist
    twist = torch.as_tensor(tw, device=dev).requires_grad_(True)
    v0 = torch.as_tensor(s.verts, device=dev).double()
    # the adjoint sums contacts with atomics, so two backward passes differ in
    # the last bits (nondet_tol)
    assert torch.autograd.gradcheck(lambda t: m.ContactEnergy.apply(v0, t, prob), (twist,),
                                    eps=1e-6, atol=1e-6, rtol=1e-4, nondet_tol=1e-9)
    # gradcheck in the vertices of the first three contacts' triangles of A
    ref = orc.detect(s)
    vsel = []
    for c in range(3):
        A = s.pairs[ref["pair"][c], 0]
        vsel += list(s.vert_off[A] + s.tris[s.tri_off[A] + ref["ta"][c]])
    vsel = np.unique(np.asarray(vsel, np.int64))
    base = torch.as_tensor(s.verts, device=dev).double()
    sub = base[torch.as_tensor(vsel, device=dev)].clone().requires_grad_(True)
    idx = torch.as_tensor(vsel, device=dev)

    def energy_of(vs):
        full = base.index_put((idx,), vs)
        return m.ContactEnergy.apply(full, torch.zeros_like(twist), prob)
    # the vertex gradient is a float32 output (entries of order 1e3 here):
    # an entry whose exact value is 0 carries float rounding of about 1e-7 of
    # the largest (atol), and float32 atomics make two passes differ in the
    # last bits (nondet_tol)
    assert torch.autograd.gradcheck(energy_of, (sub,), eps=2.0 ** -16, atol=5e-3, rtol=1e-3,
                                    nondet_tol=5e-3)
