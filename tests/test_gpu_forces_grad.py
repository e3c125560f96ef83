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
    """Per particle |F - F_ref| <= tol * sum_c |F_c| + sum_c |F_c| min(2, 1e3 S 2^-44 / d_c):
    the second term is the conditioning of the direction u = (pa - pb)/d for
    nearly touching triangles (the oracle's coordinates carry 2^-44 S of
    rounding), which also covers exact touching (d = 0 on one side, 1e-17 on
    the other: the direction is then a convention)."""
    from tests.gpu_common import world_scale
    for s in (scene_c1(), scene_pairs([2, 3, 1], [3, 1, 2], [1.0, 0.3, 0.5], [0.4, 1.0, 0.5],
                                      [0.004, 0.003, 0.005], [-0.01, 0.0, 0.002], 13, "forces")):
        prob = _problem(gctx, s, precision)
        prob.detect()
        ft, e = prob.forces()
        ref = orc.detect(s)
        ft_ref, e_ref = orc.forces(s, ref)
        ft = ft.cpu().numpy()
        mu = 1 / (1 / s.mass[s.pairs[:, 0]] + 1 / s.mass[s.pairs[:, 1]])
        mag = 1000 * np.sqrt(mu[ref["pair"]]) * (1 - ref["d"] / (2 * s.eps[ref["pair"]]))
        floor = np.ldexp(world_scale(s), -44)[ref["pair"]]
        cond = mag * np.minimum(2.0, 1e3 * floor / np.maximum(ref["d"], 1e-300))
        band = mag * (np.abs(ref["d"] - 2 * s.eps[ref["pair"]]) <= 1e-6 * s.eps[ref["pair"]])
        tot = np.zeros(s.n_particles)
        extra = np.zeros(s.n_particles)
        for col in (0, 1):
            np.add.at(tot, s.pairs[ref["pair"], col], mag)
            np.add.at(extra, s.pairs[ref["pair"], col], cond + band)
        lim = (tol * tot + extra)[:, None]
        assert np.all(np.abs(ft[:, :3] - ft_ref[:, :3]) <= lim)
        lever = 2 * (s.radius.max() + np.abs(s.poses[:, :3]).max())
        assert np.all(np.abs(ft[:, 3:] - ft_ref[:, 3:]) <= lim * lever)
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


def test_gradient_finite_differences(gctx, orc):
    """dE/dpose from the kernel against central differences (h = 1e-6) of the
    oracle's FP64 energy."""
    from tests.test_oracle_forces_grad import _apply_twist
    s = scene_c3(n_pairs=1024).subset([3, 700])
    prob = _problem(gctx, s, "fp64")
    prob.detect()
    _, gp, _ = prob.grad()
    gp = gp.cpu().numpy()
    h = 1e-6
    for i in range(s.n_particles):
        for k in range(6):
            pp, pm = s.poses.copy(), s.poses.copy()
            pp[i] = _apply_twist(s.poses[i], k, h)
            pm[i] = _apply_twist(s.poses[i], k, -h)
            fd = (orc.energy(s, poses=pp) - orc.energy(s, poses=pm)) / (2 * h)
            assert abs(fd - gp[i, k]) <= 1e-5 * np.abs(gp).max(), (i, k, fd, gp[i, k])


def test_autograd_function(gctx, orc):
    import torch
    import paper_2105_12415_gb300 as m
    s = scene_c3(n_pairs=1024).subset([5, 9])
    prob = _problem(gctx, s, "fp64")
    verts = torch.as_tensor(s.verts, device="cuda:0").requires_grad_(True)
    twist = torch.zeros((s.n_particles, 6), dtype=torch.float64, device="cuda:0", requires_grad=True)
    E = m.ContactEnergy.apply(verts, twist, prob)
    (2.0 * E).backward()
    ref = orc.detect(s)
    gv_ref, gp_ref, _ = orc.grad(s, ref)
    assert abs(float(E) - orc.forces(s, ref)[1]) <= 1e-9 * float(E)
    assert np.abs(twist.grad.cpu().numpy() - 2 * gp_ref).max() <= 1e-9 * np.abs(gp_ref).max() * 2
    assert np.abs(verts.grad.cpu().numpy() - 2 * gv_ref).max() <= 1e-5 * np.abs(gv_ref).max() * 2
