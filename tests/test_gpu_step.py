"""ContactProblem.step: detection, forces and energy, and the adjoint in one
call with one status check, optionally replayed from a CUDA graph.  Its
results equal the separate checked calls, also after list overflows that
make it grow its lists and run again."""
import numpy as np
import pytest

from gen import scene_c3, scene_tiny

pytestmark = pytest.mark.gpu


def _problem(scene, **ctx_kw):
    import torch
    import paper_2105_12415_gb300 as m
    m.build()
    ctx = m.Context(0, **ctx_kw)
    hier = m.Hierarchy.from_scene(ctx, scene)
    return m.ContactProblem.from_scene(ctx, hier, scene, torch.device("cuda:0"), precision="fp32")


def _separate(prob):
    c, _ = prob.detect()
    ft, e = prob.forces()
    gv, gp, jac = prob.grad(want_jac=True)
    return (c.to_numpy(), ft.cpu().numpy(), float(e.item()), gv.cpu().numpy(), gp.cpu().numpy(),
            jac.cpu().numpy())


def _stepped(prob, graph):
    c, ft, e, gv, gp, jac, _ = prob.step(want_jac=True, graph=graph)
    return (c.to_numpy(), ft.cpu().numpy(), float(e.item()), gv.cpu().numpy(), gp.cpu().numpy(),
            jac.cpu().numpy())


def _same(a, b):
    ca, cb = a[0], b[0]
    assert len(ca["d"]) == len(cb["d"]) > 0
    for k in ("pair", "ta", "tb"):
        assert np.array_equal(ca[k], cb[k])
    assert np.allclose(ca["d"], cb["d"], rtol=0, atol=1e-15)
    # per-particle sums: the order of the atomic additions may differ, so
    # double outputs agree to 1e-9 and the float vertex gradient to 1e-5
    for x, y in zip(a[1:], b[1:]):
        x, y = np.asarray(x), np.asarray(y)
        tol = 1e-5 if x.dtype == np.float32 else 1e-9
        assert np.allclose(x, y, rtol=tol, atol=tol * max(1.0, float(np.abs(y).max()))), (x, y)


@pytest.mark.parametrize("graph", [False, True])
def test_step_equals_separate_calls(graph):
    s = scene_c3(n_pairs=1024).subset(np.arange(0, 1024, 64))
    prob = _problem(s)
    ref = _separate(prob)
    for _ in range(3):   # replays of the same graph
        _same(_stepped(prob, graph), ref)


def test_step_grows_lists_and_recaptures():
    import torch
    s = scene_tiny(n_pairs=12, levels=(1, 2))
    prob = _problem(s)
    ref = _separate(prob)
    # a fresh problem with tiny lists: the first step overflows and grows them
    small = _problem(s, cap_level=16, cap_tiles=16, cap_candidates=16, cap_sweep=16)
    small.contacts = None
    got = _stepped(small, True)
    _same(got, ref)
    # new poses written in place are picked up by the replayed graph
    moved = s.poses.copy()
    moved[:, :3] += np.array([0.25, -0.5, 0.125])
    small.poses.copy_(torch.as_tensor(moved, device="cuda:0"))
    prob.poses.copy_(torch.as_tensor(moved, device="cuda:0"))
    _same(_stepped(small, True), _separate(prob))


def test_contacts_grouped_by_pair():
    """Detection writes its contacts grouped by pair, pairs in increasing order."""
    s = scene_c3(n_pairs=1024).subset(np.arange(0, 1024, 32))
    prob = _problem(s)
    c, _ = prob.detect()
    pairs = c.to_numpy(sort=False)["pair"]
    assert len(pairs) > 0
    assert np.all(np.diff(pairs) >= 0)


@pytest.mark.parametrize("graph", [False, True])
def test_step_copies_results_to_pinned_host_buffers(graph):
    """step(host_out=...) leaves the results of the run that succeeded in the
    caller's pinned host tensors, also when the first run overflowed its
    lists and the step grew them and ran again."""
    import torch
    s = scene_tiny(n_pairs=12, levels=(1, 2))
    small = _problem(s, cap_level=16, cap_tiles=16, cap_candidates=16, cap_sweep=16)
    n = s.n_particles
    host = {"ft": torch.empty((n, 6), dtype=torch.float64).pin_memory(),
            "gp": torch.empty((n, 6), dtype=torch.float64).pin_memory(),
            "energy": torch.empty(1, dtype=torch.float64).pin_memory(),
            "count": torch.empty(1, dtype=torch.int64).pin_memory()}
    for _ in range(2):
        c, ft, e, _, gp, _, _ = small.step(graph=graph, host_out=host)
        assert np.array_equal(host["ft"].numpy(), ft.cpu().numpy())
        assert np.array_equal(host["gp"].numpy(), gp.cpu().numpy())
        assert host["energy"].item() == e.item() and host["count"].item() == c.count.item() > 0


def test_step_copies_host_inputs_in_its_graph():
    """step(host_in=...) copies the inputs from pinned host tensors at every
    step, replayed graph included: new poses written into the host tensor
    are what the next step detects at."""
    import torch
    s = scene_tiny(n_pairs=12, levels=(1, 2))
    prob = _problem(s)
    ref = _problem(s)
    h_in = {"poses": torch.as_tensor(s.poses, dtype=torch.float64).pin_memory(),
            "eps": torch.as_tensor(s.eps, dtype=torch.float64).pin_memory()}
    for shift in (0.0, 0.25, -0.125):
        moved = s.poses.copy()
        moved[:, :3] += shift
        h_in["poses"].copy_(torch.as_tensor(moved))
        got = prob.step(want_jac=True, graph=True, host_in=h_in)
        ref.poses.copy_(torch.as_tensor(moved, device="cuda:0"))
        _same(tuple([got[0].to_numpy()] + [x.cpu().numpy() if hasattr(x, "cpu") else x
                                          for x in (got[1], float(got[2].item()), got[3],
                                                    got[4], got[5])]),
              _separate(ref))
