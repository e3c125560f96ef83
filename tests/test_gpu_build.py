"""Surrogate trees built on the GPU (mrdem_build_hierarchy_device; Sec. 4,
Algorithm 7, Appendix A): the tree shape is the host builder's (it follows
from the triangle counts), every surrogate is conservative by the oracle's
FP64 vertex distances, every node box holds its fine vertices, and
detection with the GPU-built trees returns the oracle's contact set
(Lemma 1 needs nothing else of the trees)."""
import collections

import numpy as np
import pytest

from gen import scene_c1, scene_disparity, scene_pairs, scene_particle_on_plane, scene_tiny
from tests.gpu_common import compare_contacts, gpu_scene_tensors
from tests.test_hierarchy_host import _box_contains_all, _check_conservative

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    import paper_2105_12415_gb300 as m
    m.build()
    return m.Context(0)


def _mixed():
    return scene_pairs([1, 2, 3, 4, 5], [5, 3, 1, 2, 4], [0.3, 1.0, 0.12, 0.5, 1.0],
                       [1.0, 0.5, 0.8, 0.2, 0.7], [0.003, 0.005, 0.0012, 0.002, 0.007],
                       [0.0, -0.002, 0.001, 0.0005, -0.001], 17, "build-mixed")


def _shape(ex):
    """Multiset of (level, children or -leaf size) over the nodes."""
    return collections.Counter(zip(ex["node_level"].tolist(), ex["node_child"][:, 1].tolist()))


@pytest.mark.parametrize("scene_fn", [scene_c1, _mixed, lambda: scene_disparity(1),
                                      scene_particle_on_plane])
def test_device_trees_shape_and_conservative(gctx, orc, scene_fn):
    import paper_2105_12415_gb300 as m
    s = scene_fn()
    dev = m.Hierarchy.from_scene_device(gctx, s)
    host = m.Hierarchy.from_scene(None, s)
    di, hi = dev.info(), host.info()
    for k in ("n_particles", "n_nodes", "n_tri", "n_tri_pad", "max_depth"):
        assert di[k] == hi[k], k
    ex = dev.export()
    assert _shape(ex) == _shape(host.export())
    # every fine triangle in exactly one slot, of its own particle
    sl = ex["slot_tri"] >= 0
    keys = ex["slot_particle"][sl].astype(np.int64) * (1 << 32) + ex["slot_tri"][sl]
    assert len(np.unique(keys)) == sl.sum() == di["n_tri"]
    _check_conservative(orc, s, ex)
    step = max(1, len(ex["node_delta"]) // 400)
    for node in range(0, len(ex["node_delta"]), step):
        ok, U, _, _ = _box_contains_all(ex, s, node, ex["node_box"][node])
        assert ok, node
        assert np.abs(U @ U.T - np.eye(3)).max() < 1e-6
    print(f"{s.name}: device build {dev.build_ms:.2f} ms")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_detection_with_device_trees(gctx, orc, precision):
    import torch
    import paper_2105_12415_gb300 as m
    for s in (scene_c1(), _mixed(), scene_tiny(n_pairs=16, levels=(0, 1, 2))):
        hier = m.Hierarchy.from_scene_device(gctx, s)
        t = gpu_scene_tensors(s, torch.device("cuda:0"))
        c, _ = m.detect(gctx, hier, t["pairs"], t["eps"], t["poses"], precision)
        compare_contacts(c.to_numpy(), orc.detect(s), s, precision)


def test_device_build_rejects_bad_input(gctx):
    import torch
    import paper_2105_12415_gb300 as m
    s = scene_tiny(n_pairs=2, levels=(1,))
    dev = torch.device("cuda:0")
    verts = torch.as_tensor(s.verts, device=dev)
    bad = torch.as_tensor(s.tris, device=dev).clone()
    bad[3, 1] = 10 ** 6  # a vertex index beyond its particle
    with pytest.raises(m.MrdemError):
        m.Hierarchy.build_device(gctx, s.vert_off, verts, s.tri_off, bad)
    flat = torch.as_tensor(s.tris, device=dev).clone()
    flat[0, 2] = flat[0, 1]  # a degenerate triangle
    with pytest.raises(m.MrdemError):
        m.Hierarchy.build_device(gctx, s.vert_off, verts, s.tri_off, flat)
    nan = verts.clone()
    nan[0, 0] = float("nan")
    with pytest.raises(m.MrdemError):
        m.Hierarchy.build_device(gctx, s.vert_off, nan, s.tri_off, torch.as_tensor(s.tris, device=dev))
    # the context stays usable
    h = m.Hierarchy.build_device(gctx, s.vert_off, verts, s.tri_off, torch.as_tensor(s.tris, device=dev))
    assert h.info()["n_particles"] == s.n_particles
