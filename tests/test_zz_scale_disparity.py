"""Size disparity on the GPU (the scale workload): a big particle of 81 920
triangles and radius 20 against a small one of 1 280 triangles and radius 1
(the 20:1 setting of the many-particle scale study, Sec. 6), detection in
both precision forms against the FP64 brute-force oracle over all
104 857 600 triangle pairs of each pair (Lemma 1: the same contact set).
The big particle's tree is two levels deeper than the small one's, so the
level loop runs on while the small side stays at its leaves."""
import numpy as np
import pytest

from gen import scene_disparity
from tests.gpu_common import compare_contacts, gpu_scene_tensors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disparity(orc):
    s = scene_disparity(4).subset(np.array([1, 2]))
    ref = orc.detect(s)
    return s, ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_disparity_20_to_1_parity(orc, disparity, precision):
    import torch
    import paper_2105_12415_gb300 as m
    m.build()
    ctx = m.Context(0)
    s, ref = disparity
    assert len(ref["d"]) > 0
    hier = m.Hierarchy.from_scene(ctx, s)
    info = hier.info()
    assert info["n_particles"] == 4
    t = gpu_scene_tensors(s, torch.device("cuda:0"))
    c, stats = m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], precision)
    got = c.to_numpy()
    compare_contacts(got, ref, s, precision)
    st = stats.cpu().numpy()
    assert st[20] == len(got["d"])
