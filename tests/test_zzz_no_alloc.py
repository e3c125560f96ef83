"""The allocation-free detection entry point (mrdem_detect_noalloc).

Callers that own all device memory themselves (a fixed budget handed over at
start-up, or a real-time loop that must not call cudaMalloc after
initialisation) use this call instead of mrdem_detect: its work lists live in
a fixed array inside the library.  The test calls it through the C ABI twice
in a row and checks both results against mrdem_detect, with the tolerance of
the other GPU tests, and against the FP64 oracle directly, in both
precisions on the one-pair scene (the FP32 form finishes in its own kernel,
k_exact32).  It builds everything it needs, so it also passes alone in a
fresh process (its first call then does the one-time set-up).  The file is
named so that pytest collects it after every other test file.
"""
import ctypes as C

import numpy as np
import pytest

from gen import scene_c1, scene_tiny
from tests.gpu_common import compare_contacts, gpu_scene_tensors

pytestmark = pytest.mark.gpu


def _noalloc(m, hier, t, contacts, stats, precision):
    cs = contacts.struct()
    st = m.load().mrdem_detect_noalloc(hier.handle, t["pairs"].shape[0], t["pairs"].data_ptr(),
                                       t["eps"].data_ptr(), t["poses"].data_ptr(), precision,
                                       C.byref(cs), stats.data_ptr(), None)
    return st


@pytest.mark.parametrize("scene_fn,precision", [(scene_c1, 1), (scene_c1, 0),
                                                (lambda: scene_tiny(n_pairs=16, levels=(1, 2)), 0)])
def test_noalloc_matches_detect_twice(orc, scene_fn, precision):
    import torch
    import paper_2105_12415_gb300 as m
    m.build()
    dev = torch.device("cuda:0")
    s = scene_fn()
    ctx = m.Context(0)
    hier = m.Hierarchy.from_scene(ctx, s)
    t = gpu_scene_tensors(s, dev)
    pname = "fp64" if precision == 1 else "fp32"
    ref, _ = m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], pname)
    ref = ref.to_numpy()
    assert len(ref["d"]) > 0
    oref = orc.detect(s)
    for _ in range(2):  # the array keeps the previous call's contents
        contacts = m.Contacts(4 * len(ref["d"]) + 64, dev)
        stats = torch.full((m._lib.MRDEM_STAT_COUNT,), -1, dtype=torch.int64, device=dev)
        assert _noalloc(m, hier, t, contacts, stats, precision) == m._lib.MRDEM_OK
        torch.cuda.synchronize()
        st = stats.cpu().numpy()
        assert st[m._lib.MRDEM_STAT_NOALLOC_OVERFLOW] == 0
        assert st[m._lib.MRDEM_STAT_NOALLOC_INVALID] == 0
        got = contacts.to_numpy()
        assert len(got["d"]) == len(ref["d"]) == st[m._lib.MRDEM_STAT_CONTACTS]
        compare_contacts(got, ref, s, pname)
        compare_contacts(got, oref, s, pname)


def test_noalloc_rejects_too_many_pairs():
    import torch
    import paper_2105_12415_gb300 as m
    m.build()
    dev = torch.device("cuda:0")
    s = scene_tiny(n_pairs=2, levels=(1,))
    ctx = m.Context(0)
    hier = m.Hierarchy.from_scene(ctx, s)
    t = gpu_scene_tensors(s, dev)
    big = {k: v for k, v in t.items()}
    big["pairs"] = t["pairs"][np.zeros(1025, dtype=np.int64)].contiguous()
    big["eps"] = t["eps"][np.zeros(1025, dtype=np.int64)].contiguous()
    contacts = m.Contacts(16, dev)
    stats = torch.zeros(m._lib.MRDEM_STAT_COUNT, dtype=torch.int64, device=dev)
    assert _noalloc(m, hier, big, contacts, stats, 0) == m._lib.MRDEM_ERR_INVALID
