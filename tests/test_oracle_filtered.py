"""The sphere-filtered contact set (tests/oracle_filtered.py) equals the
oracle's full brute force, bit for bit, on the one-pair workload and on
batched-workload pairs small enough for the brute force."""
import numpy as np

from gen import scene_c1, scene_c2, scene_tiny
from tests import oracle_filtered


def _same(a, b):
    for k in ("pair", "ta", "tb", "feature"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("d", "pa", "pb"):
        assert np.array_equal(a[k], b[k]), k


def test_filtered_equals_brute_force_c1(orc):
    s = scene_c1()
    ref = orc.detect(s)
    assert len(ref["d"]) > 100
    _same(oracle_filtered.contacts(orc, s), ref)


def test_filtered_equals_brute_force_batched_pairs(orc):
    s = scene_c2()
    ntri = np.diff(s.tri_off)
    work = ntri[s.pairs[:, 0]] * ntri[s.pairs[:, 1]]
    ids = [k for k in range(0, s.n_pairs, 8) if work[k] <= 1280 * 5120][:12]
    sub = s.subset(ids)
    ref = orc.detect(sub)
    assert len(ref["d"]) > 0
    _same(oracle_filtered.contacts(orc, sub), ref)
    # pair indices of the full scene are kept
    got = oracle_filtered.contacts(orc, s, ids)
    assert np.array_equal(np.unique(got["pair"]), np.unique(np.asarray(ids)[ref["pair"]]))


def test_filtered_equals_brute_force_tiny(orc):
    s = scene_tiny(n_pairs=24, levels=(0, 1, 2))
    _same(oracle_filtered.contacts(orc, s), orc.detect(s))
