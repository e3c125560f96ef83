"""Multiresolution detection (Algorithm 5) on the GPU through the C ABI against
the FP64 brute-force oracle (Lemma 1: same contact set), in both precision
forms, plus the plain FP64 GPU form, the batched workload at full size on
sampled pairs, and the edge cases."""
import numpy as np
import pytest

from gen import scene_c1, scene_c2, scene_c3, scene_pairs, scene_particle_on_plane, scene_tiny
from tests.gpu_common import compare_contacts, gpu_scene_tensors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    import paper_2105_12415_gb300 as m
    m.build()
    return m.Context(0)


def _run(gctx, scene, precision, hier=None):
    import torch
    import paper_2105_12415_gb300 as m
    dev = torch.device("cuda:0")
    if hier is None:
        hier = m.Hierarchy.from_scene(gctx, scene)
    t = gpu_scene_tensors(scene, dev)
    c, stats = m.detect(gctx, hier, t["pairs"], t["eps"], t["poses"], precision)
    return c.to_numpy(), stats.cpu().numpy(), hier


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_c1_one_pair_full_parity(gctx, orc, precision):
    s = scene_c1()
    ref = orc.detect(s)
    got, stats, _ = _run(gctx, s, precision)
    assert len(ref["d"]) > 100
    compare_contacts(got, ref, s, precision)
    assert stats[20] == len(got["d"])
    # the hierarchy pruned: far fewer fine tests than 1280^2
    assert 0 < stats[17] < 0.1 * 1280 * 1280
    # the oriented boxes pruned child pairs the spheres let through
    assert stats[30] > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiny_and_mixed_scenes(gctx, orc, precision):
    for s in (scene_tiny(n_pairs=24, levels=(0, 1, 2)),
              scene_pairs([1, 2, 3, 4], [4, 3, 1, 1], [0.1, 1.0, 0.5, 0.2], [1.0, 0.13, 0.5, 0.9],
                          [0.001, 0.0013, 0.005, 0.002], [-0.0005, 0.002, 0.0, 0.006], 21, "mixed")):
        ref = orc.detect(s)
        got, _, _ = _run(gctx, s, precision)
        compare_contacts(got, ref, s, precision)


def _scaled(scene, k):
    """The scene with geometry, positions and eps multiplied by k."""
    import dataclasses
    poses = scene.poses.copy()
    poses[:, :3] *= k
    return dataclasses.replace(scene, verts=(scene.verts * np.float32(k)).astype(np.float32),
                               poses=poses, eps=scene.eps * k, radius=scene.radius * k,
                               com=scene.com * k, name=f"{scene.name}-x{k:g}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [1e-5, 1e5])
def test_scaled_scenes(gctx, orc, precision, k):
    """Scaling geometry, positions and eps by k scales every distance: the
    contact set matches the oracle's at any scale (the FP32 form's
    double-float finishing scales each candidate by a power of two)."""
    s = _scaled(scene_tiny(n_pairs=16, levels=(1, 2)), k)
    ref = orc.detect(s)
    assert len(ref["d"]) > 0
    got, _, _ = _run(gctx, s, precision)
    compare_contacts(got, ref, s, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_particle_on_plane(gctx, orc, precision):
    """Particle-on-plane (Sec. 6): particles of 1280 to 20480 triangles over
    a one-triangle plane (the |T| : 1 extreme), penetrating, touching and
    apart; contact set and distances as the oracle's."""
    s = scene_particle_on_plane()
    ref = orc.detect(s)
    got, stats, _ = _run(gctx, s, precision)
    compare_contacts(got, ref, s, precision)
    assert np.bincount(got["pair"], minlength=s.n_pairs)[3] == 0


def test_plain_fp64_form_and_lemma1(gctx, orc):
    """The plain form (all pairs, FP64) equals the oracle, and the hierarchy's
    result equals the plain form's (Lemma 1)."""
    import torch
    import paper_2105_12415_gb300 as m
    s = scene_pairs([3, 2], [2, 3], [1.0, 0.6], [0.7, 1.0], [0.01, 0.008], [-0.004, 0.001], 31, "lemma1")
    ref = orc.detect(s)
    got, _, hier = _run(gctx, s, "fp64")
    t = gpu_scene_tensors(s, torch.device("cuda:0"))
    plain = m.detect_plain_fp64(gctx, hier, t["pairs"], t["eps"], t["poses"]).to_numpy()
    compare_contacts(plain, ref, s, "fp64")
    compare_contacts(got, plain, s, "fp64")


def test_swapped_pairs_and_self_pair(gctx, orc):
    s = scene_tiny(n_pairs=6, levels=(1, 2), seed=44)
    sw = scene_tiny(n_pairs=6, levels=(1, 2), seed=44)
    sw.pairs = s.pairs[:, ::-1].copy()
    a, _, _ = _run(gctx, s, "fp64")
    b, _, _ = _run(gctx, sw, "fp64")
    ka = sorted(zip(a["pair"].tolist(), a["ta"].tolist(), a["tb"].tolist()))
    kb = sorted(zip(b["pair"].tolist(), b["tb"].tolist(), b["ta"].tolist()))
    assert ka == kb
    # a particle against itself: every triangle touches its neighbours
    s1 = scene_tiny(n_pairs=1, levels=(1,), seed=45)
    s1.pairs = np.array([[0, 0]], np.int32)
    ref = orc.detect(s1)
    got, _, _ = _run(gctx, s1, "fp64")
    compare_contacts(got, ref, s1, "fp64", check_points=False)


def test_empty_and_far_apart(gctx):
    import torch
    import paper_2105_12415_gb300 as m
    s = scene_pairs([2], [2], [1.0], [1.0], [0.01], [5.0], 3, "far")
    got, stats, hier = _run(gctx, s, "fp32")
    assert len(got["d"]) == 0 and stats[17] == 0
    dev = torch.device("cuda:0")
    t = gpu_scene_tensors(s, dev)
    c, st = m.detect(gctx, hier, t["pairs"][:0], t["eps"][:0], t["poses"], "fp32")
    assert c.n() == 0


def test_invalid_inputs_are_latched(gctx):
    import torch
    import paper_2105_12415_gb300 as m
    s = scene_tiny(n_pairs=2, levels=(1,))
    hier = m.Hierarchy.from_scene(gctx, s)
    dev = torch.device("cuda:0")
    t = gpu_scene_tensors(s, dev)
    bad_pose = t["poses"].clone()
    bad_pose[0, 0] = float("nan")
    with pytest.raises(m.MrdemError) as e:
        m.detect(gctx, hier, t["pairs"], t["eps"], bad_pose)
    assert e.value.status == m._lib.MRDEM_ERR_NONFINITE
    bad_eps = t["eps"].clone()
    bad_eps[1] = 0.0
    with pytest.raises(m.MrdemError):
        m.detect(gctx, hier, t["pairs"], bad_eps, t["poses"])
    bad_pairs = t["pairs"].clone()
    bad_pairs[0, 1] = 99
    with pytest.raises(m.MrdemError):
        m.detect(gctx, hier, bad_pairs, t["eps"], t["poses"])
    # the context stays usable
    c, _ = m.detect(gctx, hier, t["pairs"], t["eps"], t["poses"])
    assert c.n() >= 0


def test_capacity_overflow_is_reported_and_recovered(orc):
    """Tiny work lists: the first call reports CAPACITY with the required
    sizes; the binding grows the lists and repeats; the result is exact."""
    import ctypes as C
    import torch
    import paper_2105_12415_gb300 as m
    ctx = m.Context(0, cap_level=8, cap_tiles=8, cap_candidates=8, cap_sweep=8)
    s = scene_c1()
    hier = m.Hierarchy.from_scene(ctx, s)
    dev = torch.device("cuda:0")
    t = gpu_scene_tensors(s, dev)
    contacts = m.Contacts(4, dev)
    cs = contacts.struct()
    lib = m.load()
    st = lib.mrdem_detect(ctx.handle, hier.handle, 1, t["pairs"].data_ptr(), t["eps"].data_ptr(),
                          t["poses"].data_ptr(), 1, C.byref(cs), None, None)
    assert st == 0
    req = np.zeros(5, np.int64)
    assert lib.mrdem_check(ctx.handle, None, req.ctypes.data) == m._lib.MRDEM_ERR_CAPACITY
    assert req[0] > 8 or req[1] > 8 or req[2] > 8 or req[4] > 8
    got, _ = m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], "fp64", contacts=contacts)
    compare_contacts(got.to_numpy(), orc.detect(s), s, "fp64")


@pytest.fixture(scope="module")
def c2_oracle_subset(orc):
    """The oracle's contacts of the batched workload's pairs with id = 0 mod 8
    (512 pairs), through the sphere-filtered brute force."""
    from tests import oracle_filtered
    s = scene_c2()
    ids = np.arange(0, s.n_pairs, 8)
    return s, ids, oracle_filtered.contacts(orc, s, ids)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_full_size_sampled(gctx, orc, c2_oracle_subset, precision):
    """The 4096-pair batched workload in one launch sequence (as timed by the
    benchmark): the pairs with id = 0 mod 8 (512 pairs) checked against the
    oracle contact by contact, the deepest interpenetration too, and
    properties that hold at any size checked on all pairs."""
    import torch
    import paper_2105_12415_gb300 as m
    from tests import oracle_filtered
    s, ids, ref_sub = c2_oracle_subset
    hier = m.Hierarchy.from_scene(gctx, s)
    dev = torch.device("cuda:0")
    t = gpu_scene_tensors(s, dev)
    c, stats = m.detect(gctx, hier, t["pairs"], t["eps"], t["poses"], precision)
    got = c.to_numpy()
    st = stats.cpu().numpy()
    n = len(got["d"])
    assert n == st[20] and n > 0
    # properties on every contact
    tau = 2 * s.eps[got["pair"]]
    assert np.all(got["d"] <= tau * (1 + 1e-12))
    assert np.all(np.abs(np.linalg.norm(got["pa"] - got["pb"], axis=1) - got["d"]) <= 1e-9 * np.maximum(got["d"], 1e-3))
    keys = got["pair"].astype(np.int64) * (1 << 40) + got["ta"].astype(np.int64) * (1 << 20) + got["tb"]
    assert len(np.unique(keys)) == n
    ntri = np.diff(s.tri_off)
    assert np.all(got["ta"] < ntri[s.pairs[got["pair"], 0]]) and np.all(got["tb"] < ntri[s.pairs[got["pair"], 1]])
    # the 512-pair subset, contact by contact
    sel = np.isin(got["pair"], ids)
    g2 = {k: v[sel] for k, v in got.items()}
    assert len(ref_sub["d"]) > 1000
    compare_contacts(g2, ref_sub, s, precision)
    # the pair with the most contacts (deepest interpenetration) as well
    deep = int(np.argmax(np.bincount(got["pair"], minlength=s.n_pairs)))
    ref_d = oracle_filtered.contacts(orc, s, [deep])
    g3 = {k: v[got["pair"] == deep] for k, v in got.items()}
    compare_contacts(g3, ref_d, s, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_keeps_results(orc, precision):
    """The launch-shape autotuner picks allowed values for the batch's size
    class, and detection with the chosen shapes returns the oracle's contact
    set as before; set_params clears the choice."""
    import torch
    import paper_2105_12415_gb300 as m
    from tests import oracle_filtered
    s = scene_c3(n_pairs=1024).subset(np.arange(0, 1024, 32))
    ctx = m.Context(0)
    hier = m.Hierarchy.from_scene(ctx, s)
    t = gpu_scene_tensors(s, torch.device("cuda:0"))
    ref = oracle_filtered.contacts(orc, s)
    before, _ = m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], precision)
    compare_contacts(before.to_numpy(), ref, s, precision)
    r = m.autotune(ctx, hier, t["pairs"], t["eps"], t["poses"], precision, reps=2)
    allowed = {"level_warps": {2, 4, 8}, "expand_items": {8, 16, 32}, "node_threads": {128, 256},
               "tile_warps": {2, 4, 8}, "sweep_warps": {2, 4, 8}, "exact_threads": {64, 128, 256},
               "level_kernel": {0, 1, 2}}
    for k, v in r["chosen"].items():
        assert v in allowed[k], (k, v)
    assert r["ms_default"] > 0 and r["ms_tuned"] > 0
    after, _ = m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], precision)
    compare_contacts(after.to_numpy(), ref, s, precision)
    ctx.set_params(n_iter=4)
    again, _ = m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], precision)
    compare_contacts(again.to_numpy(), ref, s, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cooperative_levels_equal_per_level_launches(c2_oracle_subset, precision):
    """All surrogate levels in one cooperative launch (level_kernel 1), and
    one launch per level with the sweep in the expanding warp (level_kernel
    2), test the same pairs as the two launches per level: the same contact
    set (the same distances and points, bit for bit) and the same counters,
    eagerly and replayed from a CUDA graph."""
    import torch
    import paper_2105_12415_gb300 as m
    s, _, _ = c2_oracle_subset
    ctx = m.Context(0)
    hier = m.Hierarchy.from_scene(ctx, s)
    t = gpu_scene_tensors(s, torch.device("cuda:0"))
    res = {}
    for lk in (0, 1, 2):
        ctx.set_params(level_kernel=lk)
        c, st = m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], precision)
        res[lk] = (c.to_numpy(), st.cpu().numpy())
    for lk in (1, 2):
        for k in ("pair", "ta", "tb", "d", "pa", "pb"):
            assert np.array_equal(res[0][0][k], res[lk][0][k]), (lk, k)
        assert np.array_equal(res[0][1], res[lk][1]), lk
    # captured into a CUDA graph and replayed
    for lk in (1, 2):
        ctx.set_params(level_kernel=lk)
        c, st = m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], precision)   # sizes the lists
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=side):
            m.detect(ctx, hier, t["pairs"], t["eps"], t["poses"], precision, contacts=c, stats=st,
                     check=False)
        torch.cuda.current_stream().wait_stream(side)
        c.count.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert m.load().mrdem_check(ctx.handle, None, None) == 0
        got = c.to_numpy()
        for k in ("pair", "ta", "tb", "d"):
            assert np.array_equal(got[k], res[0][0][k]), (lk, k)
