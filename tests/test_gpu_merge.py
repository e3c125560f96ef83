"""Redundant-contact merge (Sec. 2, the implementation note on the contact
set) on the GPU through the C ABI, against the FP64 oracle's merge on the same
input list: the partition (representatives, member counts, output order) must
be identical, since both sides take every link decision with the same FP64
operations, and the mean points equal up to summation order."""
import numpy as np
import pytest

from gen import icosphere, scene_c1, scene_regular_pair, scene_tiny
from tests.gpu_common import gpu_scene_tensors
from tests.test_oracle_contacts import _quat_from_matrix, _rotation_taking

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    import paper_2105_12415_gb300 as m
    m.build()
    return m.Context(0)


def _device_list(c, capacity=None):
    """A device contact list holding the numpy list c in its given order."""
    import torch
    import paper_2105_12415_gb300 as m
    n = len(c["pair"])
    out = m.Contacts(max(capacity or n, 1), "cuda:0")
    if n:
        out.pair[:n] = torch.as_tensor(np.asarray(c["pair"], np.int32))
        out.tri_a[:n] = torch.as_tensor(np.asarray(c["ta"], np.int32))
        out.tri_b[:n] = torch.as_tensor(np.asarray(c["tb"], np.int32))
        pa = np.asarray(c["pa"], np.float64).reshape(-1, 3)
        pb = np.asarray(c["pb"], np.float64).reshape(-1, 3)
        out.point_a[:n] = torch.as_tensor(pa)
        out.point_b[:n] = torch.as_tensor(pb)
        out.dist[:n] = torch.as_tensor(np.asarray(c["d"], np.float64))
    out.count.fill_(n)
    return out


def _merged(out, members):
    got = out.to_numpy(sort=False)
    got["members"] = members[:out.n()].cpu().numpy()
    return got


def _compare(got, ref):
    """Identical partition and order; points within the rounding of the
    member sums (sequential on the GPU, pairwise in numpy)."""
    for k in ("pair", "ta", "tb", "members"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    scale = 1.0 + np.maximum(np.abs(ref["pa"]).max(1), np.abs(ref["pb"]).max(1))
    tol = (ref["members"] + 2) * 2.0 ** -51 * scale
    assert (np.abs(got["pa"] - ref["pa"]).max(1) <= tol).all()
    assert (np.abs(got["pb"] - ref["pb"]).max(1) <= tol).all()
    assert (np.abs(got["d"] - ref["d"]) <= 4 * tol + 2.0 ** -52 * ref["d"]).all()


def _detected(gctx, scene, precision):
    import torch
    import paper_2105_12415_gb300 as m
    hier = m.Hierarchy.from_scene(gctx, scene)
    t = gpu_scene_tensors(scene, torch.device("cuda:0"))
    c, _ = m.detect(gctx, hier, t["pairs"], t["eps"], t["poses"], precision)
    return c, t, hier


@pytest.mark.parametrize("scene_fn,precision", [(scene_c1, "fp64"), (scene_c1, "fp32"),
                                                (lambda: scene_tiny(n_pairs=16, levels=(0, 1, 2)), "fp32")])
def test_merge_of_detected_contacts_matches_oracle(gctx, orc, scene_fn, precision):
    import paper_2105_12415_gb300 as m
    s = scene_fn()
    c, t, _ = _detected(gctx, s, precision)
    host = c.to_numpy(sort=False)
    ref = orc.merge_contacts(host, s.eps)
    out, members = m.merge_contacts(gctx, t["eps"], c)
    got = _merged(out, members)
    assert members[:out.n()].sum().item() == len(host["d"])
    _compare(got, ref)
    assert len(ref["d"]) < len(host["d"])  # these meshes do produce redundant contacts


def _synthetic(rng, sizes, eps, offset=40.0):
    """Clustered contact points, pair p with sizes[p] contacts spread on the
    scale of eps[p], keys unique within a pair, shuffled over the whole
    list."""
    rows = []
    for p, n in enumerate(sizes):
        if n == 0:
            continue
        k = max(1, n // 6)
        centres = rng.uniform(-1, 1, (k, 3)) * (4 * eps[p]) * np.sqrt(k) + offset
        x = centres[rng.integers(0, k, n)] + rng.normal(scale=0.6 * eps[p], size=(n, 3))
        half = rng.normal(scale=0.3 * eps[p], size=(n, 3))
        keys = rng.choice(1 << 20, size=n, replace=False)
        for i in range(n):
            rows.append((p, keys[i] >> 8, keys[i] & 255, x[i] - half[i], x[i] + half[i]))
    perm = rng.permutation(len(rows))
    rows = [rows[i] for i in perm]
    pa = np.array([r[3] for r in rows]).reshape(-1, 3)
    pb = np.array([r[4] for r in rows]).reshape(-1, 3)
    return dict(pair=np.array([r[0] for r in rows], np.int32),
                ta=np.array([r[1] for r in rows], np.int32),
                tb=np.array([r[2] for r in rows], np.int32),
                pa=pa, pb=pb, d=np.sqrt(((pa - pb) ** 2).sum(1)))


def test_synthetic_lists_every_path(gctx, orc):
    """Pairs sized for the warp path (<= 64), the shared-memory block path
    (<= 1024) and the global-scratch block path, empty pairs, and eps small
    (nothing merges) and large (everything merges)."""
    import torch
    import paper_2105_12415_gb300 as m
    rng = np.random.default_rng(7)
    sizes = [0, 1, 2, 5, 31, 32, 33, 64, 65, 200, 1024, 1025, 3000, 0, 7, 40]
    spread = rng.uniform(0.01, 0.05, len(sizes))
    c = _synthetic(rng, sizes, spread)
    eps = spread.copy()
    eps[14] = 1e-9  # no links
    eps[15] = 1e3   # one component
    ref = orc.merge_contacts(c, eps)
    got_out, members = m.merge_contacts(gctx, torch.as_tensor(eps, device="cuda:0"), _device_list(c))
    got = _merged(got_out, members)
    _compare(got, ref)
    assert (got["members"][got["pair"] == 14] == 1).all()
    assert (got["members"][got["pair"] == 15] == 40).all()
    assert 0 < len(ref["d"]) < len(c["pair"])


def test_links_at_exactly_eps(gctx, orc):
    """Points on a grid with spacing exactly eps (powers of two, far from the
    origin so the float prefilter's band is exercised): neighbours are not
    closer than eps and nothing links; at a spacing just below eps the grid
    links into one contact."""
    import torch
    import paper_2105_12415_gb300 as m
    eps = 2.0 ** -6
    for spacing, n_out in [(eps, 64), (eps * (1 - 2.0 ** -40), 1)]:
        g = np.arange(8) * spacing
        x = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
        x = np.c_[x, np.zeros(len(x))] + [32.0, -16.0, 8.0]
        c = dict(pair=np.zeros(64, np.int32), ta=np.arange(64, dtype=np.int32),
                 tb=np.zeros(64, np.int32), pa=x, pb=x + [0.0, 0.0, 2.0 ** -8],
                 d=np.full(64, 2.0 ** -8))
        ref = orc.merge_contacts(c, [eps])
        out, members = m.merge_contacts(gctx, torch.tensor([eps], dtype=torch.float64, device="cuda:0"),
                                        _device_list(c))
        got = _merged(out, members)
        _compare(got, ref)
        assert len(got["d"]) == n_out


def test_paper_example_vertex_against_vertex(gctx, orc):
    """Two regular icosahedra tip to tip: the GPU detection finds the 5 x 5
    redundant contacts of the two tips; the merge leaves one contact at the
    tips with distance g."""
    import paper_2105_12415_gb300 as m
    v, f = icosphere(0)
    qA = _quat_from_matrix(_rotation_taking(v[0], np.array([1.0, 0, 0])))
    qB = _quat_from_matrix(_rotation_taking(v[3], np.array([-1.0, 0, 0])))
    g = 0.06
    s = scene_regular_pair(0, 1.0, 2.0 + g, qA, qB, 0.05)
    for precision in ("fp64", "fp32"):
        c, t, _ = _detected(gctx, s, precision)
        assert c.n() == 25
        out, members = m.merge_contacts(gctx, t["eps"], c)
        got = _merged(out, members)
        assert len(got["d"]) == 1 and got["members"][0] == 25
        tipA = orc.pose_matrix(s.poses[0]) @ s.verts[0].astype(np.float64) + s.poses[0][:3]
        tipB = orc.pose_matrix(s.poses[1]) @ s.verts[s.vert_off[1] + 3].astype(np.float64) + s.poses[1][:3]
        np.testing.assert_allclose(got["pa"][0], tipA, rtol=0, atol=1e-12)
        np.testing.assert_allclose(got["pb"][0], tipB, rtol=0, atol=1e-12)
        assert abs(got["d"][0] - g) <= 1e-6


def test_forces_of_the_merged_list(gctx, orc):
    """The merged list feeds the force kernel: forces and energy of the GPU's
    merged contacts against the oracle's forces of the oracle's merge."""
    import paper_2105_12415_gb300 as m
    s = scene_c1()
    c, t, hier = _detected(gctx, s, "fp64")
    ref = orc.merge_contacts(c.to_numpy(sort=False), s.eps)
    out, _ = m.merge_contacts(gctx, t["eps"], c)
    ft, en = m.contact_forces(gctx, hier, t["pairs"], t["eps"], t["poses"], out, t["mass"], t["com"])
    ft_ref, en_ref = orc.forces(s, ref)
    ft = ft.cpu().numpy()
    tot = np.abs(ft_ref).sum()
    assert np.abs(ft - ft_ref).max() <= 1e-9 * tot
    assert abs(float(en.item()) - en_ref) <= 1e-9 * en_ref


def test_order_independent_and_deterministic(gctx):
    import torch
    import paper_2105_12415_gb300 as m
    rng = np.random.default_rng(9)
    sizes = [50, 300, 1500]
    eps = np.array([0.03, 0.02, 0.04])
    c = _synthetic(rng, sizes, eps)
    e = torch.as_tensor(eps, device="cuda:0")
    o1, m1 = m.merge_contacts(gctx, e, _device_list(c))
    perm = rng.permutation(len(c["pair"]))
    o2, m2 = m.merge_contacts(gctx, e, _device_list({k: v[perm] for k, v in c.items()}))
    a, b = _merged(o1, m1), _merged(o2, m2)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_capacity_invalid_and_empty(gctx, orc):
    import torch
    import paper_2105_12415_gb300 as m
    from paper_2105_12415_gb300 import _lib as L
    rng = np.random.default_rng(3)
    eps = np.array([0.02, 0.03])
    c = _synthetic(rng, [100, 100], eps)
    e = torch.as_tensor(eps, device="cuda:0")
    ref = orc.merge_contacts(c, eps)
    # an output too small: reported with the required size, then grown
    small = m.Contacts(4, "cuda:0")
    _, _ = m.merge_contacts(gctx, e, _device_list(c), out=small, check=False)
    req = np.zeros(5, np.int64)
    st = L.load().mrdem_check(gctx.handle, None, req.ctypes.data)
    assert st == L.MRDEM_ERR_CAPACITY and req[3] == len(ref["d"])
    out, members = m.merge_contacts(gctx, e, _device_list(c), out=small)
    _compare(_merged(out, members), ref)
    # a pair index out of range is latched; the context stays usable
    bad = dict(c)
    bad["pair"] = c["pair"].copy()
    bad["pair"][0] = 2
    with pytest.raises(m.MrdemError) as err:
        m.merge_contacts(gctx, e, _device_list(bad))
    assert err.value.status == L.MRDEM_ERR_NONFINITE
    with pytest.raises(m.MrdemError):
        m.merge_contacts(gctx, torch.tensor([0.02, -1.0], dtype=torch.float64, device="cuda:0"),
                         _device_list(c))
    # empty input, and no pairs at all
    out, _ = m.merge_contacts(gctx, e, _device_list({k: v[:0] for k, v in c.items()}))
    assert out.n() == 0
    out, _ = m.merge_contacts(gctx, e[:0], _device_list({k: v[:0] for k, v in c.items()}))
    assert out.n() == 0
    out, members = m.merge_contacts(gctx, e, _device_list(c))
    _compare(_merged(out, members), ref)
