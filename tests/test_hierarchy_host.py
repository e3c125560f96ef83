"""Host construction of the surrogate trees (Sec. 4, Algorithm 7, Appendix A),
checked on the CPU: conservativeness of every surrogate (FP64 oracle
distances), tree shape, Table 1 magnitude, determinism and input errors."""
import json
import os

import numpy as np
import pytest

from gen import icosphere, scene_c1, scene_pairs

HERE = os.path.dirname(os.path.abspath(__file__))


def _host(scene, **kw):
    import paper_2105_12415_gb300 as m
    p = m.default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return m.Hierarchy.build_host(scene.vert_off, scene.verts, scene.tri_off, scene.tris, p)


def _fine_tris_below(ex, node):
    """Slots (fine triangles) below a node."""
    b, c = ex["node_child"][node]
    if c < 0:
        return list(range(b, b - c))
    out = []
    for ch in range(b, b + c):
        out += _fine_tris_below(ex, ch)
    return out


def _check_conservative(orc, scene, ex):
    nn = len(ex["node_delta"])
    worst = 0.0
    for node in range(nn):
        slots = _fine_tris_below(ex, node)
        parts = ex["slot_particle"][slots]
        assert np.all(parts == parts[0])
        v, t = scene.particle(int(parts[0]))
        vid = np.unique(t[ex["slot_tri"][slots]].ravel())
        V = v[vid].astype(np.float64)
        T = np.repeat(ex["node_tri"][node][None].astype(np.float64), len(V), 0)
        d = orc.vertex_surrogate_distance(V, T)
        assert d.max() <= float(ex["node_delta"][node]), (node, d.max(), ex["node_delta"][node])
        worst = max(worst, float(ex["node_delta"][node]) - d.max())
    return worst


def test_c1_tree_shape_and_conservativeness(orc):
    s = scene_c1()
    h = _host(s)
    info = h.info()
    ex = h.export()
    assert info["n_particles"] == 2 and info["n_tri"] == 2560 and info["max_depth"] == 3
    # one root + 8 + 64 leaves of 20 triangles per particle
    assert info["n_nodes"] == 2 * 73
    lvl = ex["node_level"]
    for i in range(2):
        r = ex["root"][i]
        assert lvl[r] == 1
        nodes = np.arange(r, r + 73)
        assert (lvl[nodes] == 1).sum() == 1 and (lvl[nodes] == 2).sum() == 8 and (lvl[nodes] == 3).sum() == 64
        leaves = nodes[ex["node_child"][nodes, 1] < 0]
        assert len(leaves) == 64 and np.all(-ex["node_child"][leaves, 1] == 20)
    # every fine triangle sits in exactly one slot
    sl = ex["slot_tri"] >= 0
    keys = ex["slot_particle"][sl].astype(np.int64) * 100000 + ex["slot_tri"][sl]
    assert len(np.unique(keys)) == 2560
    _check_conservative(orc, s, ex)


@pytest.mark.parametrize("level,depth", [(1, 2), (2, 3), (3, 3), (4, 4), (5, 5)])
def test_depth_by_size(level, depth):
    s = scene_pairs([level], [1], [1.0], [1.0], [0.01], [0.0], 3, "depth")
    h = _host(s)
    ex = h.export()
    r0 = ex["root"][0]
    r1 = ex["root"][1]
    lv = ex["node_level"][r0:r1]
    assert lv.max() == depth
    child = ex["node_child"][r0:r1]
    leaves = child[:, 1] < 0
    assert np.all(-child[leaves, 1] <= 32) and np.all(-child[leaves, 1] >= 16)
    assert np.all(child[~leaves, 1] <= 8) and np.all(child[~leaves, 1] >= 2)
    # breadth-first: children follow their parent, levels never decrease
    assert np.all(np.diff(lv) >= 0)
    for k in np.nonzero(~leaves)[0]:
        b, c = child[k]
        assert b > r0 + k and np.all(ex["node_level"][b:b + c] == lv[k] + 1)


def test_conservative_on_batched_sizes(orc):
    s = scene_pairs([1, 2, 4], [3, 2, 1], [0.3, 1.0, 0.12], [1.0, 0.5, 0.8], [0.003] * 3,
                    [0.0] * 3, 8, "mixed")
    h = _host(s)
    _check_conservative(orc, s, h.export())


def test_table1_root_surrogate_magnitude():
    """Table 1, eta_r = 1: the single-triangle root of an unbumped
    unit-diameter sphere needs eps_kmax ~ r_sphere = 0.5."""
    g = json.load(open(os.path.join(HERE, "golden", "table1_root_surrogate.json")))
    from gen.icosphere import _assemble
    for nt, eps_paper in zip(g["n_triangles"], g["eps_kmax"]):
        level = {80: 1, 320: 2, 1280: 3}[nt]
        v, f = icosphere(level)
        m = ((v * 0.5).astype(np.float32), f)
        s = _assemble([m], [[0, 0, 0, 1, 0, 0, 0]], [0.5], np.zeros((0, 2)), [], "unit-diameter")
        ex = _host(s).export()
        delta = float(ex["node_delta"][ex["root"][0]])
        assert abs(delta - g["r_sphere"]) <= 0.1 * g["r_sphere"]
        assert abs(delta - eps_paper) <= 0.1 * g["r_sphere"]


def test_deterministic():
    s = scene_pairs([3], [2], [1.0], [0.4], [0.01], [0.0], 5, "det")
    a, b = _host(s).export(), _host(s).export()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_invalid_inputs():
    import paper_2105_12415_gb300 as m
    s = scene_pairs([1], [1], [1.0], [1.0], [0.01], [0.0], 5, "bad")
    bad = s.tris.copy()
    bad[5, 1] = 10_000
    with pytest.raises(m.MrdemError):
        m.Hierarchy.build_host(s.vert_off, s.verts, s.tri_off, bad)
    deg = s.tris.copy()
    deg[3] = [deg[3, 0], deg[3, 0], deg[3, 1]]
    with pytest.raises(m.MrdemError):
        m.Hierarchy.build_host(s.vert_off, s.verts, s.tri_off, deg)
    with pytest.raises(m.MrdemError):
        m.Hierarchy.build_host(np.array([0]), s.verts, np.array([0]), s.tris)


def test_fanout_bounds():
    """A split has at most `fanout` children (<= 8) whatever leaf_min asks,
    and a fanout above 8 is rejected."""
    import paper_2105_12415_gb300 as m
    s = scene_pairs([4], [2], [1.0], [0.4], [0.01], [0.0], 5, "fan")
    with pytest.raises(m.MrdemError):
        _host(s, fanout=9)
    for fan, leaf_min in ((8, 64), (3, 32), (2, 1)):
        ex = _host(s, fanout=fan, leaf_min=leaf_min).export()
        ch = ex["node_child"]
        inner = ch[:, 1] > 0
        assert inner.any()
        assert ch[inner, 1].max() <= fan
        leaves = ch[:, 1] < 0
        assert (-ch[leaves, 1]).max() <= 32


def _parents(ex):
    par = -np.ones(len(ex["node_delta"]), np.int64)
    for k, (b, c) in enumerate(ex["node_child"]):
        if c > 0:
            par[b:b + c] = k
    return par


@pytest.mark.parametrize("levels", [(3, 3), (2, 4)])
def test_ancestors_of_every_contact_pass_the_surrogate_test(orc, levels):
    """Lemma 1's premise on the built trees: for every oracle contact (fine
    pair within 2 eps), each pair of ancestors that Algorithm 5 examines on
    the way down (both sides unfold together; a side that reached its leaf
    stays there) has surrogates within delta_a + delta_b + 2 eps in FP64, so
    no certified prune can drop it."""
    s = scene_pairs([levels[0]], [levels[1]], [1.0], [1.0], [0.02], [-0.2], 9, "anc")
    c = orc.detect(s)
    assert len(c["d"]) > 50
    ex = _host(s).export()
    par = _parents(ex)
    # input triangle -> leaf node, per particle
    leaf_of = {}
    for k, (b, cnt) in enumerate(ex["node_child"]):
        if cnt < 0:
            for slot in range(b, b - cnt):
                if ex["slot_tri"][slot] >= 0:
                    leaf_of[(int(ex["slot_particle"][slot]), int(ex["slot_tri"][slot]))] = k
    R = [orc.pose_matrix(s.poses[i]) for i in range(2)]

    def world(node, i):
        T = ex["node_tri"][node].reshape(3, 3).astype(np.float64)
        return (T @ R[i].T + s.poses[i][:3]).ravel()

    def chain(leaf):
        out = [leaf]
        while par[out[-1]] >= 0:
            out.append(int(par[out[-1]]))
        return out[::-1]  # root first

    P, Q, lim = [], [], []
    for ta, tb in zip(c["ta"], c["tb"]):
        ca, cb = chain(leaf_of[(0, int(ta))]), chain(leaf_of[(1, int(tb))])
        for lvl in range(max(len(ca), len(cb))):
            na, nb = ca[min(lvl, len(ca) - 1)], cb[min(lvl, len(cb) - 1)]
            P.append(world(na, 0))
            Q.append(world(nb, 1))
            lim.append(float(ex["node_delta"][na]) + float(ex["node_delta"][nb]) + 2 * s.eps[0])
    d = orc.tri_tri(np.array(P), np.array(Q))[0]
    lim = np.array(lim)
    assert np.all(d <= lim * (1 + 1e-12)), (d - lim).max()


def test_conservative_on_large_disparate_particles(orc):
    """An 81,920-triangle particle (subdivision 6, radius 20) beside a small
    one: depth 5 with leaves of 20, every surrogate conservative."""
    from gen import scene_disparity
    s = scene_disparity(1)
    h = _host(s)
    info = h.info()
    assert info["n_tri"] == 81920 + 1280 and info["max_depth"] == 5
    _check_conservative(orc, s, h.export())


def _box_contains_all(ex, scene, node, box):
    slots = _fine_tris_below(ex, node)
    part = int(ex["slot_particle"][slots[0]])
    v, t = scene.particle(part)
    V = v[np.unique(t[ex["slot_tri"][slots]].ravel())].astype(np.float64)
    c = box[0:3].astype(np.float64)
    U = box[3:12].reshape(3, 3).astype(np.float64)
    half = box[12:15].astype(np.float64)
    proj = np.abs((V - c) @ U.T)
    return bool((proj <= half).all()), U, half, V


@pytest.mark.parametrize("which", ["c1", "disparity", "plane"])
def test_node_boxes_contain_their_fine_vertices(which):
    """Every node's oriented box holds every fine vertex below it, exactly
    in FP64 with the stored float values; the axes are orthonormal to float
    rounding; no half extent exceeds the node's vertex spread.  The plane
    particles (one triangle) get a flat box."""
    from gen import scene_disparity, scene_particle_on_plane
    s = {"c1": scene_c1, "disparity": lambda: scene_disparity(1),
         "plane": scene_particle_on_plane}[which]()
    ex = _host(s).export()
    boxes = ex["node_box"]
    assert boxes.shape == (len(ex["node_delta"]), 16)
    step = 1 if which == "c1" else 7
    for node in range(0, len(boxes), step):
        ok, U, half, V = _box_contains_all(ex, s, node, boxes[node])
        assert ok, node
        assert np.abs(U @ U.T - np.eye(3)).max() < 1e-6
        spread = np.linalg.norm(V.max(0) - V.min(0))
        assert half.max() <= spread
        if len(V) == 3:  # a single triangle: its box has no thickness
            assert half.min() <= 1e-6 * half.max()


def test_box_of_a_cuboid_is_the_cuboid():
    """A cuboid with sides 4 > 2 > 1, turned and moved: the principal axes of
    its 8 corners are its edges, so its box is the cuboid itself (half
    extents 2, 1, 0.5, centre its centre)."""
    from gen.icosphere import _assemble
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    corners = np.array([[x, y, z] for x in (-2, 2) for y in (-1, 1) for z in (-0.5, 0.5)], float)
    c0 = np.array([0.25, -0.5, 0.125])
    verts = (corners @ Q.T + c0).astype(np.float32)
    faces = np.array([[0, 1, 3], [0, 3, 2], [4, 6, 7], [4, 7, 5], [0, 4, 5], [0, 5, 1],
                      [2, 3, 7], [2, 7, 6], [0, 2, 6], [0, 6, 4], [1, 5, 7], [1, 7, 3]], np.int32)
    s = _assemble([(verts, faces)], [[0, 0, 0, 1, 0, 0, 0]], [2.3], np.zeros((0, 2)), [], "cuboid")
    ex = _host(s).export()
    box = ex["node_box"][ex["root"][0]]
    np.testing.assert_allclose(np.sort(box[12:15]), [0.5, 1.0, 2.0], rtol=1e-6)
    np.testing.assert_allclose(box[0:3], c0, atol=1e-6)
    U = box[3:12].reshape(3, 3)
    # each axis is parallel to one cuboid edge direction
    assert np.allclose(np.sort(np.abs(U @ Q).max(1)), 1.0, atol=1e-6)


def test_boxes_prune_leaf_pairs_the_surrogates_keep(orc):
    """The purpose of the boxes: on the one-pair workload, of the leaf pairs
    that pass the exact surrogate test (delta_a + delta_b + 2 eps), the
    six face axes of the two boxes separate a good share by more than 2 eps,
    and never one that holds a fine pair within 2 eps."""
    s = scene_c1()
    ex = _host(s).export()
    boxes = ex["node_box"]
    c = orc.detect(s)
    R = [orc.pose_matrix(s.poses[i]) for i in range(2)]

    def world_box(i, k):
        b = boxes[k].astype(np.float64)
        return (R[i] @ b[0:3] + s.poses[i][:3], b[3:12].reshape(3, 3) @ R[i].T, b[12:15])

    def separated(A, B, gap):
        for ax in list(A[1]) + list(B[1]):
            ra = np.abs(A[1] @ ax) @ A[2]
            rb = np.abs(B[1] @ ax) @ B[2]
            if abs((B[0] - A[0]) @ ax) > ra + rb + gap:
                return True
        return False

    leaves = [[k for k in range(len(boxes)) if ex["node_child"][k, 1] < 0 and
               ex["slot_particle"][ex["node_child"][k, 0]] == i] for i in range(2)]
    slot_leaf = {}
    for i in range(2):
        for k in leaves[i]:
            b, n = ex["node_child"][k]
            for sl in range(b, b - n):
                slot_leaf[(i, int(ex["slot_tri"][sl]))] = k
    contact_leaves = {(slot_leaf[(0, int(a))], slot_leaf[(1, int(b))]) for a, b in zip(c["ta"], c["tb"])}
    P, Q, lim, keys = [], [], [], []
    for ka in leaves[0]:
        for kb in leaves[1]:
            P.append((ex["node_tri"][ka].reshape(3, 3).astype(np.float64) @ R[0].T + s.poses[0][:3]).ravel())
            Q.append((ex["node_tri"][kb].reshape(3, 3).astype(np.float64) @ R[1].T + s.poses[1][:3]).ravel())
            lim.append(ex["node_delta"][ka] + ex["node_delta"][kb] + 2 * s.eps[0])
            keys.append((ka, kb))
    d = orc.tri_tri(np.array(P), np.array(Q))[0]
    passing = [keys[i] for i in np.flatnonzero(d <= np.array(lim))]
    cut = [k for k in passing if separated(world_box(0, k[0]), world_box(1, k[1]), 2 * s.eps[0])]
    assert contact_leaves <= set(passing)
    assert not (set(cut) & contact_leaves)
    assert len(cut) >= 0.2 * len(passing), (len(cut), len(passing))
