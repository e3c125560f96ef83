"""The oracle's contact set of large particle pairs in seconds (test
infrastructure; it uses the oracle, the product never does).

The oracle's detect tests every fine triangle pair; for the batched
workload's largest pairs (20 480 x 20 480 triangles) that takes minutes.
Here every fine triangle gets a bounding sphere in the world frame (centroid
and largest vertex distance, FP64, widened by a margin far above rounding),
and only the triangle pairs whose spheres come within 2 eps of each other go
to the oracle's own distance (oracle.tri_pairs: the world triangles and
exact distance that detect uses, so those pairs get detect's values).  A
pair outside that test is more than 2 eps apart (two sets are at least as
far apart as balls that contain them), so the contact set {d <= 2 eps} is
detect's; test_oracle_filtered pins this against detect's full brute force.
"""
import numpy as np


def _spheres(T):
    V = T.reshape(-1, 3, 3)
    c = V.mean(axis=1)
    r = np.sqrt(((V - c[:, None, :]) ** 2).sum(-1)).max(axis=1)
    return c, r


def contacts(orc, scene, pair_ids=None):
    """detect's contact dict for the pairs pair_ids of scene (pair indices as
    in scene; sorted by pair, ta, tb)."""
    from scipy.spatial import cKDTree
    pair_ids = np.arange(scene.n_pairs) if pair_ids is None else np.asarray(pair_ids)
    abt, owner = [], []
    for p in pair_ids:
        A, B = (int(x) for x in scene.pairs[p])
        TA, TB = orc.world_triangles(scene, A), orc.world_triangles(scene, B)
        ca, ra = _spheres(TA)
        cb, rb = _spheres(TB)
        tau = 2.0 * scene.eps[p]
        scale = np.abs(TA).max() + np.abs(TB).max()
        margin = 1e-9 * scale + 1e-6 * tau
        cand = cKDTree(cb).query_ball_point(ca, ra + rb.max() + tau + margin)
        ii = np.repeat(np.arange(len(ca)), [len(c) for c in cand])
        jj = np.fromiter((j for c in cand for j in c), dtype=np.int64, count=len(ii))
        if len(ii):
            gap = np.sqrt(((ca[ii] - cb[jj]) ** 2).sum(1)) - ra[ii] - rb[jj]
            keep = gap <= tau + margin
            ii, jj = ii[keep], jj[keep]
        if len(ii):
            abt.append(np.stack([np.full(len(ii), A), ii, np.full(len(ii), B), jj], axis=1))
            owner.append(np.full(len(ii), p, np.int64))
    if not abt:
        return {"pair": np.empty(0, np.int32), "ta": np.empty(0, np.int32),
                "tb": np.empty(0, np.int32), "d": np.empty(0), "pa": np.empty((0, 3)),
                "pb": np.empty((0, 3)), "feature": np.empty(0, np.int32)}
    abt = np.concatenate(abt)
    owner = np.concatenate(owner)
    d, pa, pb, f = orc.tri_pairs(scene, abt)
    hit = d <= 2.0 * scene.eps[owner]
    o = np.lexsort((abt[hit, 3], abt[hit, 1], owner[hit]))
    return {"pair": owner[hit][o].astype(np.int32), "ta": abt[hit, 1][o].astype(np.int32),
            "tb": abt[hit, 3][o].astype(np.int32), "d": d[hit][o], "pa": pa[hit][o],
            "pb": pb[hit][o], "feature": f[hit][o]}
