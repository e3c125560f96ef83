"""Helpers shared by the GPU parity tests."""
import numpy as np

# Tolerances (stated for every comparison with the FP64 oracle):
#  * contact sets equal except pairs whose oracle distance lies within
#    1e-6 eps of the threshold 2 eps (plus the rounding floor below);
#  * distances: |d - d_ref| <= TOL_D * max(d_ref, eps) + K_U * u * S, TOL_D =
#    1e-12 for the FP64 form and 1e-5 for the FP32 form; u = 2^-53 and S =
#    |t_A| + |t_B| + r_A + r_B bounds the world coordinates the oracle
#    computes with.  The floor is the rounding of the two FP64 computations
#    themselves: the oracle moves both triangles into the world frame, the
#    GPU moves B into A's frame, each coordinate with an error of a few u S,
#    and the distance is 1-Lipschitz in the vertices; K_U = 8 bounds the
#    sum (the precision report prints the measured largest error in units of
#    u S: below 1 on every parity workload);
#  * closest points: the distance fixes them only up to ties (parallel
#    features), so every contact's points are checked for validity instead:
#    p_a on A's world triangle and p_b on B's within K_P u S, and
#    | |p_a - p_b| - d_ref | within the distance tolerance.  K_P = 64: a
#    closest point is found by projections and clamps whose rounding is not
#    damped the way the distance's is (the distance is flat along a tie);
#  * forces / torques: per particle |F - F_ref| <= 1e-5 * sum_c |F_c| (FP32
#    form), 1e-9 (FP64 form), plus per contact the effect of the rounding
#    floor (see test_forces_match_oracle).
BAND = 1e-6
TOL_D = {"fp64": 1e-12, "fp32": 1e-5}
U = 2.0 ** -53
K_U = 8
K_P = 64


def gpu_scene_tensors(scene, device):
    import torch
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)  # noqa: E731
    return dict(pairs=t(scene.pairs, torch.int32), eps=t(scene.eps, torch.float64),
                poses=t(scene.poses, torch.float64), mass=t(scene.mass, torch.float64),
                com=t(scene.com, torch.float64))


def world_scale(scene):
    """S per pair: a bound of the world coordinates of the pair's vertices."""
    A, B = scene.pairs[:, 0], scene.pairs[:, 1]
    t = np.linalg.norm(scene.poses[:, :3], axis=1)
    r = 1.06 * scene.radius
    return t[A] + t[B] + r[A] + r[B]


def _point_to_triangles(p, T):
    """FP64 distance of points p [n, 3] to triangles T [n, 9] (oracle)."""
    import oracle
    d, _ = oracle.point_triangle(p, T)
    return d


def compare_contacts(got, ref, scene, precision, check_points=True, report=None, poses=None):
    """Contact sets (sorted dicts) equal outside the threshold band; distances
    within tolerance; closest points valid (on the triangles at `poses`,
    default the scene's).  Returns the largest distance error relative to
    max(d_ref, eps) and stores the largest errors in units of u S in
    `report` (a dict) when given."""
    import oracle
    eps_of_pair = scene.eps
    floor = K_U * U * world_scale(scene)
    tau = 2 * eps_of_pair
    kg = set(zip(got["pair"].tolist(), got["ta"].tolist(), got["tb"].tolist()))
    kr = set(zip(ref["pair"].tolist(), ref["ta"].tolist(), ref["tb"].tolist()))
    ref_d = dict(zip(zip(ref["pair"].tolist(), ref["ta"].tolist(), ref["tb"].tolist()), ref["d"].tolist()))
    missing = kr - kg
    for k in missing:
        p = k[0]
        assert abs(ref_d[k] - tau[p]) <= BAND * eps_of_pair[p] + floor[p], ("missing contact", k, ref_d[k], tau[p])
    extra = kg - kr
    got_d = dict(zip(zip(got["pair"].tolist(), got["ta"].tolist(), got["tb"].tolist()), got["d"].tolist()))
    for k in extra:
        p = k[0]
        assert abs(got_d[k] - tau[p]) <= BAND * eps_of_pair[p] + TOL_D[precision] * tau[p] + floor[p], ("extra contact", k, got_d[k], tau[p])
    # distances on the common set
    common = np.array(sorted(kg & kr))
    if len(common) == 0:
        return 0.0
    gi = {k: i for i, k in enumerate(zip(got["pair"].tolist(), got["ta"].tolist(), got["tb"].tolist()))}
    ri = {k: i for i, k in enumerate(zip(ref["pair"].tolist(), ref["ta"].tolist(), ref["tb"].tolist()))}
    ig = np.array([gi[tuple(k)] for k in common])
    ir = np.array([ri[tuple(k)] for k in common])
    e = eps_of_pair[common[:, 0]]
    fl = floor[common[:, 0]]
    us = U * world_scale(scene)[common[:, 0]]
    adiff = np.abs(got["d"][ig] - ref["d"][ir])
    err = (adiff - fl).clip(0) / np.maximum(ref["d"][ir], e)
    if report is not None:
        report["distance_uS"] = float((adiff / us).max())
    assert err.max() <= TOL_D[precision], err.max()
    if check_points:
        # the points of every common contact lie on their triangles, at the
        # contact's distance from each other
        A = scene.pairs[common[:, 0], 0]
        B = scene.pairs[common[:, 0], 1]
        TA = np.empty((len(common), 9))
        TB = np.empty((len(common), 9))
        for i in np.unique(np.concatenate([A, B])):
            W = oracle.world_triangles(scene, i, poses=poses)
            sa = A == i
            TA[sa] = W[common[sa, 1]]
            sb = B == i
            TB[sb] = W[common[sb, 2]]
        pa, pb = got["pa"][ig], got["pb"][ig]
        da = _point_to_triangles(pa, TA)
        db = _point_to_triangles(pb, TB)
        sep = np.abs(np.linalg.norm(pa - pb, axis=1) - ref["d"][ir])
        if report is not None:
            report["points_on_triangles_uS"] = float((np.maximum(da, db) / us).max())
            report["separation_uS"] = float((sep / us).max())
        fp = K_P * us
        assert np.all(da <= fp) and np.all(db <= fp), (da.max(), db.max())
        assert np.all(sep <= TOL_D[precision] * np.maximum(ref["d"][ir], e) + fl), sep.max()
    return float(err.max())
