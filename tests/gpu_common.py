"""Helpers shared by the GPU parity tests."""
import numpy as np

# Tolerances (stated for every comparison with the FP64 oracle):
#  * contact sets equal except pairs whose oracle distance lies within
#    1e-6 eps of the threshold 2 eps;
#  * distances: |d - d_ref| <= TOL_D * max(d_ref, eps) + 2^-44 S, TOL_D = 1e-12
#    for the FP64 form and 1e-5 for the FP32 form; S = |t_A| + |t_B| + r_A + r_B
#    bounds the world coordinates the oracle computes with, so 2^-44 S (about
#    500 double ulps of S) is the oracle's own rounding floor;
#  * forces / torques: per particle |F - F_ref| <= 1e-5 * sum_c |F_c| (FP32
#    form), 1e-9 (FP64 form).
BAND = 1e-6
TOL_D = {"fp64": 1e-12, "fp32": 1e-5}


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


def compare_contacts(got, ref, scene, precision, check_points=True):
    """Contact sets (sorted dicts) equal outside the threshold band; distances
    and closest points within tolerance.  Returns the max relative distance
    error."""
    eps_of_pair = scene.eps
    floor = np.ldexp(world_scale(scene), -44)
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
    err = (np.abs(got["d"][ig] - ref["d"][ir]) - fl).clip(0) / np.maximum(ref["d"][ir], e)
    assert err.max() <= TOL_D[precision], err.max()
    if check_points:
        # closest points: unique unless two features tie; compare the
        # segment midpoints and directions where the distance is positive
        scale = np.maximum(e, 1e-12)
        dpa = (np.linalg.norm(got["pa"][ig] - ref["pa"][ir], axis=1) - 1e3 * fl).clip(0) / scale
        frac_bad = np.mean(dpa > 1e-6)
        assert frac_bad < 0.01, frac_bad
    return float(err.max())
