"""Precision report: the largest error of each GPU output against the FP64
oracle, for the FP32 and FP64 forms, on the parity workloads.

Run on a GPU host (not collected by pytest):

    python tests/precision_report.py profiles/precision_report.md

Outputs and how their errors are measured (the same quantities the parity
tests bound):
  contact set      contacts missing / extra against the oracle, and how many
                   of those lie within 1e-6 eps of the threshold 2 eps;
  distance         max |d - d_ref| / max(d_ref, eps) over the common contacts;
  distance_uS      max |d - d_ref| in units of u S (u = 2^-53, S = |t_A| +
                   |t_B| + r_A + r_B: the world coordinates' magnitude), the
                   rounding floor of the distance tolerance;
  closest points   max |p_a - p_a,ref| / eps over common contacts with d > 0;
  points_uS        largest distance of p_a from A's triangle (p_b from B's),
                   in units of u S (the closest-point floor of the tests);
  force, torque    per particle max |F - F_ref| / sum_c |F_c| (torque: over
                   sum_c |F_c| times the largest lever);
  energy           |E - E_ref| / E_ref;
  pose gradient    max |g - g_ref| / max |g_ref| (the differentiation
                   workload, which has no touching pairs);
  Jacobian blocks  max |J - J_ref| / max |J_ref|;
  vertex gradient  max |g - g_ref| / max |g_ref| (a float output).
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def _workloads():
    from gen import scene_c1, scene_c2, scene_c3, scene_disparity, scene_particle_on_plane
    c2 = scene_c2()
    ntri = np.diff(c2.tri_off)
    small = [k for k in range(0, c2.n_pairs, 8)
             if ntri[c2.pairs[k, 0]] * ntri[c2.pairs[k, 1]] <= 1280 * 5120][:48]
    return [("one pair, 1280 triangles", scene_c1(), False),
            ("batched workload, 48 sampled pairs", c2.subset(small), False),
            ("differentiation, 8 pairs of 5120", scene_c3().subset(np.arange(0, 1024, 128)), True),
            ("particle on plane", scene_particle_on_plane(), False),
            ("size disparity 20:1, 2 pairs", scene_disparity(2), False)]


def _contact_errors(got, ref, scene):
    key = lambda c: list(zip(c["pair"].tolist(), c["ta"].tolist(), c["tb"].tolist()))  # noqa: E731
    kg, kr = key(got), key(ref)
    sg, sr = set(kg), set(kr)
    dref = dict(zip(kr, ref["d"].tolist()))
    dgot = dict(zip(kg, got["d"].tolist()))
    eps = scene.eps
    near = lambda k, d: abs(d - 2 * eps[k[0]]) <= 1e-6 * eps[k[0]]  # noqa: E731
    missing = sr - sg
    extra = sg - sr
    common = sorted(sg & sr)
    gi = {k: i for i, k in enumerate(kg)}
    ri = {k: i for i, k in enumerate(kr)}
    from tests.gpu_common import U, world_scale
    uS = U * world_scale(scene)
    derr = perr = duS = 0.0
    for k in common:
        e = eps[k[0]]
        derr = max(derr, abs(dgot[k] - dref[k]) / max(dref[k], e))
        duS = max(duS, abs(dgot[k] - dref[k]) / uS[k[0]])
        if dref[k] > 0:
            perr = max(perr, float(np.linalg.norm(got["pa"][gi[k]] - ref["pa"][ri[k]])) / e)
    # closest points: largest distance of p_a (p_b) from A's (B's) world
    # triangle, in units of u S
    pts = 0.0
    if common:
        import oracle
        ig = np.array([gi[k] for k in common])
        A = scene.pairs[[k[0] for k in common], 0]
        B = scene.pairs[[k[0] for k in common], 1]
        TA = np.empty((len(common), 9))
        TB = np.empty((len(common), 9))
        ta = np.array([k[1] for k in common])
        tb = np.array([k[2] for k in common])
        for i in np.unique(np.concatenate([A, B])):
            W = oracle.world_triangles(scene, i)
            TA[A == i] = W[ta[A == i]]
            TB[B == i] = W[tb[B == i]]
        da, _ = oracle.point_triangle(got["pa"][ig], TA)
        db, _ = oracle.point_triangle(got["pb"][ig], TB)
        us = np.array([uS[k[0]] for k in common])
        pts = float((np.maximum(da, db) / us).max())
    return {"missing": len(missing), "missing_in_band": sum(near(k, dref[k]) for k in missing),
            "extra": len(extra), "extra_in_band": sum(near(k, dgot[k]) for k in extra),
            "distance": derr, "distance_uS": duS, "points": perr, "points_uS": pts,
            "common": len(common)}


def _force_errors(ft, e, ft_ref, e_ref, ref, scene):
    mu = 1 / (1 / scene.mass[scene.pairs[:, 0]] + 1 / scene.mass[scene.pairs[:, 1]])
    mag = 1000 * np.sqrt(mu[ref["pair"]]) * (1 - ref["d"] / (2 * scene.eps[ref["pair"]]))
    tot = np.zeros(scene.n_particles)
    for col in (0, 1):
        np.add.at(tot, scene.pairs[ref["pair"], col], mag)
    lever = 2 * (scene.radius.max() + np.abs(scene.poses[:, :3]).max())
    has = tot > 0
    f = np.abs(ft[:, :3] - ft_ref[:, :3]).max(1)[has] / tot[has] if has.any() else np.zeros(1)
    t = np.abs(ft[:, 3:] - ft_ref[:, 3:]).max(1)[has] / (tot[has] * lever) if has.any() else np.zeros(1)
    return {"force": float(f.max()), "torque": float(t.max()),
            "energy": abs(e - e_ref) / max(e_ref, 1e-300)}


def _implicit_rows(m, ctx, orc):
    """The implicit step on the four-particle chain against the oracle's
    Picard fixed point: broad phase (exact equality), Picard and Newton steps
    in both forms (largest velocity error relative to the largest velocity),
    and the contact Hessian blocks (relative to the largest entry)."""
    import dataclasses

    import torch

    import oracle.implicit as imp
    from gen import scene_chain
    dev = torch.device("cuda:0")
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    s = scene_chain(4, seed=41)
    bound = imp.bounding_radius(s)
    pairs = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    eps = imp.pair_eps(s.radius, pairs[:, 0], pairs[:, 1])
    vel = np.random.default_rng(2).normal(scale=0.1, size=(s.n_particles, 6))
    dt = 2e-4
    P, V, it, _ = imp.implicit_euler_step(s, vel, pairs, eps, dt, tol=2e-13, max_iter=2000)
    hier = m.Hierarchy.from_scene(ctx, s)
    inertia = 0.4 * s.mass * s.radius ** 2
    gp, _ = m.broad_phase(ctx, t(s.poses), t(bound), t(s.radius))
    rows = [{"workload": "chain: broad phase", "form": "fp64",
             "error": 0.0 if np.array_equal(gp.cpu().numpy(), pairs) else float("inf")}]
    args = (t(s.poses), t(vel), t(s.mass), t(inertia), t(pairs, torch.int32), t(eps), dt)
    for form, tol in (("fp64", 1e-11), ("fp32", 1e-5)):
        _, Vp, itp, _ = m.implicit_euler_step(ctx, hier, *args, precision=form, tol=tol)
        _, Vn, itn, _ = m.implicit_euler_step_newton(ctx, hier, *args, precision=form, tol=tol)
        scale = np.abs(V).max()
        rows.append({"workload": f"chain: Picard step ({itp} iterations, oracle {it})", "form": form,
                     "error": float(np.abs(Vp.cpu().numpy() - V).max() / scale)})
        rows.append({"workload": f"chain: Newton step ({itn} iterations)", "form": form,
                     "error": float(np.abs(Vn.cpu().numpy() - V).max() / scale)})
    base = dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((s.n_particles, 3)))
    c = orc.detect(base)
    Href = imp.contact_hessian(base, c)
    tp = t(pairs, torch.int32)
    cont, _ = m.detect(ctx, hier, tp, t(eps), t(s.poses), "fp64")
    blocks, _ = m.contact_hessian(ctx, hier, tp, t(eps), t(s.poses), cont, t(s.mass))
    H = np.zeros_like(Href)
    for p, (a, b) in enumerate(pairs):
        idx = np.r_[6 * a:6 * a + 6, 6 * b:6 * b + 6]
        H[np.ix_(idx, idx)] += blocks[p].cpu().numpy()
    rows.append({"workload": "chain: contact Hessian blocks", "form": "fp64",
                 "error": float(np.abs(H - Href).max() / np.abs(Href).max())})
    return rows


def main(out_path=None):
    import torch

    import oracle
    import paper_2105_12415_gb300 as m
    if not torch.cuda.is_available():
        raise SystemExit("needs a GPU")
    m.build()
    oracle.build()
    ctx = m.Context(0)
    dev = torch.device("cuda:0")
    rows = []
    for name, s, grads in _workloads():
        ref = oracle.detect(s)
        ft_ref, e_ref = oracle.forces(s, ref)
        gref = oracle.grad(s, ref) if grads else None
        hier = m.Hierarchy.from_scene(ctx, s)
        for form in ("fp32", "fp64"):
            prob = m.ContactProblem.from_scene(ctx, hier, s, dev, precision=form)
            c, _ = prob.detect()
            got = c.to_numpy()
            row = {"workload": name, "form": form, "contacts": len(ref["d"])}
            row.update(_contact_errors(got, ref, s))
            ft, e = prob.forces()
            row.update(_force_errors(ft.cpu().numpy(), float(e.item()), ft_ref, e_ref, ref, s))
            if grads:
                gv, gp, jac = prob.grad(want_jac=True)
                gv_ref, gp_ref, jac_ref = gref
                row["pose_grad"] = float(np.abs(gp.cpu().numpy() - gp_ref).max() / np.abs(gp_ref).max())
                row["jacobian"] = float(np.abs(jac.cpu().numpy().reshape(jac_ref.shape) - jac_ref).max()
                                        / np.abs(jac_ref).max())
                row["vertex_grad"] = float(np.abs(gv.cpu().numpy() - gv_ref).max() / np.abs(gv_ref).max())
            rows.append(row)
            print(row, flush=True)
    cols = ["workload", "form", "contacts", "missing", "missing_in_band", "extra", "extra_in_band",
            "distance", "distance_uS", "points", "points_uS", "force", "torque", "energy", "pose_grad", "jacobian", "vertex_grad"]
    fmt = lambda v: (f"{v:.2e}" if isinstance(v, float) else str(v))  # noqa: E731
    lines = ["| " + " | ".join(cols) + " |", "|" + "---|" * len(cols)]
    for r in rows:
        lines.append("| " + " | ".join(fmt(r.get(k, "")) for k in cols) + " |")
    text = "\n".join(lines) + "\n"
    irows = _implicit_rows(m, ctx, oracle)
    text += "\nImplicit step (row f1), largest error relative to the largest value:\n\n"
    text += "| quantity | form | error |\n|---|---|---|\n"
    for r in irows:
        text += f"| {r['workload']} | {r['form']} | {r['error']:.2e} |\n"
    print(text)
    if out_path:
        how = __doc__[__doc__.index("Outputs and how"):].strip()
        with open(out_path, "w") as f:
            f.write("# Precision report: GPU outputs against the FP64 oracle\n\n"
                    f"Command: `python tests/precision_report.py {out_path}`\n\n"
                    f"{how}\n\n{text}")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
