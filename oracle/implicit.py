"""FP64 CPU oracle of the implicit time step (test infrastructure only: the
tests and bench.py's CPU-baseline leg use it; the product path never does).

Broad phase: the particle pairs whose bounding spheres, each widened by the
pair's eps, overlap, by brute force over all pairs.

Implicit Euler step (Algorithm 3, with the force law of Sec. 2): the paper's
Picard iteration.  Starting from the current velocities, repeat: find the
contacts of every candidate pair at the guessed geometry, compute the
contact forces and torques there, set the guessed velocities to
v + dt (F / m + g) and omega + dt tau / I, and move the guessed geometry from
the step's start by dt times the guessed velocities (translation of the
centre of mass; rotation by the rotation vector dt omega, applied in the
world frame); stop when the guessed velocities no longer change.  The
fixed point is the implicit Euler solution; damping or acceleration of the
iteration (Sec. 6) change the path to it, not the point, and are left out.

Contact Hessian (`contact_hessian`): the second derivatives of the contact
energy in the pose twists with the closest points free, in closed form per
contact (the closest-point parameters eliminated by the implicit function
theorem), for Newton's method on the same equations.

Readings (the paper leaves them open): the particles' inertia is that of a
solid sphere of the particle's radius, I = 2/5 m r^2 (isotropic, so no
gyroscopic term); gravity g = (0, 0, -9.81); the contact forces are those of
the unmerged contact set (the energy's, whose derivatives a Newton step
uses); the particles' centres of mass are their body-frame origins.
"""
from __future__ import annotations

import numpy as np

from . import detect, forces

G_DEFAULT = np.array([0.0, 0.0, -9.81])


def bounding_radius(scene):
    """Largest body-frame vertex distance from the origin, per particle."""
    out = np.empty(scene.n_particles)
    for i in range(scene.n_particles):
        v, _ = scene.particle(i)
        out[i] = np.sqrt((v.astype(np.float64) ** 2).sum(1)).max()
    return out


def pair_eps(radius, i, j, eps_rel=0.01):
    """eps of a pair: eps_rel times the smaller diameter (Sec. 6 states eps
    relative to the particle diameter)."""
    return eps_rel * 2.0 * np.minimum(radius[i], radius[j])


def broad_phase(centres, bound, radius, eps_rel=0.01, chunk=2048):
    """All pairs i < j with |c_i - c_j| <= bound_i + bound_j + 2 eps_ij, by
    brute force over all pairs; sorted by (i, j)."""
    centres = np.asarray(centres, np.float64)
    n = len(centres)
    out_i, out_j = [], []
    for a in range(0, n, chunk):
        c = centres[a:a + chunk]
        d = np.sqrt(((c[:, None, :] - centres[None, :, :]) ** 2).sum(-1))
        ii = np.arange(a, a + len(c))[:, None]
        jj = np.arange(n)[None, :]
        lim = bound[ii] + bound[jj] + 2.0 * pair_eps(radius, ii, jj, eps_rel)
        sel = (jj > ii) & (d <= lim)
        i, j = np.nonzero(sel)
        out_i.append(i + a)
        out_j.append(j)
    i = np.concatenate(out_i) if out_i else np.zeros(0, np.int64)
    j = np.concatenate(out_j) if out_j else np.zeros(0, np.int64)
    o = np.lexsort((j, i))
    return np.stack([i[o], j[o]], 1).astype(np.int32)


def _quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def rotvec_quat(r):
    """Unit quaternion of the rotation by the rotation vector r."""
    th = float(np.linalg.norm(r))
    if th == 0.0:
        return np.array([1.0, 0.0, 0.0, 0.0])
    return np.concatenate([[np.cos(th / 2)], np.sin(th / 2) * np.asarray(r) / th])


def moved_poses(poses, vel, dt):
    """The step's geometry update: centre + dt v, orientation turned by
    dt omega in the world frame."""
    out = np.array(poses, np.float64, copy=True)
    for i in range(len(out)):
        out[i, :3] = poses[i, :3] + dt * vel[i, :3]
        q = _quat_mul(rotvec_quat(dt * vel[i, 3:]), poses[i, 3:] / np.linalg.norm(poses[i, 3:]))
        out[i, 3:] = q / np.linalg.norm(q)
    return out


def implicit_euler_step(scene, vel, pairs, eps, dt, g=G_DEFAULT, k_s=1000.0, tol=1e-13,
                        max_iter=200):
    """One implicit Euler step by Picard iteration (Algorithm 3).  scene:
    meshes, poses (step start), masses; vel [n, 6] (v, omega) at the start;
    pairs / eps: the candidate pairs and their eps.  Returns (poses, vel,
    iterations, history of the velocity change per iteration)."""
    import dataclasses
    n = scene.n_particles
    m = np.asarray(scene.mass, np.float64)
    inertia = 0.4 * m * np.asarray(scene.radius, np.float64) ** 2
    base = dataclasses.replace(scene, pairs=np.asarray(pairs, np.int32).reshape(-1, 2),
                               eps=np.asarray(eps, np.float64), com=np.zeros((n, 3)))
    v0 = np.asarray(vel, np.float64)
    guess = v0.copy()
    hist = []
    for it in range(1, max_iter + 1):
        poses = moved_poses(scene.poses, guess, dt)
        if base.n_pairs:
            c = detect(base, poses=poses)
            ft, _ = forces(base, c, k_s=k_s, poses=poses)
        else:
            ft = np.zeros((n, 6))
        new = np.empty_like(guess)
        new[:, :3] = v0[:, :3] + dt * (ft[:, :3] / m[:, None] + g)
        new[:, 3:] = v0[:, 3:] + dt * ft[:, 3:] / inertia[:, None]
        change = float(np.abs(new - guess).max())
        scale = float(np.abs(new).max()) + 1e-300
        hist.append(change / scale)
        guess = new
        if change <= tol * scale:
            break
    return moved_poses(scene.poses, guess, dt), guess, it, hist


def implicit_euler_step_newton(scene, vel, pairs, eps, dt, g=G_DEFAULT, k_s=1000.0, tol=1e-13,
                               max_iter=100, stiffness="gauss-newton"):
    """The same implicit Euler step solved by Newton's method in the
    velocities instead of Picard: residual
      r_i = M_i (V_i - V0_i) / dt - (F_i, tau_i)(geometry moved by dt V) - (m_i g, 0)
    (M = diag(m, m, m, I, I, I)), Jacobian approximated by M / dt + dt K with K
    the pairs' Gauss-Newton blocks sum e''(d) J J^T (the contact stiffness in
    the pose unknowns, barycentrics frozen).  The residual is exact, so the
    converged velocities are the implicit Euler solution; an approximate
    Jacobian only slows the convergence.  stiffness="hessian" uses the full
    pose Hessian (`pose_hessian`, closest points free) instead of the blocks,
    stiffness="analytic" the same Hessian in closed form (`contact_hessian`,
    in the form the differences see), "analytic-sym" its symmetric form.
    Each step is halved until the residual's largest entry drops
    (backtracking line search).  Returns (poses, vel, iterations)."""
    import dataclasses

    from . import grad
    n = scene.n_particles
    m = np.asarray(scene.mass, np.float64)
    inertia = 0.4 * m * np.asarray(scene.radius, np.float64) ** 2
    Mdiag = np.concatenate([np.repeat(m[:, None], 3, 1), np.repeat(inertia[:, None], 3, 1)], 1).ravel()
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    base = dataclasses.replace(scene, pairs=pairs, eps=np.asarray(eps, np.float64),
                               com=np.zeros((n, 3)))
    v0 = np.asarray(vel, np.float64)
    V = v0.copy()
    gext = np.zeros((n, 6))
    gext[:, :3] = m[:, None] * g

    def residual(V):
        poses = moved_poses(scene.poses, V, dt)
        c, ft = None, np.zeros((n, 6))
        if base.n_pairs:
            c = detect(base, poses=poses)
            ft, _ = forces(base, c, k_s=k_s, poses=poses)
        return (Mdiag * (V - v0).ravel()) / dt - ft.ravel() - gext.ravel(), poses, c

    def stiffness_matrix(poses, c):
        K = np.zeros((6 * n, 6 * n))
        if not base.n_pairs:
            return K
        if stiffness == "hessian":
            return pose_hessian(scene, poses, pairs, eps, k_s=k_s)
        if stiffness == "analytic-sym":
            return contact_hessian(base, c, poses=poses, k_s=k_s)
        if stiffness == "analytic":
            _, gp, _ = grad(base, c, k_s=k_s, poses=poses)
            return twist_hessian_fd_form(contact_hessian(base, c, poses=poses, k_s=k_s), gp)
        _, _, jac = grad(base, c, k_s=k_s, poses=poses)
        for p, (a, b) in enumerate(pairs):
            idx = np.r_[6 * a:6 * a + 6, 6 * b:6 * b + 6]
            K[np.ix_(idx, idx)] += jac[p]
        return K

    r, poses, c = residual(V)
    for it in range(1, max_iter + 1):
        scale = float(np.abs(Mdiag * V.ravel()).max()) / dt + 1e-300
        rn = float(np.abs(r).max())
        if rn <= tol * scale:
            break
        dV = np.linalg.solve(np.diag(Mdiag / dt) + dt * stiffness_matrix(poses, c), -r).reshape(n, 6)
        # backtracking: halve the step until the residual's largest entry
        # drops (the contact set and the closest features change between
        # iterates, so a full step can overshoot)
        lam = 1.0
        while True:
            rt, pt, ct = residual(V + lam * dV)
            if float(np.abs(rt).max()) < rn or lam < 2.0 ** -30:
                break
            lam *= 0.5
        V, r, poses, c = V + lam * dV, rt, pt, ct
    return moved_poses(scene.poses, V, dt), V, it


def twisted_pose(pose, k, h):
    """A pose moved by h along twist coordinate k: a world translation
    (k < 3) or a left rotation about the particle origin (k >= 3)."""
    p = np.array(pose, np.float64, copy=True)
    if k < 3:
        p[k] += h
        return p
    ax = np.zeros(3)
    ax[k - 3] = 1.0
    q = _quat_mul(rotvec_quat(h * ax), p[3:] / np.linalg.norm(p[3:]))
    p[3:] = q / np.linalg.norm(q)
    return p


def pose_hessian(scene, poses, pairs, eps, k_s=1000.0, h=1e-6):
    """Second derivatives of the contact energy in the particles' pose twists
    (translation, left rotation about the origin), [6n, 6n]: central
    differences of the analytic gradient dE/dpose (the oracle's `grad`), so
    the closest points are free to move (unlike the Gauss-Newton blocks,
    whose barycentrics are frozen).  Accurate to O(h^2) where the contact
    set and the closest features do not change within h."""
    import dataclasses

    from . import grad
    n = scene.n_particles
    base = dataclasses.replace(scene, pairs=np.asarray(pairs, np.int32).reshape(-1, 2),
                               eps=np.asarray(eps, np.float64), com=np.zeros((n, 3)))

    def gradient(P):
        c = detect(base, poses=P)
        return grad(base, c, k_s=k_s, poses=P)[1].ravel()

    H = np.zeros((6 * n, 6 * n))
    for i in range(n):
        for k in range(6):
            Pp, Pm = np.array(poses, copy=True), np.array(poses, copy=True)
            Pp[i] = twisted_pose(poses[i], k, h)
            Pm[i] = twisted_pose(poses[i], k, -h)
            H[:, 6 * i + k] = (gradient(Pp) - gradient(Pm)) / (2 * h)
    return H


def _barycentric(p, T):
    """Barycentric coordinates of p in triangle T [3, 3] (least squares in
    the triangle's plane)."""
    A = np.stack([T[1] - T[0], T[2] - T[0]], 1)
    s = np.linalg.lstsq(A, p - T[0], rcond=None)[0]
    return np.array([1.0 - s[0] - s[1], s[0], s[1]])


def _skew(r):
    return np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]], [-r[1], r[0], 0.0]])


def contact_hessian(scene, contacts, poses=None, k_s=1000.0, active_tol=1e-9):
    """Second derivatives of the contact energy E = sum_c e(d_c) (Sec. 2 force
    law, e(d) = K_s sqrt(mu) eps (1 - d/(2 eps))^2) in the particles' pose
    twists (world translation; world rotation increment theta about the
    particle's origin, applied on the left of R), [6n, 6n], symmetric, with
    the closest points free to move.

    Per contact with d > 0, from its closest points and their triangles:
      * the active features: the triangle corners with a barycentric weight
        of the closest point above active_tol (a vertex, an edge or the face
        of each triangle);
      * phi(X, s) = |P(s) - Q(s)|^2 / 2, X the six world corners, s the free
        barycentric parameters of the active features (none for a vertex,
        one for an edge, two for a face), P and Q linear in s and X; at the
        optimum grad_s phi = 0, so g(X) = min_s phi has grad g = phi_X and
        Hess g = phi_XX - phi_Xs phi_ss^-1 phi_sX (implicit function
        theorem); d = sqrt(2 g) gives grad d = grad g / d and
        Hess d = Hess g / d - grad g grad g^T / d^3;
      * Hess_X e = e''(d) grad d grad d^T + e'(d) Hess d, e' = -K_s sqrt(mu)
        (1 - d/(2 eps)), e'' = K_s sqrt(mu) / (2 eps);
      * to the twists: X_v(delta) = exp([theta]x)(X_v - t) + t + delta_t, so
        dX_v = [I, -[X_v - t]x] and the rotation block gains
        sum_v sym(g_v r_v^T) - (g_v . r_v) I with g_v = dE/dX_v and
        r_v = X_v - t (the second-order term of the exponential).
    Contacts at d = 0 (crossing triangles) are skipped: d is not
    differentiable there; so are contacts between parallel features (more
    than two free parameters: an edge lying on a face, two faces), where the
    closest points are not unique.  The central differences of the analytic gradient
    in `pose_hessian` move the rotation of the perturbed pose, which adds
    -1/2 [dE/dtheta]x to each particle's rotation block (the commutator of
    two rotations); `twist_hessian_fd_form` adds it."""
    from . import world_triangles
    poses = scene.poses if poses is None else poses
    n = scene.n_particles
    H = np.zeros((6 * n, 6 * n))
    tri_cache = {}

    def tris(i):
        if i not in tri_cache:
            tri_cache[i] = world_triangles(scene, i, poses)
        return tri_cache[i]

    for k in range(len(contacts["d"])):
        d = float(contacts["d"][k])
        if not d > 0.0:
            continue
        p = int(contacts["pair"][k])
        A, B = int(scene.pairs[p, 0]), int(scene.pairs[p, 1])
        eps = float(scene.eps[p])
        ks = k_s * np.sqrt(1.0 / (1.0 / scene.mass[A] + 1.0 / scene.mass[B]))
        TA = tris(A)[contacts["ta"][k]].reshape(3, 3)
        TB = tris(B)[contacts["tb"][k]].reshape(3, 3)
        X = np.concatenate([TA, TB])                       # [6, 3]
        wa = _barycentric(contacts["pa"][k], TA)
        wb = _barycentric(contacts["pb"][k], TB)
        SA = [i for i in range(3) if wa[i] > active_tol]
        SB = [i for i in range(3) if wb[i] > active_tol]
        sig = np.zeros(6)
        sig[SA] = wa[SA] / wa[SA].sum()
        sig[[3 + i for i in SB]] = -wb[SB] / wb[SB].sum()
        r = sig @ X                                         # P - Q
        # d sigma / d s for the free parameters
        dsig = []
        for j in SA[1:]:
            col = np.zeros(6)
            col[j], col[SA[0]] = 1.0, -1.0
            dsig.append(col)
        for j in SB[1:]:
            col = np.zeros(6)
            col[3 + j], col[3 + SB[0]] = -1.0, 1.0
            dsig.append(col)
        if len(dsig) > 2:
            continue   # parallel features (an edge on a face, two faces): not twice differentiable
        gg = np.kron(sig, r)                                # grad g, [18]
        Hg = np.kron(np.outer(sig, sig), np.eye(3))         # phi_XX
        if dsig:
            D = np.array(dsig)                              # [q, 6]
            G = D @ X                                       # [q, 3]: dr/ds
            M = np.zeros((18, len(dsig)))
            for q in range(len(dsig)):
                M[:, q] = np.kron(D[q], r) + np.kron(sig, G[q])
            Hg = Hg - M @ np.linalg.solve(G @ G.T, M.T)
        dd = gg / d
        Hd = Hg / d - np.outer(gg, gg) / d ** 3
        e1 = -ks * (1.0 - d / (2.0 * eps))
        e2 = ks / (2.0 * eps)
        HX = e2 * np.outer(dd, dd) + e1 * Hd
        gX = (e1 * dd).reshape(6, 3)
        # chain rule to the two particles' twists
        J = np.zeros((18, 12))
        R2 = np.zeros((12, 12))
        for v in range(6):
            blk, t = (0, poses[A, :3]) if v < 3 else (6, poses[B, :3])
            rv = X[v] - t
            J[3 * v:3 * v + 3, blk:blk + 3] = np.eye(3)
            J[3 * v:3 * v + 3, blk + 3:blk + 6] = -_skew(rv)
            gr = np.outer(gX[v], rv)
            R2[blk + 3:blk + 6, blk + 3:blk + 6] += 0.5 * (gr + gr.T) - (gX[v] @ rv) * np.eye(3)
        H12 = J.T @ HX @ J + R2
        idx = np.r_[6 * A:6 * A + 6, 6 * B:6 * B + 6]
        H[np.ix_(idx, idx)] += H12
    return H


def twist_hessian_fd_form(H, grad_pose):
    """The Hessian as `pose_hessian`'s central differences see it: each
    particle's rotation block plus -1/2 [dE/dtheta]x (differentiating the
    twist gradient while the pose itself rotates)."""
    out = np.array(H, copy=True)
    for i in range(len(grad_pose)):
        out[6 * i + 3:6 * i + 6, 6 * i + 3:6 * i + 6] -= 0.5 * _skew(grad_pose[i, 3:])
    return out
