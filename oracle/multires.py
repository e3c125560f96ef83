"""FP64 CPU oracle of the multiresolution implicit Euler step (Algorithm 6).
Test infrastructure only: the tests and bench.py's CPU-baseline leg use it;
the product path never does.

Algorithm 6 interleaves the Picard loop of Algorithm 3 with the unfolding of
the surrogate trees: every particle pair keeps an active set across the
Picard iterations; each iteration tests the active set at the guessed
geometry, widens it where a surrogate comparison did not rule out contact,
narrows it where a group of children certainly contributes nothing, and
uses the contacts found on surrogate levels as an implicit guess (with
reduced weight) until the trees are unfolded where contacts are.

The active set of a pair is written here as a cut through the product of the
two trees: a list of node pairs (a, b) such that every pair of fine
triangles lies below exactly one listed pair, in depth-first order of the
product tree (the children of a pair follow each other, A's child index
major).  The product tree is the one Algorithm 5 unfolds: the children of
(a, b) are (a_i, b_j) over the children of both sides, a leaf side staying
as it is while the other unfolds.  Per item and iteration (exact FP64
distances of the world-frame surrogate triangles):
  - bottom (the paper's contact-free outcome): distance > delta_a + delta_b
    + 2 eps; by conservativeness no fine pair below it is a contact;
  - a pair of leaves that is not bottom: its fine triangle pairs are compared
    exactly and those within 2 eps are the iteration's fine contacts;
  - any other pair that is not bottom: a surrogate contact (threshold
    tau = delta_a + delta_b + 2 eps in place of 2 eps), and the item is
    widened: replaced by its children for the next iteration.
Narrowing: when all children of a pair are listed next to each other and
all are bottom, they are replaced by the pair ("If all children of a
surrogate triangle do certainly not contribute a contact point anymore,
they are replaced with their parent").  The memory set U is kept as two
flags on the items: a pair made by narrowing carries N; the children of a
widened item carrying N or V carry V; a group with a V member is never
narrowed (removal vetoed once re-added).  The iteration stops when the
Picard criterion holds and the iteration neither widened nor narrowed
anything (no tree node unfolded and the active sets did not change).  At
that point no surrogate pair is in contact, every fine contact lies below a
listed pair of leaves and was found, and the velocities are the plain
implicit Euler step's fixed point (the paper's correctness lemma for
Algorithm 6).

Surrogate contact forces: the force law of Sec. 2 with tau in place of 2 eps,
times the weight w (the paper damps coarse-level contributions without a
value; w = 1/4 here): F = w k_s sqrt(mu) (1 - d / tau) u, u = (p_a - p_b)/d,
or minus A's surrogate normal when the surrogates cross, applied at
(p_a + p_b)/2, torques about the body origins.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import forces, pose_matrix, tri_pairs, tri_tri
from .implicit import G_DEFAULT, moved_poses

V_BIT = 1          # removal vetoed (the memory set U)
N_BIT = 2          # made by narrowing
BOT, LEAF, WIDEN = 0, 1, 2


class Trees:
    """The surrogate trees of all particles as plain arrays (a hierarchy's
    export: node_tri, node_delta, node_child, node_level, root, slot_tri)."""

    def __init__(self, ex):
        self.tri = np.asarray(ex["node_tri"], np.float64).reshape(-1, 3, 3)
        self.delta = np.asarray(ex["node_delta"], np.float64)
        self.child = np.asarray(ex["node_child"], np.int64).reshape(-1, 2)
        self.level = np.asarray(ex["node_level"], np.int64)
        self.root = np.asarray(ex["root"], np.int64)
        self.slot_tri = np.asarray(ex["slot_tri"], np.int64)
        n = len(self.delta)
        self.parent = np.full(n, -1, np.int64)
        self.particle = np.full(n, -1, np.int64)
        for i, r in enumerate(self.root):
            stack = [int(r)]
            while stack:
                v = stack.pop()
                self.particle[v] = i
                b, c = self.child[v]
                if c > 0:
                    self.parent[b:b + c] = v
                    stack.extend(range(b, b + c))

    def leaf(self, v):
        return self.child[v, 1] < 0

    def leaf_tris(self, v):
        b, c = self.child[v]
        t = self.slot_tri[b:b - c]
        return t[t >= 0]

    def sides(self, v):
        """The child set of v as one side of a pair: its children, or v itself
        when v is a leaf."""
        b, c = self.child[v]
        return list(range(b, b + c)) if c > 0 else [int(v)]

    def children(self, a, b):
        return [(x, y) for x in self.sides(a) for y in self.sides(b)]

    def parent_pair(self, a, b):
        """The pair whose unfolding made (a, b), or None for the root pair: the
        sides on the deeper level came from their parents, a shallower side
        (a leaf) stayed."""
        k = max(self.level[a], self.level[b])
        pa = int(self.parent[a]) if self.level[a] == k else int(a)
        pb = int(self.parent[b]) if self.level[b] == k else int(b)
        if pa < 0 or pb < 0:
            return None
        return pa, pb

    def child_index(self, a, b, par):
        """(position of (a, b) among the children of par, number of children)."""
        sa, sb = self.sides(par[0]), self.sides(par[1])
        return sa.index(a) * len(sb) + sb.index(b), len(sa) * len(sb)


def initial_frontier(trees, pairs):
    """One item per pair: the two roots."""
    return [(p, int(trees.root[A]), int(trees.root[B]), 0) for p, (A, B) in enumerate(pairs)]


def _world(trees, v, R, t):
    return trees.tri[v] @ R.T + t


def frontier_test(scene, trees, poses, pairs, eps, frontier):
    """Outcome of every item at the given poses.  Returns (status list, fine
    contacts sorted by (pair, ta, tb) like the oracle's detect, surrogate
    contacts as a dict of arrays: item, pair, a, b, d, pa, pb, tau, n (A's
    world surrogate normal))."""
    Rs = [pose_matrix(q) for q in poses]
    n = len(frontier)
    P = np.empty((n, 9))
    Q = np.empty((n, 9))
    tau = np.empty(n)
    for k, (p, a, b, _) in enumerate(frontier):
        A, B = pairs[p]
        P[k] = _world(trees, a, Rs[A], poses[A][:3]).ravel()
        Q[k] = _world(trees, b, Rs[B], poses[B][:3]).ravel()
        tau[k] = trees.delta[a] + trees.delta[b] + 2.0 * eps[p]
    if n:
        d, pa, pb, _ = tri_tri(P, Q)
    else:
        d = np.zeros(0)
        pa = pb = np.zeros((0, 3))
    status = []
    abt, owner = [], []
    sur = dict(item=[], pair=[], a=[], b=[], d=[], pa=[], pb=[], tau=[], n=[])
    for k, (p, a, b, _) in enumerate(frontier):
        if d[k] > tau[k]:
            status.append(BOT)
        elif trees.leaf(a) and trees.leaf(b):
            status.append(LEAF)
            A, B = pairs[p]
            ta, tb = trees.leaf_tris(a), trees.leaf_tris(b)
            for x in ta:
                for y in tb:
                    abt.append((A, x, B, y))
                    owner.append(p)
        else:
            status.append(WIDEN)
            T = P[k].reshape(3, 3)
            nrm = np.cross(T[1] - T[0], T[2] - T[0])
            for key, val in (("item", k), ("pair", p), ("a", a), ("b", b), ("d", d[k]),
                             ("pa", pa[k]), ("pb", pb[k]), ("tau", tau[k]), ("n", nrm)):
                sur[key].append(val)
    sur = {k: np.asarray(v) for k, v in sur.items()}
    fine = dict(pair=np.zeros(0, np.int32), ta=np.zeros(0, np.int32), tb=np.zeros(0, np.int32),
                d=np.zeros(0), pa=np.zeros((0, 3)), pb=np.zeros((0, 3)))
    if abt:
        abt = np.asarray(abt, np.int32)
        owner = np.asarray(owner, np.int32)
        fd, fpa, fpb, _ = tri_pairs(scene, abt, poses=poses)
        keep = fd <= 2.0 * np.asarray(eps)[owner]
        fine = dict(pair=owner[keep], ta=abt[keep, 1], tb=abt[keep, 3], d=fd[keep],
                    pa=fpa[keep], pb=fpb[keep])
        o = np.lexsort((fine["tb"], fine["ta"], fine["pair"]))
        fine = {k: v[o] for k, v in fine.items()}
    return status, fine, sur


def frontier_update(trees, frontier, status):
    """The next active sets: widened items replaced by their children,
    complete all-bottom sibling groups without a vetoed member replaced by
    their parent (flag N), everything else kept.  Returns (frontier, number
    of widened items, number of narrowed groups)."""
    n = len(frontier)
    mark = [0] * n     # 1: emits the group's parent, 2: dropped into it
    parent = [None] * n
    for i, (p, a, b, fl) in enumerate(frontier):
        if status[i] != BOT or fl & V_BIT:
            continue
        par = trees.parent_pair(a, b)
        if par is None:
            continue
        c, size = trees.child_index(a, b, par)
        if c != 0 or i + size > n:
            continue
        ok = True
        for k in range(size):
            p2, a2, b2, f2 = frontier[i + k]
            if (p2 != p or status[i + k] != BOT or f2 & V_BIT
                    or trees.parent_pair(a2, b2) != par
                    or trees.child_index(a2, b2, par)[0] != k):
                ok = False
                break
        if ok:
            mark[i] = 1
            parent[i] = par
            for k in range(1, size):
                mark[i + k] = 2
    out = []
    widened = narrowed = 0
    for i, (p, a, b, fl) in enumerate(frontier):
        if mark[i] == 1:
            out.append((p, parent[i][0], parent[i][1], N_BIT))
            narrowed += 1
        elif mark[i] == 2:
            continue
        elif status[i] == WIDEN:
            widened += 1
            cf = V_BIT if fl & (N_BIT | V_BIT) else 0
            out.extend((p, x, y, cf) for x, y in trees.children(a, b))
        else:
            out.append((p, a, b, fl))
    return out, widened, narrowed


def surrogate_forces(scene, pairs, eps, poses, sur, weight=0.25, k_s=1000.0):
    """Forces and torques [n, 6] (about the body origins) and energy of the
    surrogate contacts."""
    ft = np.zeros((scene.n_particles, 6))
    en = 0.0
    m = np.asarray(scene.mass, np.float64)
    for k in range(len(sur.get("d", []))):
        p = int(sur["pair"][k])
        A, B = pairs[p]
        mu = 1.0 / (1.0 / m[A] + 1.0 / m[B])
        ks = weight * k_s * np.sqrt(mu)
        d, tau = float(sur["d"][k]), float(sur["tau"][k])
        pa, pb = sur["pa"][k], sur["pb"][k]
        if d > 0.0:
            u = (pa - pb) / d
        else:
            u = -sur["n"][k] / np.linalg.norm(sur["n"][k])
        F = ks * (1.0 - d / tau) * u
        xc = 0.5 * (pa + pb)
        ft[A, :3] += F
        ft[A, 3:] += np.cross(xc - poses[A][:3], F)
        ft[B, :3] -= F
        ft[B, 3:] += np.cross(xc - poses[B][:3], -F)
        s = 1.0 - d / tau
        en += ks * 0.5 * tau * s * s
    return ft, en


def multires_implicit_euler_step(scene, trees, vel, pairs, eps, dt, g=G_DEFAULT, k_s=1000.0,
                                 weight=0.25, tol=1e-13, max_iter=200):
    """One implicit Euler step by the multiresolution Picard iteration of
    Algorithm 6 (module docstring).  Returns (poses, vel, iterations,
    history of the relative velocity change, per-iteration record: frontier
    size, widened, narrowed, fine and surrogate contacts)."""
    n = scene.n_particles
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    eps = np.asarray(eps, np.float64)
    m = np.asarray(scene.mass, np.float64)
    inertia = 0.4 * m * np.asarray(scene.radius, np.float64) ** 2
    base = dataclasses.replace(scene, pairs=pairs, eps=eps, com=np.zeros((n, 3)))
    v0 = np.asarray(vel, np.float64)
    guess = v0.copy()
    frontier = initial_frontier(trees, pairs)
    hist, record = [], []
    it = 0
    for it in range(1, max_iter + 1):
        poses = moved_poses(scene.poses, guess, dt)
        status, fine, sur = frontier_test(scene, trees, poses, pairs, eps, frontier)
        ft = np.zeros((n, 6))
        if len(fine["d"]):
            ft, _ = forces(base, fine, k_s=k_s, poses=poses)
        fs, _ = surrogate_forces(scene, pairs, eps, poses, sur, weight, k_s)
        ft = ft + fs
        new = np.empty_like(guess)
        new[:, :3] = v0[:, :3] + dt * (ft[:, :3] / m[:, None] + g)
        new[:, 3:] = v0[:, 3:] + dt * ft[:, 3:] / inertia[:, None]
        change = float(np.abs(new - guess).max())
        scale = float(np.abs(new).max()) + 1e-300
        frontier, widened, narrowed = frontier_update(trees, frontier, status)
        hist.append(change / scale)
        record.append(dict(items=len(status), widened=widened, narrowed=narrowed,
                           fine=len(fine["d"]), surrogate=len(sur.get("d", []))))
        guess = new
        if change <= tol * scale and widened == 0 and narrowed == 0:
            break
    return moved_poses(scene.poses, guess, dt), guess, it, hist, record
