"""Work counts of the multiresolution detection (Algorithm 5), the set-based
form against the pair-list form this library implements, and the brute force
(comparison-based method on every triangle pair), on the CPU: an analogue of
the paper's tables of triangle comparisons (Sec. 6).

Run (not collected by pytest):

    python tests/work_counts_report.py [out.md]

Both forms use the same FP64 surrogate test, the exact distance of the two
triangles (surrogate or fine) against delta_a + delta_b + 2 eps (delta = 0
for a fine triangle), so they differ only in which triangle pairs they test:
  * pair lists: a surviving pair unfolds into the children of its surrogate
    side(s) (a fine side stays), leaf against leaf into the fine pairs;
  * set-based (Algorithm 5 as printed): per round, every triangle of A's
    active set against every triangle of B's; a triangle that passes against
    any counterpart enters the next round (a surrogate by its children, a
    fine triangle as itself); the rounds end when both sets hold fine
    triangles only.
Both end with the same contact set (the brute force's).  The hybrid column
counts, of the fine pairs that the pair lists test, how many the FP64
penalty sweep (Eq. 3/4, four iterations, the library's default constants)
leaves unconverged (the paper's odot, which falls back to the
comparison-based method).  Uses the oracle's distance and sweep and the
library's host-built trees (the trees are what is counted).
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


class Tree:
    """World-frame view of one particle's tree: items are ('n', node) for a
    surrogate and ('t', slot) for a fine triangle."""

    def __init__(self, ex, scene, orc, i, pose):
        self.ex, self.i = ex, i
        R = orc.pose_matrix(pose)
        self.node_w = ex["node_tri"].reshape(-1, 3, 3).astype(np.float64) @ R.T + pose[:3]
        v, t = scene.particle(i)
        self.fine_w = (v.astype(np.float64) @ R.T + pose[:3])[t]   # [n_tri, 3, 3]

    def tri(self, item):
        kind, k = item
        if kind == "n":
            return self.node_w[k].ravel()
        return self.fine_w[self.ex["slot_tri"][k]].ravel()

    def delta(self, item):
        return float(self.ex["node_delta"][item[1]]) if item[0] == "n" else 0.0

    def children(self, item):
        if item[0] == "t":
            return [item]
        b, c = self.ex["node_child"][item[1]]
        if c < 0:
            return [("t", s) for s in range(b, b - c)]
        return [("n", k) for k in range(b, b + c)]

    def root(self):
        return ("n", int(self.ex["root"][self.i]))


def _passes(orc, TA, TB, pairs, eps):
    if not pairs:
        return np.zeros(0, bool), np.zeros(0)
    P = np.array([TA.tri(a) for a, _ in pairs])
    Q = np.array([TB.tri(b) for _, b in pairs])
    d = orc.tri_tri(P, Q)[0]
    lim = np.array([TA.delta(a) + TB.delta(b) for a, b in pairs]) + 2 * eps
    return d <= lim, d


def pair_list_counts(orc, TA, TB, eps):
    work = [(TA.root(), TB.root())]
    tests, fine_tests, contacts, fine_pairs = 0, 0, 0, []
    while work:
        ok, _ = _passes(orc, TA, TB, work, eps)
        tests += len(work)
        nxt = []
        for (a, b), p in zip(work, ok):
            if a[0] == "t" and b[0] == "t":
                fine_tests += 1
                fine_pairs.append((a, b))
                contacts += int(p)
                continue
            if p:
                nxt += [(x, y) for x in TA.children(a) for y in TB.children(b)]
        work = nxt
    return tests, fine_tests, contacts, fine_pairs


def set_based_counts(orc, TA, TB, eps):
    SA, SB = [TA.root()], [TB.root()]
    tests, rounds = 0, 0
    while True:
        pairs = [(a, b) for a in SA for b in SB]
        ok, _ = _passes(orc, TA, TB, pairs, eps)
        tests += len(pairs)
        rounds += 1
        final = all(a[0] == "t" for a in SA) and all(b[0] == "t" for b in SB)
        if final:
            return tests, rounds, int(ok.sum())
        ma = sorted({a for (a, _), p in zip(pairs, ok) if p})
        mb = sorted({b for (_, b), p in zip(pairs, ok) if p})
        SA = sorted({c for a in ma for c in TA.children(a)})
        SB = sorted({c for b in mb for c in TB.children(b)})
        if not SA or not SB:
            return tests, rounds, 0


def main(out_path=None):
    import oracle
    import paper_2105_12415_gb300 as m
    from gen import scene_c1, scene_c2
    oracle.build()
    p = m.default_params()
    rows = []
    c2 = scene_c2()
    ntri = np.diff(c2.tri_off)
    sizes = ntri[c2.pairs[:, 0]] * ntri[c2.pairs[:, 1]]
    order = np.argsort(sizes)
    picks = [int(order[int(q * (len(order) - 1))]) for q in (0.2, 0.5, 0.7, 0.85, 0.95)]
    work = [("one pair (c1), 1280 x 1280", scene_c1(), 0)]
    for k in picks:
        work.append((f"batched pair {k}, {ntri[c2.pairs[k, 0]]} x {ntri[c2.pairs[k, 1]]}",
                     c2.subset(np.array([k])), 0))
    for name, s, pi in work:
        h = m.Hierarchy.build_host(s.vert_off, s.verts, s.tri_off, s.tris, p)
        ex = h.export()
        a, b = s.pairs[pi]
        TA, TB = Tree(ex, s, oracle, a, s.poses[a]), Tree(ex, s, oracle, b, s.poses[b])
        eps = float(s.eps[pi])
        pl_tests, fine_tests, contacts, fine_pairs = pair_list_counts(oracle, TA, TB, eps)
        sb_tests, rounds, sb_contacts = set_based_counts(oracle, TA, TB, eps)
        ref = oracle.detect(s)
        assert contacts == sb_contacts == len(ref["d"]), (contacts, sb_contacts, len(ref["d"]))
        P = np.array([TA.tri(x) for x, _ in fine_pairs]).reshape(-1, 9)
        Q = np.array([TB.tri(y) for _, y in fine_pairs]).reshape(-1, 9)
        sw = oracle.sweep(P, Q, eps, n_iter=p.n_iter, rho_reg=p.rho_reg, rho_iter=p.rho_iter,
                          conv_c=p.conv_c) if len(P) else {"converged": np.zeros(0, bool)}
        unconv = int((~sw["converged"]).sum())
        brute = int(np.diff(s.tri_off)[a] * np.diff(s.tri_off)[b])
        rows.append(dict(workload=name, brute=brute, pair_list=pl_tests, fine=fine_tests,
                         set_based=sb_tests, rounds=rounds, contacts=contacts, odot=unconv))
        print(rows[-1], flush=True)
    cols = ["workload", "brute", "pair_list", "fine", "set_based", "rounds", "contacts", "odot"]
    head = ["workload", "brute force (all triangle pairs)", "pair lists: tests", "of which fine",
            "set-based: tests", "set-based rounds", "contacts", "sweep unconverged (odot)"]
    lines = ["| " + " | ".join(head) + " |", "|" + "---|" * len(head)]
    for r in rows:
        lines.append("| " + " | ".join(str(r[c]) for c in cols) + " |")
    text = "\n".join(lines) + "\n"
    print(text)
    if out_path:
        how = __doc__[:__doc__.index("Run (not")].strip()
        rule = __doc__[__doc__.index("Both forms"):].strip()
        with open(out_path, "w") as f:
            f.write("# Work counts: pair lists, set-based Algorithm 5, brute force\n\n"
                    f"{how}\n\nCommand: `python tests/work_counts_report.py {out_path}` "
                    "(CPU only)\n\n" + rule + "\n\n" + text)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
