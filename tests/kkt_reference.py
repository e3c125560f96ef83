"""Independent second implementation of the triangle-triangle distance used to
pin the oracle: enumerate every pair of faces (3 vertices, 3 edges, interior
of each triangle), solve the unconstrained least-squares problem on the two
affine hulls, keep the solutions whose barycentric weights are all >= 0 and
return the smallest distance.  The distance between two triangles is a convex
problem whose minimiser lies in the relative interior of some face pair, where
it is a stationary point of that face pair's hull problem (the KKT
conditions), so the enumeration is exact; crossing triangles appear as an
edge-interior pair with distance 0.  Pure numpy, shares nothing with the
oracle."""
import itertools

import numpy as np

FACES = [(0,), (1,), (2,), (0, 1), (1, 2), (0, 2), (0, 1, 2)]


def kkt_distance(P, Q, tol=1e-9):
    P = np.asarray(P, np.float64).reshape(-1, 3, 3)
    Q = np.asarray(Q, np.float64).reshape(-1, 3, 3)
    n = len(P)
    best = np.full(n, np.inf)
    for fa, fb in itertools.product(FACES, FACES):
        A = P[:, list(fa)]
        B = Q[:, list(fb)]
        a0, b0 = A[:, 0], B[:, 0]
        cols = [A[:, i] - a0 for i in range(1, len(fa))] + [-(B[:, j] - b0) for j in range(1, len(fb))]
        if cols:
            M = np.stack(cols, axis=2)                      # n x 3 x m
            rhs = b0 - a0
            sol = np.einsum("nij,nj->ni", np.linalg.pinv(M), rhs)
            k = len(fa) - 1
            lam = np.concatenate([1 - sol[:, :k].sum(1, keepdims=True), sol[:, :k]], 1)
            mu = np.concatenate([1 - sol[:, k:].sum(1, keepdims=True), sol[:, k:]], 1)
            x = np.einsum("ni,nij->nj", lam, A)
            y = np.einsum("ni,nij->nj", mu, B)
            ok = (lam >= -tol).all(1) & (mu >= -tol).all(1)
        else:
            x, y = a0, b0
            ok = np.ones(n, bool)
        d = np.linalg.norm(x - y, axis=1)
        best = np.where(ok & (d < best), d, best)
    return best


def grid_distance(P, Q, m=40):
    """Upper bound by sampling both triangles on a barycentric grid."""
    P = np.asarray(P, np.float64).reshape(3, 3)
    Q = np.asarray(Q, np.float64).reshape(3, 3)
    w = [(i / m, j / m) for i in range(m + 1) for j in range(m + 1 - i)]
    w = np.array([(1 - a - b, a, b) for a, b in w])
    X, Y = w @ P, w @ Q
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    return float(np.sqrt(d2.min()))
