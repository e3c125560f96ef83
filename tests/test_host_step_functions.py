"""The implicit step's device functions (csrc/mrdem_step.cuh) built for the
host and checked against the FP64 oracle: the broad phase driven through the
same steps as its kernels (with the buckets' particles scattered in shuffled
order, as the kernel's atomics may), the pose update, the Picard velocity
update and the per-contact Hessian block.  These are the functions the
kernels of mrdem_step.cu run; the GPU tests check the kernels themselves."""
import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np
import pytest

from gen import scene_packing

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2105_12415_gb300", "csrc")
DP = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def hs(tmp_path_factory):
    so = tmp_path_factory.mktemp("hs") / "libhs.so"
    # no contraction into fused multiply-adds: the kernels round the
    # decisive operations one by one
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC",
                           "-I", CSRC, os.path.join(ROOT, "tests", "host_step_harness.cpp"),
                           "-o", str(so)])
    lib = C.CDLL(str(so))
    lib.hs_broad_phase.restype = C.c_longlong
    lib.hs_broad_phase.argtypes = [C.c_int, DP, DP, DP, C.c_double, C.POINTER(C.c_int), DP,
                                   C.c_longlong, C.c_uint]
    lib.hs_move_poses.argtypes = [C.c_int, DP, DP, C.c_double, DP]
    lib.hs_contact_hessian.argtypes = [DP, DP, DP, DP, C.c_double, C.c_double, DP]
    lib.hs_picard.argtypes = [C.c_int, DP, DP, DP, DP, DP, C.c_double, DP, DP]
    lib.hs_particle_motion.restype = C.c_double
    lib.hs_particle_motion.argtypes = [DP, DP, C.c_double]
    lib.hs_newton_residual.argtypes = [C.c_int, DP, DP, DP, DP, DP, DP, C.c_double, DP, DP]
    return lib


@pytest.fixture(scope="module")
def imp(orc):
    import oracle.implicit as imp
    return imp


def _d(a):
    return np.ascontiguousarray(a, np.float64)


def _broad(hs, poses, bound, radius, shuffle=0, eps_rel=0.01):
    P, B, R = _d(poses), _d(bound), _d(radius)
    cap = 64 * len(B) + 64
    pairs = np.zeros((cap, 2), np.int32)
    eps = np.zeros(cap)
    total = hs.hs_broad_phase(len(B), P.ctypes.data_as(DP), B.ctypes.data_as(DP),
                              R.ctypes.data_as(DP), eps_rel,
                              pairs.ctypes.data_as(C.POINTER(C.c_int)), eps.ctypes.data_as(DP),
                              cap, shuffle)
    assert total <= cap
    return pairs[:total], eps[:total]


def _bound(s):
    return np.array([np.sqrt((s.particle(i)[0].astype(np.float64) ** 2).sum(1)).max()
                     for i in range(s.n_particles)])


@pytest.mark.parametrize("n,fraction,levels,seed", [(300, 0.35, (1, 2), 1), (2000, 0.5, (1,), 2),
                                                    (50, 0.55, (1, 2), 3)])
def test_broad_phase_functions_equal_oracle(hs, imp, n, fraction, levels, seed):
    s, _, _ = scene_packing(n, fraction, levels=levels, r_min=1.0, r_max=10.0, seed=seed)
    bound = _bound(s)
    ref = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    assert len(ref) > n // 10
    for shuffle in (0, 7, 1234):
        pairs, eps = _broad(hs, s.poses, bound, s.radius, shuffle)
        assert np.array_equal(pairs, ref)
        assert np.array_equal(eps, imp.pair_eps(s.radius, ref[:, 0], ref[:, 1]))


def test_broad_phase_functions_edge_cases(hs, imp):
    P = np.zeros((5, 7))
    P[:, 3] = 1.0
    pairs, eps = _broad(hs, P, np.zeros(5), np.zeros(5))
    assert pairs.tolist() == [[i, j] for i in range(5) for j in range(i + 1, 5)]
    rng = np.random.default_rng(0)
    P = np.zeros((42, 7))
    P[:, 3] = 1.0
    P[:20, :3] = rng.normal(size=(20, 3))
    P[20:40, :3] = 1e12 + rng.normal(size=(20, 3))   # cell coordinates clamped
    P[40, :3] = (5.0, 5.0, 5.0)
    P[41, :3] = (5.0, 5.0, 6.02)                     # at the limit distance
    b = np.full(42, 0.5)
    pairs, _ = _broad(hs, P, b, b, shuffle=3)
    assert np.array_equal(pairs, imp.broad_phase(P[:, :3], b, b))


def test_pose_update_function_equals_oracle(hs, imp):
    s, _, _ = scene_packing(200, 0.3, levels=(1,), seed=5)
    V = np.random.default_rng(7).normal(size=(200, 6)) * 3.0
    V[0, 3:] = 0.0
    for dt in (1e-3, 0.5):
        out = np.zeros((200, 7))
        hs.hs_move_poses(200, _d(s.poses).ctypes.data_as(DP), _d(V).ctypes.data_as(DP), dt,
                         out.ctypes.data_as(DP))
        ref = imp.moved_poses(s.poses, V, dt)
        assert np.abs(out - ref).max() <= 1e-14 * (1.0 + np.abs(ref).max())


def test_picard_function_rounds_like_the_formula(hs):
    rng = np.random.default_rng(8)
    n = 1000
    v0, guess, ft = rng.normal(size=(n, 6)), rng.normal(size=(n, 6)), rng.normal(size=(n, 6)) * 100
    mass, inertia = rng.uniform(0.5, 2.0, n), rng.uniform(0.1, 1.0, n)
    g = np.array([0.5, -1.0, -9.81])
    dt = 1e-3
    vel, norms = guess.copy(), np.zeros(2)
    hs.hs_picard(n, _d(v0).ctypes.data_as(DP), _d(ft).ctypes.data_as(DP), _d(mass).ctypes.data_as(DP),
                 _d(inertia).ctypes.data_as(DP), _d(g).ctypes.data_as(DP), dt,
                 vel.ctypes.data_as(DP), norms.ctypes.data_as(DP))
    want = np.empty((n, 6))
    want[:, :3] = v0[:, :3] + dt * (ft[:, :3] / mass[:, None] + g)
    want[:, 3:] = v0[:, 3:] + dt * ft[:, 3:] / inertia[:, None]
    assert np.array_equal(vel, want)
    assert norms[0] == np.abs(want - guess).max() and norms[1] == np.abs(want).max()


def test_hessian_block_function_equals_oracle(hs, imp, orc):
    """Per contact, the compact block of the kernel (Z, N and the
    exponential map's term) equals the oracle's elimination over the six
    corners, on every generic feature pair."""
    from tests.test_oracle_implicit import FACING, _colliding_pair, _icosahedra_facing, _one_contact
    scenes = [_icosahedra_facing(a, b) for a, b in FACING]
    for seed in (4, 8, 11):
        s, _, pairs, eps = _colliding_pair(imp, seed=seed)
        scenes.append(dataclasses.replace(s, pairs=pairs, eps=eps, com=np.zeros((2, 3))))
    n_checked = 0
    for s in scenes:
        c = orc.detect(s)
        TA, TB = orc.world_triangles(s, 0), orc.world_triangles(s, 1)
        ks = 1000.0 * np.sqrt(s.mass[0] * s.mass[1] / (s.mass[0] + s.mass[1]))
        for k in range(len(c["d"])):
            out = np.zeros(144)
            st = hs.hs_contact_hessian(_d(TA[c["ta"][k]]).ctypes.data_as(DP),
                                       _d(TB[c["tb"][k]]).ctypes.data_as(DP),
                                       _d(s.poses[0, :3]).ctypes.data_as(DP),
                                       _d(s.poses[1, :3]).ctypes.data_as(DP), ks, float(s.eps[0]),
                                       out.ctypes.data_as(DP))
            assert st == 0
            ref = imp.contact_hessian(s, _one_contact(c, k))
            assert np.abs(out.reshape(12, 12) - ref).max() <= 1e-12 * np.abs(ref).max()
            n_checked += 1
    assert n_checked > 100
    # crossing triangles: skipped (d = 0)
    T = np.array([0.0, 0, 0, 1, 0, 0, 0, 1, 0])
    U = np.array([0.2, 0.2, -0.5, 0.2, 0.2, 0.5, 0.9, 0.9, 0.0])
    out = np.zeros(144)
    z = np.zeros(3)
    assert hs.hs_contact_hessian(_d(T).ctypes.data_as(DP), _d(U).ctypes.data_as(DP),
                                 _d(z).ctypes.data_as(DP), _d(z).ctypes.data_as(DP), 1.0, 0.1,
                                 out.ctypes.data_as(DP)) == 1
    assert (out == 0).all()


def test_newton_residual_function_rounds_like_the_formula(hs):
    rng = np.random.default_rng(11)
    n = 500
    v0, v, ft = rng.normal(size=(n, 6)), rng.normal(size=(n, 6)), rng.normal(size=(n, 6)) * 50
    mass, inertia = rng.uniform(0.5, 2.0, n), rng.uniform(0.1, 1.0, n)
    g, dt = np.array([0.3, 0.0, -9.81]), 1e-3
    res, norms = np.zeros((n, 6)), np.zeros(2)
    hs.hs_newton_residual(n, *[_d(a).ctypes.data_as(DP) for a in (v0, v, ft, mass, inertia, g)], dt,
                          res.ctypes.data_as(DP), norms.ctypes.data_as(DP))
    Md = np.concatenate([np.repeat(mass[:, None], 3, 1), np.repeat(inertia[:, None], 3, 1)], 1)
    gext = np.zeros((n, 6))
    gext[:, :3] = mass[:, None] * g
    want = (Md * (v - v0)) / dt - ft - gext
    assert np.array_equal(res, want)
    assert norms[0] == np.abs(want).max() and norms[1] == np.abs(Md * v).max() / dt


def test_particle_motion_function(hs, imp):
    """|dt| + angle R, with the angle of the relative rotation, against the
    largest displacement of sampled points of the bounding sphere (which it
    bounds, and nearly reaches for the farthest point)."""
    rng = np.random.default_rng(14)
    for _ in range(200):
        a = np.concatenate([rng.normal(size=3), rng.normal(size=4)])
        b = a.copy()
        b[:3] += rng.normal(size=3) * rng.uniform(0, 0.1)
        r = rng.normal(size=3) * rng.uniform(0, 0.5)
        b[3:] = imp._quat_mul(imp.rotvec_quat(r), a[3:] / np.linalg.norm(a[3:])) * rng.uniform(0.5, 2)
        R = rng.uniform(0.1, 3.0)
        got = hs.hs_particle_motion(_d(a).ctypes.data_as(DP), _d(b).ctypes.data_as(DP), R)
        want = np.linalg.norm(b[:3] - a[:3]) + np.linalg.norm(r) * R
        assert abs(got - want) <= 1e-12 * (1 + want)
        # it bounds every point's displacement
        x = rng.normal(size=(64, 3))
        x = R * x / np.linalg.norm(x, axis=1, keepdims=True)
        Ra = orc_matrix(a[3:])
        Rb = orc_matrix(b[3:])
        disp = np.linalg.norm((x @ Rb.T + b[:3]) - (x @ Ra.T + a[:3]), axis=1).max()
        assert disp <= got * (1 + 1e-12)


def orc_matrix(q):
    q = np.asarray(q, np.float64) / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_broad_phase_functions_with_size_disparity(hs, imp):
    """Big particles (radius 20) among small ones (radius 1): the size
    classes give the oracle's list bit for bit."""
    from gen.icosphere import scene_scale
    s, _ = scene_scale(n_small=3000, n_big=4, fraction=0.2)
    bound = _bound(s)
    ref = imp.broad_phase(s.poses[:, :3], bound, s.radius)
    assert (ref[:, 0] < 4).sum() >= 3 and (ref[:, 0] >= 4).sum() > 100   # big-small and small-small
    for shuffle in (0, 5):
        pairs, eps = _broad(hs, s.poses, bound, s.radius, shuffle)
        assert np.array_equal(pairs, ref)
        assert np.array_equal(eps, imp.pair_eps(s.radius, ref[:, 0], ref[:, 1]))


def _cg_system(rng, n, n_edges, spd=True):
    pairs = np.array(sorted({tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(n_edges)}),
                     np.int32)
    Q = rng.normal(size=(len(pairs), 12, 12))
    blocks = Q @ Q.transpose(0, 2, 1) if spd else -50.0 * np.repeat(np.eye(12)[None], len(pairs), 0)
    mass, inertia = rng.uniform(0.5, 2.0, n), rng.uniform(0.1, 1.0, n)
    return pairs, np.ascontiguousarray(blocks), mass, inertia


def _dense(n, pairs, blocks, mass, inertia, dt):
    Md = np.concatenate([np.repeat(mass[:, None], 3, 1), np.repeat(inertia[:, None], 3, 1)], 1).ravel()
    A = np.diag(Md / dt)
    for p, (a, b) in enumerate(pairs):
        idx = np.r_[6 * a:6 * a + 6, 6 * b:6 * b + 6]
        A[np.ix_(idx, idx)] += dt * blocks[p]
    return A, Md


def test_cg_functions_assemble_the_newton_matrix(hs):
    """The solve's per-element functions apply M/dt + dt K (pair blocks in
    row-major 12x12, A's twist first) and its diagonal exactly as the
    assembled dense matrix; the serial sequence of the solve's kernels
    reaches its solution, and stops at negative curvature with the flagged
    step."""
    hs.hs_cg_matvec.argtypes = [C.c_int, C.c_longlong, C.POINTER(C.c_int), DP, DP, DP, C.c_double,
                                DP, DP, DP]
    hs.hs_cg_solve.restype = C.c_int
    hs.hs_cg_solve.argtypes = [C.c_int, C.c_longlong, C.POINTER(C.c_int), DP, DP, DP, C.c_double, DP,
                               DP, C.c_int, C.c_double, C.POINTER(C.c_int)]
    rng = np.random.default_rng(12)
    n, dt = 40, 0.05
    pairs, blocks, mass, inertia = _cg_system(rng, n, 90)
    A, Md = _dense(n, pairs, blocks, mass, inertia, dt)
    ip = lambda a: np.ascontiguousarray(a, np.int32).ctypes.data_as(C.POINTER(C.c_int))  # noqa: E731
    p = rng.normal(size=6 * n)
    ap, diag = np.zeros(6 * n), np.zeros(6 * n)
    hs.hs_cg_matvec(n, len(pairs), ip(pairs), blocks.ctypes.data_as(DP), _d(mass).ctypes.data_as(DP),
                    _d(inertia).ctypes.data_as(DP), dt, p.ctypes.data_as(DP), ap.ctypes.data_as(DP),
                    diag.ctypes.data_as(DP))
    assert np.abs(ap - A @ p).max() <= 1e-12 * np.abs(A @ p).max()
    assert np.abs(diag - np.diag(A)).max() <= 1e-12 * np.abs(np.diag(A)).max()
    b = rng.normal(size=6 * n)
    x = np.zeros(6 * n)
    brk = C.c_int()
    it = hs.hs_cg_solve(n, len(pairs), ip(pairs), blocks.ctypes.data_as(DP), _d(mass).ctypes.data_as(DP),
                        _d(inertia).ctypes.data_as(DP), dt, b.ctypes.data_as(DP), x.ctypes.data_as(DP),
                        400, 1e-13, C.byref(brk))
    assert brk.value == 0 and 0 < it < 400
    want = np.linalg.solve(A, b)
    assert np.abs(x - want).max() <= 1e-10 * np.abs(want).max()
    # negative curvature along the first direction
    n = 6
    pairs = np.array([[0, 1], [2, 3], [4, 5]], np.int32)
    blocks = np.ascontiguousarray(-50.0 * np.repeat(np.eye(12)[None], 3, 0))
    mass, inertia = rng.uniform(0.5, 2.0, n), rng.uniform(0.1, 1.0, n)
    dt = 0.5
    A, Md = _dense(n, pairs, blocks, mass, inertia, dt)
    b = rng.normal(size=6 * n)
    x = np.zeros(6 * n)
    it = hs.hs_cg_solve(n, 3, ip(pairs), blocks.ctypes.data_as(DP), _d(mass).ctypes.data_as(DP),
                        _d(inertia).ctypes.data_as(DP), dt, b.ctypes.data_as(DP), x.ctypes.data_as(DP),
                        10, 1e-10, C.byref(brk))
    d = np.where(np.diag(A) > 0, np.diag(A), Md / dt)
    z = b / d
    pap = z @ A @ z
    assert pap < 0 and it == 0 and brk.value == 1
    assert np.abs(x - (b @ z) / -pap * z).max() <= 1e-12 * np.abs(x).max()


def test_pose_point_function_equals_oracle(hs, orc):
    """World points R v + t of the kernels that build world triangles
    (Hessian blocks, candidate refinement) against the oracle's pose matrix,
    for unit and unnormalised quaternions."""
    hs.hs_pose_points.argtypes = [DP, C.c_int, DP, DP]
    rng = np.random.default_rng(15)
    v = rng.normal(size=(50, 3))
    for _ in range(20):
        pose = np.concatenate([rng.normal(size=3) * 10, rng.normal(size=4) * rng.uniform(0.5, 2)])
        out = np.zeros((50, 3))
        hs.hs_pose_points(_d(pose).ctypes.data_as(DP), 50, _d(v).ctypes.data_as(DP),
                          out.ctypes.data_as(DP))
        want = v @ orc.pose_matrix(pose).T + pose[:3]
        assert np.abs(out - want).max() <= 1e-13 * (1 + np.abs(want).max())
