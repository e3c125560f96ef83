"""GPU triangle-pair kernels (Sec. 3) through the C ABI against the FP64 oracle:
the comparison-based distance in both precision forms and the float penalty
sweep with its certificate."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    import paper_2105_12415_gb300 as m
    m.build()
    return m.Context(0)


def _families(rng, n):
    P1 = rng.normal(size=(n, 9))
    Q1 = rng.normal(size=(n, 9)) + np.tile(rng.normal(size=(n, 3)), 3)
    # near contact: Q is P moved along its normal by ~eps and sideways
    P = rng.normal(size=(n, 3, 3))
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    Q = (P + rng.uniform(-0.05, 0.1, size=(n, 1, 1)) * nrm[:, None, :]
         + rng.normal(scale=0.5, size=(n, 1, 3)) + rng.normal(scale=0.02, size=(n, 3, 3)))
    # far from the origin (large coordinates, small gaps)
    off = rng.uniform(-50, 50, size=(n, 1, 3))
    P3 = (rng.normal(scale=0.05, size=(n, 3, 3)) + off).reshape(n, 9)
    Q3 = (rng.normal(scale=0.05, size=(n, 3, 3)) + off + rng.normal(scale=0.05, size=(n, 1, 3))).reshape(n, 9)
    return (np.concatenate([P1, P.reshape(n, 9), P3]), np.concatenate([Q1, Q.reshape(n, 9), Q3]))


def test_exact_distance_fp64_matches_oracle(gctx, orc):
    import torch
    import paper_2105_12415_gb300 as m
    rng = np.random.default_rng(101)
    P, Q = _families(rng, 40000)
    d_ref, pa_ref, pb_ref, f_ref = orc.tri_tri(P, Q)
    dev = torch.device("cuda:0")
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    eps = np.full(len(P), 0.05)
    out = m.triangle_distance(gctx, T(P), T(Q), T(eps), precision="fp64")
    d = out["d"].cpu().numpy()
    err = np.abs(d - d_ref) / np.maximum(d_ref, 0.05)
    assert err.max() <= 1e-12, err.max()
    # the feature code is not unique (a vertex whose closest point lies on an
    # edge ties with that edge-edge test); the closest points are, except for
    # parallel features, so compare those
    pa, pb = out["pa"].cpu().numpy(), out["pb"].cpu().numpy()
    dev_pts = np.maximum(np.linalg.norm(pa - pa_ref, axis=1), np.linalg.norm(pb - pb_ref, axis=1))
    assert np.mean(dev_pts <= 1e-9) > 0.999
    assert np.all(np.abs(np.linalg.norm(pa - pb, axis=1) - d) <= 1e-12 * np.maximum(d, 1))


def test_exact_distance_fp32_form(gctx, orc):
    """FP32 form: pairs within 2 eps get double-float final values (about 48
    significant bits); the contact decision matches the oracle outside a
    1e-6 eps band."""
    import torch
    import paper_2105_12415_gb300 as m
    rng = np.random.default_rng(102)
    P, Q = _families(rng, 40000)
    d_ref, _, _, _ = orc.tri_tri(P, Q)
    dev = torch.device("cuda:0")
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    eps = np.maximum(0.5 * d_ref * rng.uniform(0.9, 1.1, size=len(P)), 1e-3)  # many near 2 eps
    out = m.triangle_distance(gctx, T(P), T(Q), T(eps), precision="fp32")
    d = out["d"].cpu().numpy()
    tau = 2 * eps
    feat = out["feature"].cpu().numpy()
    hit = (d <= tau) & (feat != -2)    # -2: the float test decided "beyond 2 eps"
    hit_ref = d_ref <= tau
    band = np.abs(d_ref - tau) <= 1e-6 * eps
    assert np.all((hit == hit_ref) | band)
    assert np.all((feat != -2) | (d_ref > tau) | band)
    err = np.abs(d - d_ref) / np.maximum(d_ref, eps)
    assert err[hit_ref].max() <= 1e-5, err[hit_ref].max()
    # the double-float finishing is far more accurate than the contract
    assert err[hit_ref & hit].max() <= 1e-9, err[hit_ref & hit].max()
    pa, pb = out["pa"].cpu().numpy(), out["pb"].cpu().numpy()
    gap = np.abs(np.linalg.norm(pa - pb, axis=1) - d)
    assert gap[hit].max() <= 1e-9 * max(1.0, float(np.abs(P).max())), gap[hit].max()


def test_sweep_matches_oracle_and_certificate_is_sound(gctx, orc):
    import torch
    import paper_2105_12415_gb300 as m
    rng = np.random.default_rng(103)
    P, Q = _families(rng, 30000)
    # translate each pair so that P's first vertex is the origin (the kernel's frame)
    o = P[:, :3].copy()
    P0 = P - np.tile(o, 3)
    Q0 = Q - np.tile(o, 3)
    d_ref, _, _, _ = orc.tri_tri(P0, Q0)
    eps = np.full(len(P), 0.02)
    p = gctx.params
    ref = orc.sweep(P0.astype(np.float32).astype(np.float64), Q0.astype(np.float32).astype(np.float64),
                    eps, n_iter=p.n_iter, rho_reg=p.rho_reg, rho_iter=p.rho_iter, conv_c=p.conv_c)
    dev = torch.device("cuda:0")
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    out = m.triangle_distance(gctx, T(P0), T(Q0), T(eps), precision="fp64")
    gap = out["gap"].cpu().numpy().astype(np.float64)
    scale = np.abs(np.concatenate([P0, Q0], 1)).max(1)
    ok = np.isnan(gap) | (gap <= d_ref + 1e-5 * scale)
    assert ok.all()
    x = out["x"].cpu().numpy().astype(np.float64)
    # the float iteration follows the FP64 one (same steps, float rounding)
    diff = np.abs(x - ref["x"]).max(1)
    assert np.median(diff) < 1e-5 and np.mean(diff < 1e-3) > 0.99
    conv = out["converged"].cpu().numpy().astype(bool)
    assert np.mean(conv == ref["converged"]) > 0.99
