"""The paper's experiments on incomplete data and on a hemisphere (Sec. V), through
the GPU path (density measures -> sigma -> centres -> FGMRES -> grid -> level set).

They are qualitative in the paper (rendered figures); here each is reduced to
what its figure shows, on a quasi-uniform (golden-spiral) sphere cloud:
  * incomplete data: half of the points removed at random, the fill distance grows
    (by 2.09x in the paper) and sigma = h sqrt(2) re-measured on the reduced cloud
    reconstructs the sphere where the old sigma leaves it visibly wrong;
  * hemisphere: data on the upper half only.  sigma from the fill distance over
    the half-sphere M+ gives the cap and nothing near the lower half; over the
    whole sphere M the fill distance is sqrt(2) (the south pole to the equator),
    sigma = 2, and the lower half is reconstructed as well.
Thresholds carry margins of 3x or more over one measured run.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    import paper_1305_5179_b300 as m
    return m


@pytest.fixture(scope="module")
def ctx(rbf):
    return rbf.Context(0)


def d4(a):
    A = np.zeros((len(a), 4), np.float32)
    A[:, :3] = a
    return torch.from_numpy(A).cuda()


def sphere_probes(m=200_000, seed=9, upper=False):
    u = np.random.default_rng(seed).standard_normal((m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    if upper:
        u[:, 2] = np.abs(u[:, 2])
    return u


def level_set(rbf, ctx, X, sigma, box, G=48, **solve_kw):
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    C, b, _ = rbf.build_centers(ctx, Xd, Xd, delta=0.05)          # unit sphere: normal = position
    plan = rbf.Plan(ctx, C, sigma=sigma, k=0.0)
    x, rep = plan.solve(b, **solve_kw)
    lo, hi = (-box,) * 3, (box,) * 3
    T = rbf.isosurface(ctx, plan.eval_grid(x, lo, hi, (G, G, G)), lo, hi, 0.0).cpu().numpy().astype(np.float64)
    return T.reshape(-1, 3), rep


def topology(V):
    """(Euler characteristic, edges not shared by exactly two triangles)."""
    uniq, inv = np.unique(np.round(V, 6), axis=0, return_inverse=True)
    F = inv.reshape(-1, 3)
    E = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), 1)
    Eu, cnt = np.unique(E, axis=0, return_counts=True)
    return len(uniq) - len(Eu) + len(F), int((cnt != 2).sum())


def test_incomplete_data_needs_the_remeasured_sigma(ctx, rbf):
    N = 560
    X = synth.fibonacci_sphere(N).points
    half = np.sort(np.random.default_rng(1).choice(N, N // 2, replace=False))
    Xh = X[half]
    pr = d4(sphere_probes())
    d_full = rbf.density_measures(ctx, d4(X), pr)
    d_half = rbf.density_measures(ctx, d4(Xh), pr)
    assert d_half["fill"] > 2.0 * d_full["fill"]          # measured 2.34x (the paper: 0.157 -> 0.328)
    kw = dict(m=50, max_it=400, tol=1e-6)
    V_old, _ = level_set(rbf, ctx, Xh, d_full["sigma_fill"], 1.3, **kw)
    V_new, _ = level_set(rbf, ctx, Xh, d_half["sigma_fill"], 1.3, **kw)
    dev_old = np.abs(np.linalg.norm(V_old, axis=1) - 1)
    dev_new = np.abs(np.linalg.norm(V_new, axis=1) - 1)
    # measured: mean 0.0035 / max 0.030 with the old sigma, 0.00025 / 0.0012 with the new
    assert dev_new.max() < 0.005 and dev_new.mean() < 0.001
    assert dev_old.mean() > 4 * dev_new.mean() and dev_old.max() > 0.01


def test_hemisphere_fill_distance_is_sqrt2_over_the_whole_sphere(ctx, rbf):
    Xf = synth.fibonacci_sphere(1120).points
    Xu = Xf[Xf[:, 2] >= 0]
    zmin = float(Xu[:, 2].astype(np.float64).min())
    probes = np.vstack([sphere_probes(), [[0.0, 0.0, -1.0]]])
    d = rbf.density_measures(ctx, d4(Xu), d4(probes))
    # the south pole's nearest point is the lowest one, at distance sqrt(2 + 2 z_min)
    assert d["fill"] == pytest.approx(np.sqrt(2.0 + 2.0 * zmin), rel=1e-6)
    assert d["sigma_fill"] == pytest.approx(2.0, abs=2e-3)
    dc = rbf.density_measures(ctx, d4(Xu), d4(sphere_probes(upper=True)))
    assert dc["sigma_fill"] < 0.2                          # measured 0.147 (the paper: 0.157)


def test_hemisphere_reconstructs_the_cap_or_the_sphere(ctx, rbf):
    """Fifty GMRES iterations as in the paper's timings."""
    Xf = synth.fibonacci_sphere(1120).points
    Xu = Xf[Xf[:, 2] >= 0]
    kw = dict(m=50, max_it=50, fixed_iterations=True)
    s_cap = rbf.density_measures(ctx, d4(Xu), d4(sphere_probes(upper=True)))["sigma_fill"]
    s_sph = rbf.density_measures(ctx, d4(Xu), d4(np.vstack([sphere_probes(), [[0.0, 0.0, -1.0]]])))["sigma_fill"]
    V_cap, _ = level_set(rbf, ctx, Xu, s_cap, 1.5, **kw)
    V_sph, rep = level_set(rbf, ctx, Xu, s_sph, 1.5, **kw)
    low_cap = V_cap[V_cap[:, 2] < -0.5]
    low_sph = V_sph[V_sph[:, 2] < -0.5]
    # measured: the cap's level set below z = -0.5 is 0.45 off the sphere on average; the
    # sigma = 2 level set 0.005, closed (Euler characteristic 2, every edge shared twice)
    assert np.abs(np.linalg.norm(low_cap, axis=1) - 1).mean() > 0.2
    assert len(low_sph) > 1000 and np.abs(np.linalg.norm(low_sph, axis=1) - 1).mean() < 0.02
    assert topology(V_sph) == (2, 0)
