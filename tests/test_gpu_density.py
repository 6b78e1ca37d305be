"""Density measures of Sec. IV on the GPU (rbf_density_measures) against the
FP64 oracle, the paper's worked example and closed forms."""
import json
import math
import os

import numpy as np
import pytest

import oracle
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


def f4(X):
    A = np.zeros((len(X), 4), dtype=np.float32)
    A[:, :3] = X
    return torch.from_numpy(A).cuda()


def test_halton_example_of_the_paper(rbf, ctx):
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "density_halton25.json")))
    P = synth.halton(25, bases=(2, 3), start=1)
    X = np.c_[P, np.zeros(25)]
    m = 1201
    u = np.linspace(0.0, 1.0, m)
    gx, gy = np.meshgrid(u, u, indexing="ij")
    probes = np.c_[gx.ravel(), gy.ravel(), np.zeros(m * m)]
    d = rbf.density_measures(ctx, f4(X), f4(probes))
    half = 0.5 * 10.0 ** -(g["printed_digits"])
    assert abs(d["q"] - g["q"]) <= half
    assert abs(d["fill"] - g["fill"]) <= half + 1.0 / (m - 1)
    X32 = X.astype(np.float32).astype(np.float64)
    o = oracle.density_measures(X32, probes.astype(np.float32).astype(np.float64))
    for key in ("q", "h_max", "mean_nn", "fill"):
        assert d[key] == pytest.approx(o[key], rel=2e-6), key
    assert d["sigma_hmax"] == pytest.approx(d["h_max"] * math.sqrt(2), rel=1e-12)


def test_torus_sector_against_oracle(rbf, ctx):
    theta = 0.12
    cl = synth.torus(int(1_000_000 * theta / (2 * math.pi)), noise=1e-3, seed=8, theta_max=theta)
    clean = synth.torus(5000, noise=0.0, seed=9, theta_max=theta)
    X = cl.points.astype(np.float32).astype(np.float64)
    Pr = clean.points.astype(np.float32).astype(np.float64)
    d, nn = rbf.density_measures(ctx, f4(X), f4(Pr), return_nn=True)
    nn = nn.cpu().numpy().astype(np.float64)
    o_nn = oracle.nn_distances(X)
    assert np.abs(nn - o_nn).max() <= 2e-6 * o_nn.max()
    assert d["q"] == pytest.approx(0.5 * o_nn.min(), rel=2e-6, abs=1e-9)
    assert d["h_max"] == pytest.approx(o_nn.max(), rel=2e-6)
    assert d["mean_nn"] == pytest.approx(o_nn.mean(), rel=2e-6)
    assert d["fill"] == pytest.approx(oracle.fill_distance(X, Pr), rel=2e-6)
    # an explicit, coarser search cell gives the same distances
    d2, nn2 = rbf.density_measures(ctx, f4(X), f4(Pr), cell=4 * d["cell"], return_nn=True)
    assert np.array_equal(nn, nn2.cpu().numpy().astype(np.float64))
    assert d2["fill"] == d["fill"]


def test_lattice_duplicates_and_far_points(rbf, ctx):
    s = 0.05
    g = np.arange(12) * s
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    c = g[:-1] + s / 2
    Pr = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    d = rbf.density_measures(ctx, f4(X), f4(Pr))
    assert d["q"] == pytest.approx(s / 2, rel=1e-6)
    assert d["h_max"] == pytest.approx(s, rel=1e-6) and d["mean_nn"] == pytest.approx(s, rel=1e-6)
    assert d["fill"] == pytest.approx(s * math.sqrt(3) / 2, rel=1e-6)
    Xd = np.concatenate([X, X[:3]])
    assert rbf.density_measures(ctx, f4(Xd))["q"] == 0.0
    two = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    t = rbf.density_measures(ctx, f4(two))
    assert t["q"] == pytest.approx(2.5, rel=1e-6) and t["h_max"] == pytest.approx(5.0, rel=1e-6)
    assert math.isnan(t["fill"])


def test_batch_sigma_rule_matches_generator(rbf, ctx):
    """The batched workload's sigma is 3 x the mean nearest-neighbour spacing of each
    cloud (computed by the generator with a k-d tree); the GPU mean agrees."""
    for cl in synth.batch(nclouds=4, nmin=500, nmax=3000, seed=3):
        d = rbf.density_measures(ctx, f4(cl.points.astype(np.float64)))
        assert 3.0 * d["mean_nn"] == pytest.approx(cl.params["sigma"], rel=1e-5)


def test_invalid_inputs(rbf, ctx):
    with pytest.raises(rbf.RbfError):
        rbf.density_measures(ctx, f4(np.zeros((1, 3))))
    bad = np.zeros((10, 3))
    bad[3, 1] = np.nan
    with pytest.raises(rbf.RbfError):
        rbf.density_measures(ctx, f4(bad))
    with pytest.raises(rbf.RbfError):
        rbf.density_measures(ctx, f4(np.random.default_rng(0).uniform(0, 1, (10, 3))), f4(bad))


def test_benchmark_size_sampled(rbf, ctx):
    """The benchmark's cloud (the 1,000,000-point torus, noise 1e-3, seed 0): sampled
    nearest-neighbour distances by brute force over all points, the separation and
    h_max against the extremes of the GPU's own per-point distances, and the fill
    distance over a 2,000-probe subset of the noise-free torus against the oracle."""
    X = synth.torus(1_000_000, noise=1e-3, seed=0).points.astype(np.float32).astype(np.float64)
    Pr = synth.torus(1_000_000, noise=0.0, seed=1).points.astype(np.float32).astype(np.float64)
    d, nn = rbf.density_measures(ctx, f4(X), f4(Pr), return_nn=True)
    nn = nn.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(3)
    rows = np.concatenate([rng.choice(len(X), 300, replace=False), [int(nn.argmin()), int(nn.argmax())]])
    o = oracle.nn_distances(X, rows)
    assert np.abs(nn[rows] - o).max() <= 2e-6 * o.max() + 1e-9
    assert d["q"] == pytest.approx(0.5 * nn.min(), rel=1e-7) and d["h_max"] == pytest.approx(nn.max(), rel=1e-7)
    assert d["mean_nn"] == pytest.approx(nn.mean(), rel=1e-6)
    sub = Pr[rng.choice(len(Pr), 2000, replace=False)]
    ds = rbf.density_measures(ctx, f4(X), f4(sub))
    assert ds["fill"] == pytest.approx(oracle.fill_distance(X, sub), rel=2e-6)
    assert d["fill"] >= ds["fill"]
