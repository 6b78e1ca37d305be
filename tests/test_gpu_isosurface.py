"""Step 4 without rendering: the level set of the grid field on the GPU
(rbf_isosurface) against the oracle's marching tetrahedra on the same float32
field, and on the C1 reconstruction."""
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


def _compare(rbf, ctx, f32, lo, hi, iso=0.0):
    T = rbf.isosurface(ctx, torch.from_numpy(f32).cuda(), lo, hi, iso).cpu().numpy().astype(np.float64)
    To, counts = oracle.isosurface(f32.astype(np.float64), lo, hi, iso)
    assert len(T) == len(To)
    step = (np.asarray(hi, float) - np.asarray(lo, float)) / (np.array(f32.shape[::-1]) - 1)
    if len(T):
        assert np.abs(T - To).max() <= 2e-6 * max(1.0, np.abs(To).max()) + 1e-6 * step.max()
    return T, To


def test_linear_field_and_single_cell(rbf, ctx):
    a = np.array([0.3, -0.5, 0.8])
    lo, hi = (-1.0, -0.7, -0.6), (0.9, 1.1, 0.8)
    xs = [np.linspace(lo[d], hi[d], g) for d, g in enumerate((13, 11, 9))]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    f = (a[0] * X + a[1] * Y + a[2] * Z - 0.1).astype(np.float32)
    T, _ = _compare(rbf, ctx, f, lo, hi)
    n = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
    live = np.linalg.norm(n, axis=1) > 1e-10
    assert np.all(n[live] @ a > 0)
    one = np.array([[[-1.0, 1.0], [1.0, 1.0]], [[1.0, 1.0], [1.0, 2.0]]], dtype=np.float32)   # one cell
    _compare(rbf, ctx, one, (0, 0, 0), (1, 1, 1))


@pytest.mark.parametrize("shape", ["sphere", "torus"])
def test_signed_distance_fields(rbf, ctx, shape):
    g = np.linspace(-1.0, 1.0, 41)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    if shape == "sphere":
        f = np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 0.63
    else:
        f = np.sqrt((np.sqrt(X ** 2 + Y ** 2) - 0.55) ** 2 + Z ** 2) - 0.23
    _compare(rbf, ctx, f.astype(np.float32), (-1.0,) * 3, (1.0,) * 3)


def test_nan_cells_empty_and_capacity(rbf, ctx):
    g = np.linspace(-1.0, 1.0, 17)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    f = (np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 0.7).astype(np.float32)
    f[:, :, :5] = np.nan
    _compare(rbf, ctx, f, (-1.0,) * 3, (1.0,) * 3)
    pos = np.ones((5, 6, 7), dtype=np.float32)
    assert len(rbf.isosurface(ctx, torch.from_numpy(pos).cuda(), (0, 0, 0), (1, 1, 1))) == 0
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    g_ = rbf._grid((-1.0,) * 3, (1.0,) * 3, (17, 17, 17))
    import ctypes
    n = ctypes.c_int64(0)
    small = torch.empty((1, 9), dtype=torch.float32, device="cuda")
    st = rbf.lib().rbf_isosurface(ctx._h, rbf._ptr(fd), ctypes.byref(g_), 0.0, None, 0, 0.0, rbf._ptr(small), 1,
                                  ctypes.byref(n), None)
    assert st == 1 and n.value > 1                       # RBF_ERR_INVALID, count still reported


def test_c1_reconstructed_sphere(rbf, ctx, sphere_c1):
    """The whole path on C1: oracle weights, GPU 64^3 grid, GPU level set; the
    triangles match the oracle's on the same field, and every vertex lies within
    delta/2 of the unit sphere."""
    C, b = oracle.build_centers(sphere_c1.points, sphere_c1.normals, 0.05)
    C32 = np.zeros((len(C), 4), dtype=np.float32)
    C32[:, :3] = C
    xo, _ = oracle.solve_dense(C32[:, :3].astype(np.float64), b, float(np.float32(0.1)))
    plan = rbf.Plan(ctx, torch.from_numpy(C32).cuda(), sigma=0.1, k=0.0)
    f = plan.eval_grid(torch.from_numpy(xo).cuda(), (-1.2,) * 3, (1.2,) * 3, (64, 64, 64))
    T, _ = _compare(rbf, ctx, f.cpu().numpy(), (-1.2,) * 3, (1.2,) * 3)
    r = np.linalg.norm(T.reshape(-1, 3), axis=1)
    assert np.abs(r - 1.0).max() <= 0.025
    # restricted to a band wider than the cloud's gaps (mean spacing about 0.09) plus
    # a cell: the same surface (this field has no stray sheets to remove)
    P = np.zeros((1500, 4), dtype=np.float32)
    P[:, :3] = sphere_c1.points
    Tb = rbf.isosurface(ctx, f, (-1.2,) * 3, (1.2,) * 3, points=torch.from_numpy(P).cuda(), band=0.2)
    assert 0.99 * len(T) <= len(Tb) <= len(T)


def test_band_matches_oracle(rbf, ctx):
    """Cells are kept when their centre is within the band of a data point; the GPU
    decision equals the oracle's (no cell centre lies within rounding of the band)."""
    g = np.linspace(-1.0, 1.0, 33)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    f = (np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 0.63).astype(np.float32)
    cl = synth.sphere(400, seed=5, radius=0.63)
    keep = cl.points[cl.points[:, 2] > 0.1]                 # data on a cap only
    P = np.zeros((len(keep), 4), dtype=np.float32)
    P[:, :3] = keep
    band = 0.11
    step = 2.0 / 32
    c = -1.0 + (np.stack(np.meshgrid(np.arange(32), np.arange(32), np.arange(32), indexing="ij"), -1) + 0.5) * step
    d = np.sqrt(((c.reshape(-1, 1, 3) - keep[None].astype(np.float64)) ** 2).sum(-1)).min(1)
    assert np.abs(d - band).min() > 1e-5                   # no borderline cell
    T = rbf.isosurface(ctx, torch.from_numpy(f).cuda(), (-1.0,) * 3, (1.0,) * 3, points=torch.from_numpy(P).cuda(),
                       band=band).cpu().numpy().astype(np.float64)
    To, counts = oracle.isosurface(f.astype(np.float64), (-1.0,) * 3, (1.0,) * 3, points=P, band=band)
    assert len(T) == len(To) and 0 < len(To) < len(oracle.isosurface(f.astype(np.float64), (-1.0,) * 3, (1.0,) * 3)[0])
    assert np.abs(T - To).max() <= 2e-6


def test_benchmark_size_field(rbf, ctx):
    """The benchmark's level set: the 256^3 grid field of the 3,000,000-centre torus (20
    RAS-FGMRES iterations).  A 24^3 crop through the surface gives the oracle's triangles
    exactly; over the whole grid, with the band of 0.03, every sampled vertex lies within
    the band plus half a cell diagonal of a cloud point."""
    from scipy.spatial import cKDTree
    cl = synth.torus(1_000_000, noise=1e-3, seed=0)
    C, b, _ = rbf.build_centers(ctx, torch.from_numpy(cl.points).cuda(), torch.from_numpy(cl.normals).cuda(),
                                delta=0.01)
    plan = rbf.Plan(ctx, C, sigma=0.02, k=6.0)
    x, _ = plan.solve(b, m=20, max_it=20, fixed_iterations=True, precond="schwarz", core=96, block=128, shift=1.0,
                      escalate=True)
    pad = 0.01 + 3 * 0.02
    lo = tuple(cl.points.min(0).astype(np.float64) - pad)
    hi = tuple(cl.points.max(0).astype(np.float64) + pad)
    G = 256
    f = plan.eval_grid(x, lo, hi, (G, G, G))
    step = (np.asarray(hi) - np.asarray(lo)) / (G - 1)
    # crop around the node nearest to a surface point on the outer equator, (1.35, 0, 0)
    c = np.round((np.array([1.35, 0.0, 0.0]) - np.asarray(lo)) / step).astype(int)
    i0 = np.clip(c - 12, 0, G - 24)
    fc = f[i0[2]:i0[2] + 24, i0[1]:i0[1] + 24, i0[0]:i0[0] + 24].cpu().numpy().copy()
    clo = tuple(float(np.float32(lo[d])) + i0[d] * float(np.float32(step[d])) for d in range(3))
    chi = tuple(clo[d] + 23 * float(np.float32(step[d])) for d in range(3))
    T, To = _compare(rbf, ctx, fc, clo, chi)
    assert len(T) > 500
    P = np.zeros((len(cl.points), 4), dtype=np.float32)
    P[:, :3] = cl.points
    Tb = rbf.isosurface(ctx, f, lo, hi, 0.0, torch.from_numpy(P).cuda(), 0.03).cpu().numpy().astype(np.float64)
    assert len(Tb) > 1_000_000
    V = Tb.reshape(-1, 3)[np.random.default_rng(0).choice(len(Tb) * 3, 20000, replace=False)]
    dist, _ = cKDTree(cl.points.astype(np.float64)).query(V)
    assert dist.max() <= 0.03 + 0.5 * np.linalg.norm(step) + 1e-6
