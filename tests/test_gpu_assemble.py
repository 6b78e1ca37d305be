"""GPU parity of the assembled truncated matrix (Algorithm 2) and its CSR product.

The assembled rows are compared with the oracle's brute-force rows of the same
float32 centres (as float64):
  * entry sets: exact (the library decides the cut-off as the pair count does,
    float32 with a float64 repeat near the radius, so it equals the float64 test);
  * values: relative error below 2^-21 + 7 x 2^-24 ln(2) t, t = -log2(A_ij): the
    float32 squared distance carries at most 7 roundings of 2^-24 relative
    (differences, squares, sums, the scale), ex2.approx below 2^-21 relative;
  * padding: rows padded to multiples of 4 with (own position, 0) entries;
  * product: |y - y64|_2 / |y64|_2 <= 1e-5 against the oracle, 3e-6 against the
    matrix-free product (two float32 sums of the same terms);
  * solve: the assembled operator inside FGMRES reaches the same float64 residual.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32 = np.float32


@pytest.fixture(scope="module")
def rbf():
    import paper_1305_5179_b300 as m
    return m


@pytest.fixture(scope="module")
def ctx(rbf):
    return rbf.Context(0)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def c4(C):
    C32 = np.zeros((len(C), 4), dtype=np.float32)
    C32[:, :3] = C
    return dev(C32), C32[:, :3].astype(np.float64)


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def torus_patch(theta, seed, N_full=1_000_000, delta=0.01):
    cl = synth.torus(int(N_full * theta / (2 * math.pi)), noise=1e-3, seed=seed, theta_max=theta)
    return oracle.build_centers(cl.points, cl.normals, delta)


def check_rows(plan, C64, sigma, k, rows, radius_sigmas=0.0):
    """Assembled rows at binned positions ``rows`` against the oracle's rows."""
    perm = plan.export_binning()[0].cpu().numpy().astype(np.int64)
    rp, col, val = plan.export_csr()
    rp_h = rp.cpu().numpy()
    ent = oracle.truncated_entries(C64, sigma, k, perm[rows], radius_sigmas=radius_sigmas)
    for p, (cols64, vals64) in zip(rows, ent):
        a, b = int(rp_h[p]), int(rp_h[p + 1])
        c = col[a:b].cpu().numpy().astype(np.int64)
        v = val[a:b].cpu().numpy().astype(np.float64)
        nreal = len(cols64)
        assert b - a == (nreal + 3) // 4 * 4, (p, b - a, nreal)
        assert (v[:nreal] > 0).all() and (v[nreal:] == 0).all() and (c[nreal:] == p).all()
        cc = perm[c[:nreal]]
        order = np.argsort(cc)
        assert np.array_equal(cc[order], cols64), p
        t = -np.log2(vals64)
        bound = 2.0 ** -21 + 7 * 2.0 ** -24 * math.log(2.0) * t
        err = np.abs(v[:nreal][order] - vals64) / vals64
        assert (err <= bound).all(), (p, float((err / bound).max()))
    return rp_h


def test_assembled_torus_patch_matches_oracle_rows(ctx, rbf):
    C, _ = torus_patch(0.05, seed=3)
    Cd, C64 = c4(C)
    sigma, k = float(F32(0.02)), float(F32(6.0))
    plan = rbf.Plan(ctx, Cd, sigma=0.02, k=6.0)
    nnz, stored = plan.assemble()
    assert nnz == plan.count_pairs()
    n = len(C)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.choice(n, 48, replace=False), [0, 1, n - 2, n - 1]]))
    rp_h = check_rows(plan, C64, sigma, k, rows)
    assert rp_h[0] == 0 and rp_h[-1] == stored and (rp_h % 4 == 0).all() and (np.diff(rp_h) >= 4).all()
    assert nnz <= stored < nnz + 4 * n


def test_spmv_matches_oracle_and_matrix_free(ctx, rbf):
    C, _ = torus_patch(0.05, seed=4)
    Cd, C64 = c4(C)
    plan = rbf.Plan(ctx, Cd, sigma=0.02, k=6.0)
    plan.assemble()
    rng = np.random.default_rng(2)
    z = rng.standard_normal(len(C)).astype(np.float32)
    y = plan.spmv(dev(z)).cpu().numpy().astype(np.float64)
    ymf = plan.matvec(dev(z)).cpu().numpy().astype(np.float64)
    assert rel2(y, ymf) <= 3e-6
    rows = rng.choice(len(C), 4000, replace=False)
    y64, _ = oracle.kernel_rows(C64, z.astype(np.float64), float(F32(0.02)), float(F32(6.0)), rows)
    assert rel2(y[rows], y64) <= 1e-5


def test_assembled_dense_sphere_c1(ctx, rbf, sphere_c1):
    """Untruncated plan (k = 0): every pair closer than 13 sigma is stored; the product
    equals the dense oracle product (the omitted entries are below 2.2e-37)."""
    C, _ = oracle.build_centers(sphere_c1.points, sphere_c1.normals, 0.05)
    Cd, C64 = c4(C)
    s = float(F32(0.1))
    plan = rbf.Plan(ctx, Cd, sigma=0.1, k=0.0)
    nnz, stored = plan.assemble()
    d2 = ((C64[:, None, :] - C64[None, :, :]) ** 2).sum(-1)
    assert nnz == int((d2 < (13.0 * s) ** 2).sum())
    check_rows(plan, C64, s, 0.0, np.array([0, 17, 2250, len(C) - 1]), radius_sigmas=13.0)
    z = np.random.default_rng(3).standard_normal(len(C))
    y = plan.spmv(dev(z.astype(np.float32))).cpu().numpy().astype(np.float64)
    A = oracle.dense_matrix(C64, s)
    assert rel2(y, A @ z.astype(np.float32).astype(np.float64)) <= 1e-5


def test_assembled_isolated_and_single_centres(ctx, rbf):
    """Rows holding only their diagonal: one real entry and three padding entries each;
    the product is the identity."""
    C = np.arange(5, dtype=np.float64)[:, None] * np.array([[3.0, 0.0, 0.0]])
    Cd, C64 = c4(C)
    plan = rbf.Plan(ctx, Cd, sigma=0.1, k=6.0)
    assert plan.assemble() == (5, 20)
    rp, col, val = plan.export_csr()
    assert rp.cpu().tolist() == [0, 4, 8, 12, 16, 20]
    v = val.cpu().numpy().reshape(5, 4)
    assert (v[:, 0] == 1.0).all() and (v[:, 1:] == 0).all()
    c = col.cpu().numpy().reshape(5, 4)
    assert (c == np.arange(5)[:, None]).all()
    z = np.array([1.5, -2.0, 3.25, 0.0, 7.0], dtype=np.float32)
    assert np.array_equal(plan.spmv(dev(z)).cpu().numpy(), z)
    one = rbf.Plan(ctx, dev(np.zeros((1, 4), np.float32)), sigma=0.1, k=6.0)
    assert one.assemble() == (1, 4)


def test_assemble_size_cap_and_release(ctx, rbf):
    C, _ = torus_patch(0.02, seed=6)
    Cd, _ = c4(C)
    plan = rbf.Plan(ctx, Cd, sigma=0.02, k=6.0)
    with pytest.raises(rbf.RbfError) as ei:
        plan.assemble(max_bytes=1 << 20)
    assert ei.value.status == 2 and ei.value.nnz == plan.count_pairs() and ei.value.stored >= ei.value.nnz
    z = dev(np.ones(len(C), np.float32))
    with pytest.raises(rbf.RbfError) as ei:
        plan.spmv(z)
    assert ei.value.status == 1
    plan.assemble()
    y = plan.spmv(z)
    plan.release_csr()
    with pytest.raises(rbf.RbfError):
        plan.spmv(z)
    assert torch.isfinite(y).all()


def test_solve_with_assembled_operator(ctx, rbf):
    """FGMRES on the assembled matrix: same convergence as matrix-free on the
    well-conditioned sphere (sigma below the spacing), residual checked in float64
    by the oracle; and the same fixed-iteration residual on a torus patch with RAS."""
    cl = synth.sphere(400, seed=4)
    C, b = oracle.build_centers(cl.points, cl.normals, 0.05)
    Cd, C64 = c4(C)
    b32 = b.astype(np.float32)
    s = float(F32(0.04))
    plan = rbf.Plan(ctx, Cd, sigma=0.04, k=0.0)
    with pytest.raises(rbf.RbfError):
        plan.solve(dev(b32), m=40, max_it=10, assembled=True)
    plan.assemble()
    x, rep = plan.solve(dev(b32), m=40, max_it=600, tol=1e-8, assembled=True)
    assert rep["converged"] == 1 and rep["residual_true"] <= 1e-8, rep
    r = oracle.residual_rows(C64, b32.astype(np.float64), x.cpu().numpy(), s, 0.0)
    assert np.linalg.norm(r) / np.linalg.norm(b32) == pytest.approx(rep["residual_true"], rel=1e-6)
    xm, repm = plan.solve(dev(b32), m=40, max_it=600, tol=1e-8)
    assert abs(rep["iterations"] - repm["iterations"]) <= 3

    C, b = torus_patch(0.05, seed=7)
    Cd, _ = c4(C)
    b32 = b.astype(np.float32)
    plan = rbf.Plan(ctx, Cd, sigma=0.02, k=6.0)
    plan.assemble()
    kw = dict(precond="schwarz", core=96, block=128, shift=1e-4, escalate=True, m=20, max_it=40,
              fixed_iterations=True)
    _, ra = plan.solve(dev(b32), assembled=True, **kw)
    _, rm = plan.solve(dev(b32), **kw)
    assert ra["iterations"] == rm["iterations"] == 40
    assert ra["residual_true"] == pytest.approx(rm["residual_true"], rel=0.05)


def test_assembled_at_the_bench_size(ctx, rbf):
    """The benchmark's sector (0 <= theta < 0.6 of the 1,000,000-point torus, 286,476 centres,
    2.56e9 entries, 20.5 GB of CSR): sampled rows against the oracle's rows, the product on
    sampled rows, the entry count against the pair count."""
    C, _ = torus_patch(0.6, seed=0)
    Cd, C64 = c4(C)
    s, k = float(F32(0.02)), float(F32(6.0))
    plan = rbf.Plan(ctx, Cd, sigma=0.02, k=6.0)
    nnz, stored = plan.assemble()
    assert nnz == plan.count_pairs()
    rng = np.random.default_rng(5)
    check_rows(plan, C64, s, k, np.sort(rng.choice(len(C), 40, replace=False)))
    z = rng.standard_normal(len(C)).astype(np.float32)
    y = plan.spmv(dev(z)).cpu().numpy().astype(np.float64)
    rows = rng.choice(len(C), 3000, replace=False)
    y64, _ = oracle.kernel_rows(C64, z.astype(np.float64), s, k, rows)
    assert rel2(y[rows], y64) <= 1e-5
    plan.release_csr()
