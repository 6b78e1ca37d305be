"""The benchmark workload at full size, in the configuration bench.py times:
1,000,000 torus points (R = 1, r = 0.35, noise 1e-3), delta 0.01 -> 3,000,000
centres, sigma 0.02, cut-off 6 sigma, Schwarz subdomains of 128 (core 96, shift 1),
50 FGMRES iterations, 256^3 grid.  Sampled outputs against the FP64 oracle: 10,000
rows of the product and of the true residual, 10,000 grid nodes."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

F32 = np.float32
SIGMA, K, DELTA = 0.02, 6.0, 0.01


@pytest.fixture(scope="module")
def c2():
    import paper_1305_5179_b300 as rbf
    ctx = rbf.Context(0)
    cl = synth.torus(1_000_000, noise=1e-3, seed=0)
    C, b, _ = rbf.build_centers(ctx, torch.from_numpy(cl.points).cuda(), torch.from_numpy(cl.normals).cuda(),
                                delta=DELTA)
    plan = rbf.Plan(ctx, C, sigma=SIGMA, k=K)
    x, rep = plan.solve(b, m=50, max_it=50, fixed_iterations=True, precond="schwarz", core=96, block=128,
                        shift=1.0, escalate=True)
    C64 = C[:, :3].double().cpu().numpy()
    rows = np.random.default_rng(5).choice(len(C64), 10_000, replace=False)
    return rbf, plan, C, b, x, rep, C64, rows, cl


def test_c2_product_sampled_rows(c2):
    rbf, plan, C, b, x, rep, C64, rows, cl = c2
    z = torch.randn(C.shape[0], device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    y = plan.matvec(z).double().cpu().numpy()
    y64, cnt = oracle.kernel_rows(C64, z.double().cpu().numpy(), float(F32(SIGMA)), float(F32(K)), rows)
    err = np.linalg.norm(y[rows] - y64) / np.linalg.norm(y64)
    print(f"\n  C2 product, 10,000 rows: relative error {err:.2e}, {cnt / len(rows):.0f} pairs per row")
    assert err <= 1e-5


def test_c2_solve_residual_sampled_rows(c2):
    rbf, plan, C, b, x, rep, C64, rows, cl = c2
    xs = x.cpu().numpy()
    r, (rn, bn) = plan.residual(b, x)
    r64 = oracle.residual_rows(C64, b.double().cpu().numpy(), xs, float(F32(SIGMA)), float(F32(K)), rows)
    scale, _ = oracle.kernel_rows(C64, np.abs(xs), float(F32(SIGMA)), float(F32(K)), rows)
    assert np.abs(r.cpu().numpy()[rows] - r64).max() <= 1e-11 * scale.max()
    assert rep["residual_true"] == pytest.approx(rn / bn, rel=1e-9)
    assert rep["precond_failed_blocks"] == 0
    # Krylov stagnation on a numerically singular system, not a missing interpolant (the
    # matrix is positive definite): on a 19,098-centre sector of this cloud 9.7% of |b| lies
    # in eigenvectors with |lambda| < 1e-6 lambda_max (0.06% without the position noise), and
    # GMRES does not resolve those components; measured 0.114 after these 50 iterations
    assert rep["residual_true"] < 0.2
    print(f"  C2 after 50 RAS-FGMRES iterations: relative residual {rep['residual_true']:.4f}")


def test_c2_grid_sampled_nodes(c2):
    rbf, plan, C, b, x, rep, C64, rows, cl = c2
    pad = DELTA + 3 * SIGMA
    lo = cl.points.min(0).astype(np.float64) - pad
    hi = cl.points.max(0).astype(np.float64) + pad
    f = plan.eval_grid(x, lo, hi, (256, 256, 256)).cpu().numpy().ravel().astype(np.float64)
    idx = np.random.default_rng(6).choice(256 ** 3, 10_000, replace=False)
    P = oracle.grid_nodes(lo.astype(np.float32), hi.astype(np.float32), (256, 256, 256), idx)
    f64 = oracle.eval_points(C64, x.cpu().numpy(), float(F32(SIGMA)), float(F32(K)), P)
    rng_f = f64.max() - f64.min()
    err = np.abs(f[idx] - f64).max()
    print(f"  C2 grid, 10,000 nodes: max error {err:.2e} = {err / rng_f:.2e} of the field range")
    assert err <= 1e-4 * rng_f
