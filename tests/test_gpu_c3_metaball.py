"""Mixed-precision configuration at full size: 4,000,000 points on a metaball
surface (8 seeded Gaussian blobs, density proportional to 1 + 9 u^3 in height),
offsets +-0.005 -> 12,000,000 centres, sigma 0.01, cut-off 6 sigma.  The float32
product, the float64-class (double-float) true residual and the solver's
refinement are checked against the FP64 oracle on 10,000 sampled rows."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

F32 = np.float32
SIGMA, K, DELTA = 0.01, 6.0, 0.005


@pytest.fixture(scope="module")
def c3():
    import paper_1305_5179_b300 as rbf
    ctx = rbf.Context(0)
    cl = synth.metaball(4_000_000, seed=0)
    pts = torch.from_numpy(cl.points).cuda()
    nrm = torch.from_numpy(cl.normals).cuda()
    C, b, _ = rbf.build_centers(ctx, pts, nrm, delta=DELTA)
    plan = rbf.Plan(ctx, C, sigma=SIGMA, k=K)
    C64 = C[:, :3].double().cpu().numpy()
    rows = np.random.default_rng(3).choice(len(C64), 10_000, replace=False)
    return rbf, ctx, plan, C, b, C64, rows


def test_c3_product_on_sampled_rows(c3):
    rbf, ctx, plan, C, b, C64, rows = c3
    assert C.shape[0] == 12_000_000
    z = torch.randn(C.shape[0], device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    y = plan.matvec(z).double().cpu().numpy()
    y64, _ = oracle.kernel_rows(C64, z.double().cpu().numpy(), float(F32(SIGMA)), float(F32(K)), rows)
    err = np.linalg.norm(y[rows] - y64) / np.linalg.norm(y64)
    print(f"\n  C3 float32 product, 10,000 sampled rows: relative error {err:.2e}")
    assert err <= 1e-5


def test_c3_refinement_residual_on_sampled_rows(c3):
    rbf, ctx, plan, C, b, C64, rows = c3
    x, rep = plan.solve(b, m=20, max_it=20, fixed_iterations=True)
    r, _ = plan.residual(b, x)
    xs = x.cpu().numpy()
    r64 = oracle.residual_rows(C64, b.double().cpu().numpy(), xs, float(F32(SIGMA)), float(F32(K)), rows)
    scale, _ = oracle.kernel_rows(C64, np.abs(xs), float(F32(SIGMA)), float(F32(K)), rows)
    err = np.abs(r.cpu().numpy()[rows] - r64).max() / scale.max()
    print(f"  C3 double-float residual, 10,000 sampled rows: max error {err:.2e} of max sum|a x|; "
          f"true relative residual after 20 iterations {rep['residual_true']:.3e}")
    assert err <= 1e-11
    assert np.isfinite(rep["residual_true"]) and rep["residual_true"] < 1.0
