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
    assert rep["residual_true"] == pytest.approx(float(np.linalg.norm(r.cpu().numpy()) / np.linalg.norm(
        b.double().cpu().numpy())), rel=1e-9)


def test_c3_refinement_residuals_agree_at_every_restart(c3, capsys):
    """FP64 refinement (every FGMRES(50) restart recomputes b - A~ x in double-float): the
    library's true residual after 50, 100, 150 and 200 iterations agrees with the
    oracle's float64 rows (10,000 sampled) to 1e-11 of max sum |a x| at every restart,
    the reported relative residual equals the norm of the library's residual vector,
    and every restart lowers it.  The refinement does not stagnate within reach: on
    B300 the same solve measured 5.8e-5 after 400, 1.9e-5 after 1,000 and 9.0e-6 after
    2,000 iterations (about 0.12 s per iteration), so node residual 1e-6 on this
    configuration is a matter of many thousands of iterations, not of precision."""
    rbf, ctx, plan, C, b, C64, rows = c3
    bh = b.double().cpu().numpy()
    hist = []
    for k in (50, 100, 150, 200):
        x, rep = plan.solve(b, m=50, max_it=k, fixed_iterations=True)
        assert rep["iterations"] == k
        r, (rn, bn) = plan.residual(b, x)
        xs = x.cpu().numpy()
        r64 = oracle.residual_rows(C64, bh, xs, float(F32(SIGMA)), float(F32(K)), rows)
        scale, _ = oracle.kernel_rows(C64, np.abs(xs), float(F32(SIGMA)), float(F32(K)), rows)
        err = np.abs(r.cpu().numpy()[rows] - r64).max() / scale.max()
        assert err <= 1e-11, (k, err)
        assert rep["residual_true"] == pytest.approx(rn / bn, rel=1e-9)
        hist.append((k, rep["residual_true"], float(np.linalg.norm(r64) / np.linalg.norm(bh[rows])), err))
    with capsys.disabled():
        print("\n  C3 refinement (iterations, true relative residual, sampled-row oracle residual, row error):",
              ", ".join(f"{k}: {t:.3e} / {o:.3e} / {e:.1e}" for k, t, o, e in hist))
    t = [h[1] for h in hist]
    assert all(b_ < a_ for a_, b_ in zip(t, t[1:]))                     # every restart gains
    assert t[-1] < 1e-3
