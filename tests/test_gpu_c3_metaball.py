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


LAM5 = 1.0     # shift of the block solves the network learns (relative to the unit diagonal)


def _c5_train(rbf, ctx, plans, per_plan, seed):
    """200,000 exact float64 shifted block solves (lambda LAM5) drawn from the training
    plans, and the network trained on them (40 epochs of 512 at step size 3e-4: with 20
    epochs at 1e-3 the iterations to 1e-4 on C3 varied from 135 to 234 with the order of
    the same samples; at 3e-4 both orders gave 146-150)."""
    Xs, Ys = [], []
    rng = np.random.default_rng(seed)
    for plan in plans:
        bid = torch.from_numpy(rng.integers(0, plan.n // 64, per_plan).astype(np.int32)).cuda()
        R = torch.from_numpy(rng.standard_normal((per_plan, 64)).astype(np.float32)).cuda()
        X, Y, failed = rbf.mlp_make_data(plan, LAM5, bid, R)
        assert failed == 0
        Xs.append(X)
        Ys.append(Y)
    X = torch.cat(Xs)
    Y = torch.cat(Ys)
    perm = torch.from_numpy(rng.permutation(X.shape[0])).cuda()
    X, Y = X[perm].contiguous(), Y[perm].contiguous()
    net = rbf.MLP(ctx, synth.mlp_init(seed=1))
    l0, _ = net.loss_grad(X[:8192].contiguous(), Y[:8192].contiguous(), grad=False)
    hist = net.train(X, Y, epochs=40, batch=512, lr=3e-4)
    l1, _ = net.loss_grad(X[:8192].contiguous(), Y[:8192].contiguous(), grad=False)
    return net, X.shape[0], (l0, hist[0], hist[-1], l1)


def test_c5_learned_preconditioner_on_c2_and_c3(c3, capsys):
    """Configuration 5: the network trained on 200,000 exact float64 block solves from
    seeded training clouds disjoint from the test clouds (torus sector and metaball of
    seed 1000, at the densities of configurations 2 and 3), then used as the FGMRES(50)
    preconditioner on the configuration-2 torus (3,000,000 centres) and the
    configuration-3 metaball (12,000,000 centres), against no preconditioner and the
    exact shifted block solves it learns (subdomains of 64, shift LAM5).

    Node residual 1e-6 is out of reach within these budgets for every method, so the
    comparison is (a) the true residual after 50 iterations and (b) on C3, relative
    residual 1e-4: the network reaches it, and the plain solve has not after as many
    iterations.  The numbers measured on B300 are in the print and in the design notes."""
    rbf, ctx, plan3, C3, b3, _, _ = c3
    sector = synth.torus(95_492, noise=1e-3, seed=1000, theta_max=0.6)
    Ct, _, _ = rbf.build_centers(ctx, torch.from_numpy(sector.points).cuda(), torch.from_numpy(sector.normals).cuda(),
                                 delta=0.01)
    meta = synth.metaball(4_000_000, seed=1000)
    Cm, _, _ = rbf.build_centers(ctx, torch.from_numpy(meta.points).cuda(), torch.from_numpy(meta.normals).cuda(),
                                 delta=DELTA)
    pt = rbf.Plan(ctx, Ct, sigma=0.02, k=K)
    pm = rbf.Plan(ctx, Cm, sigma=SIGMA, k=K)
    net, ns, hist = _c5_train(rbf, ctx, [pt, pm], 100_000, seed=5)
    assert ns == 200_000 and hist[3] < 0.8 * hist[0]          # loss on 8,192 samples, after vs before
    del pt, pm, Cm, Ct
    torus = synth.torus(1_000_000, noise=1e-3, seed=0)
    C2, b2, _ = rbf.build_centers(ctx, torch.from_numpy(torus.points).cuda(), torch.from_numpy(torus.normals).cuda(),
                                  delta=0.01)
    plan2 = rbf.Plan(ctx, C2, sigma=0.02, k=K)
    methods = (("none", dict(precond="none")),
               ("ras64", dict(precond="schwarz", core=64, block=64, shift=LAM5)),
               ("learned", dict(precond="mlp", mlp=net, mlp_lambda=LAM5)))
    out = {}
    for name, plan, b in (("C2", plan2, b2), ("C3", plan3, b3)):
        res = {}
        for meth, kw in methods:
            x, rep = plan.solve(b, m=50, max_it=50, tol=1e-6, **kw)
            assert rep["iterations"] == 50 and not rep["converged"]
            res[meth] = (rep["residual_true"], rep["ms_setup"] + rep["ms_solve"], rep["precond_failed_blocks"])
        out[name] = res
    tol = {}
    for meth in ("learned", "ras64"):               # time to 1e-4 on C3
        x, rep = plan3.solve(b3, m=50, max_it=300, tol=1e-4, **dict(methods)[meth])
        tol[meth] = (bool(rep["converged"]), rep["iterations"], rep["residual_true"],
                     rep["ms_setup"] + rep["ms_solve"])
    k = tol["learned"][1]
    x, rep = plan3.solve(b3, m=50, max_it=k, fixed_iterations=True)   # plain, as many iterations
    tol["none"] = (bool(rep["residual_true"] <= 1e-4), rep["iterations"], rep["residual_true"],
                   rep["ms_setup"] + rep["ms_solve"])
    with capsys.disabled():
        print("\n  C5 (true residual after 50 iterations, ms, fallback blocks):", out,
              f"training loss (before, epoch 1, epoch 40, after) {[round(float(h), 4) for h in hist]} on {ns} solves")
        print("  C5 on C3 to 1e-4 (converged, iterations, residual, ms; plain after the network's iterations):", tol)
    for name in ("C2", "C3"):
        assert all(np.isfinite(v[0]) for v in out[name].values()) and out[name]["learned"][2] == 0
    g2 = {k2: out["C2"]["none"][0] / v[0] for k2, v in out["C2"].items()}
    g3 = {k2: out["C3"]["none"][0] / v[0] for k2, v in out["C3"].items()}
    assert 0.8 <= g2["learned"] <= 1.2                                 # C2: no gain
    assert g3["learned"] > 1.5 and g3["ras64"] > 1.5                   # C3: both gain
    assert tol["learned"][0] and tol["ras64"][0]
    assert not tol["none"][0]          # the plain solve is still above 1e-4 after the network's iterations
    assert tol["learned"][1] < 200      # measured: 146 (plain FGMRES: 272)
