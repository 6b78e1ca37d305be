"""Batched configuration at full size: 512 ellipsoids and tori with log-uniform sizes
500-20,000 points (seed 0), offsets +-0.02 -> 8.97M centres, sigma = 3 x each cloud's
mean nearest-neighbour spacing, cut-off 6 sigma, all problems in one batch.

The batched product and the batched solve run in the launch configuration the
benchmark times (tensor-core product over (problem, segment) items, block-Jacobi
subdomains of 32 with shift 1e-3, FGMRES(50), 50 steps in one CUDA graph).  Eight
clouds spread over the size range are checked against the FP64 oracle: the product
on sampled rows, and the true relative residual each cloud reports against the
oracle's float64 residual over all of the cloud's rows."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

K, DELTA = 6.0, 0.02


@pytest.fixture(scope="module")
def c4():
    import paper_1305_5179_b300 as rbf
    ctx = rbf.Context(0)
    clouds = synth.batch(nclouds=512, seed=0)
    Cs, bs, plans, sig = [], [], [], []
    for cl in clouds:
        C, b, _ = rbf.build_centers(ctx, torch.from_numpy(cl.points).cuda(), torch.from_numpy(cl.normals).cuda(),
                                    delta=DELTA)
        s = float(np.float32(cl.params["sigma"]))
        Cs.append(C)
        bs.append(b)
        sig.append(s)
        plans.append(rbf.Plan(ctx, C, sigma=s, k=K))
    batch = rbf.Batch(ctx, plans)
    sizes = np.array([len(C) for C in Cs])
    order = np.argsort(sizes)
    picks = [int(order[i]) for i in np.linspace(0, len(order) - 1, 8).astype(int)]   # smallest .. largest
    offs = np.concatenate([[0], np.cumsum(sizes)])
    return rbf, batch, Cs, bs, sig, picks, offs


def test_c4_batched_product_on_sampled_rows(c4):
    rbf, batch, Cs, bs, sig, picks, offs = c4
    assert batch.n == int(offs[-1]) and 8_500_000 < batch.n < 9_500_000
    z = torch.randn(batch.n, device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    y = batch.matvec(z).double().cpu().numpy()
    zh = z.double().cpu().numpy()
    rng = np.random.default_rng(5)
    for p in picks:
        n = len(Cs[p])
        rows = rng.choice(n, min(n, 400), replace=False)
        C64 = Cs[p][:, :3].double().cpu().numpy()
        y64, _ = oracle.kernel_rows(C64, zh[offs[p]:offs[p] + n], sig[p], K, rows)
        err = np.linalg.norm(y[offs[p]:offs[p] + n][rows] - y64) / np.linalg.norm(y64)
        assert err <= 1e-5, (p, n, err)


def test_c4_batched_solve_residuals_against_the_oracle(c4, capsys):
    rbf, batch, Cs, bs, sig, picks, offs = c4
    b = torch.cat(bs)
    x, reps, st = batch.solve(b, m=50, max_it=50, precond="schwarz", core=32, block=32, shift=1e-3, escalate=True,
                              fixed_iterations=True)
    assert st["precond_failed_blocks"] == 0 and all(r["iterations"] == 50 for r in reps)
    xs = x.cpu().numpy()
    out = []
    for p in picks:
        n = len(Cs[p])
        C64 = Cs[p][:, :3].double().cpu().numpy()
        b64 = bs[p].double().cpu().numpy()
        r64 = oracle.residual_rows(C64, b64, xs[offs[p]:offs[p] + n], sig[p], K)
        true = float(np.linalg.norm(r64) / np.linalg.norm(b64))
        out.append((n, reps[p]["residual_true"], true))
        assert reps[p]["residual_true"] == pytest.approx(true, rel=1e-6, abs=1e-12), (p, n)
    with capsys.disabled():
        print("\n  C4, 8 clouds (centres, reported residual, oracle residual):",
              ", ".join(f"{n}: {r:.3e} / {t:.3e}" for n, r, t in out))
    med = float(np.median([r["residual_true"] for r in reps]))
    assert med < 1e-3          # measured on B300: median 4.5e-4 over the 512 clouds
