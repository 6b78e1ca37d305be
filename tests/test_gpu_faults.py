"""Failure detection without a GPU fault: a bounded wait that runs out and reports
RBF_ERR_TIMEOUT with the context still usable; a Cholesky block that fails and falls
back (or succeeds after shift escalation), reported; a solve stopped by its iteration
cap, reported as RBF_ERR_NOT_CONVERGED with its true residual."""
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


def c4(C):
    C32 = np.zeros((len(C), 4), dtype=np.float32)
    C32[:, :3] = C
    return torch.from_numpy(C32).cuda(), C32[:, :3].astype(np.float64)


def test_expired_wait_reports_timeout_and_the_context_survives(ctx, rbf):
    L = rbf.lib()
    for limit in (1_000_000, 20_000):            # 1 ms, 20 us
        assert L.rbf_probe_wait_expiry(ctx._h, limit, None) == 6      # RBF_ERR_TIMEOUT
        assert "bounded wait" in L.rbf_last_error(ctx._h).decode()
        # the next product on the same context runs and is right
        cl = synth.sphere(300, seed=3)
        C, _ = oracle.build_centers(cl.points, cl.normals, 0.05)
        Cd, C64 = c4(C)
        plan = rbf.Plan(ctx, Cd, sigma=0.1, k=6.0)
        z = np.random.default_rng(0).standard_normal(len(C)).astype(np.float32)
        y = plan.matvec(torch.from_numpy(z).cuda()).cpu().numpy().astype(np.float64)
        y64, _ = oracle.kernel_rows(C64, z.astype(np.float64), float(F32(0.1)), 6.0)
        assert np.linalg.norm(y - y64) <= 1e-5 * np.linalg.norm(y64)


def test_failed_cholesky_falls_back_or_escalates(ctx, rbf):
    """Exact duplicate centres make their blocks singular: without escalation some
    factorisations fail and those blocks act as the identity (counted); with escalation
    the shift grows until every block factorises."""
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (300, 3))
    C = np.concatenate([X, X[:150]])               # 150 exact duplicates
    Cd, _ = c4(C)
    plan = rbf.Plan(ctx, Cd, sigma=0.3, k=0.0)
    failed = plan.schwarz_setup(core=64, block=64, shift=0.0, escalate=False)
    assert failed > 0
    v = torch.from_numpy(rng.standard_normal(len(C)).astype(np.float32)).cuda()
    assert torch.isfinite(plan.schwarz_apply(v)).all()
    assert plan.schwarz_setup(core=64, block=64, shift=1e-7, escalate=True) == 0
    assert torch.isfinite(plan.schwarz_apply(v)).all()
    b = torch.from_numpy(rng.standard_normal(len(C)).astype(np.float32)).cuda()
    _, rep = plan.solve(b, precond="schwarz", core=64, block=64, shift=0.0, escalate=False, m=10, max_it=10,
                        fixed_iterations=True)
    assert rep["precond_failed_blocks"] == failed and rep["status"] == "RBF_OK"


def test_iteration_cap_reports_not_converged_with_the_true_residual(ctx, rbf, sphere_c1):
    C, b = oracle.build_centers(sphere_c1.points, sphere_c1.normals, 0.05)
    Cd, C64 = c4(C)
    b32 = b.astype(np.float32)
    plan = rbf.Plan(ctx, Cd, sigma=0.1, k=0.0)
    x, rep = plan.solve(torch.from_numpy(b32).cuda(), m=5, max_it=5, tol=1e-14)
    assert rep["status"] == "RBF_ERR_NOT_CONVERGED" and rep["converged"] == 0 and rep["iterations"] == 5
    r = oracle.residual_rows(C64, b32.astype(np.float64), x.cpu().numpy(), float(F32(0.1)), 0.0)
    assert rep["residual_true"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b32), rel=1e-6)
    assert 1e-14 < rep["residual_true"] < 1.0


def test_residual_share_beyond_the_accumulator_range_reports_range(ctx, rbf):
    """The double-float residual adds each row's source-side shares into a 128-bit
    fixed-point accumulator.  Weights of 1e15 make shares far above its limit
    min(2^44, 2^46 / (4 tiles)): the kernel runs normally, raises the context's error
    word and the call returns RBF_ERR_RANGE; the native float64 mode has no such
    limit and matches the oracle; the next call on the context is unaffected."""
    rng = np.random.default_rng(11)
    X = rng.uniform(0, 0.2, (3000, 3))
    Cd, C64 = c4(X)
    sigma, k = 0.02, 6.0
    plan = rbf.Plan(ctx, Cd, sigma=sigma, k=k)
    ntiles = plan.info()["nchunks"]
    lim = min(2.0 ** 44, 2.0 ** 46 / (4 * ntiles))
    b = torch.zeros(len(X), device="cuda")
    big = np.full(len(X), 1e15)
    assert 0.5 * big[0] > lim                     # one close pair already exceeds it
    with pytest.raises(rbf.RbfError) as e:
        plan.residual(b, torch.from_numpy(big).cuda(), mode="df")
    assert e.value.status == 9 and "range" in str(e.value)
    r64 = oracle.residual_rows(C64, np.zeros(len(X)), big, float(F32(sigma)), k)
    r, _ = plan.residual(b, torch.from_numpy(big).cuda(), mode="f64")
    assert np.abs(r.cpu().numpy() - r64).max() <= 1e-11 * np.abs(r64).max()
    x = rng.standard_normal(len(X))
    r, _ = plan.residual(b, torch.from_numpy(x).cuda(), mode="df")
    r64 = oracle.residual_rows(C64, np.zeros(len(X)), x, float(F32(sigma)), k)
    scale, _ = oracle.kernel_rows(C64, np.abs(x), float(F32(sigma)), k)     # sum_j |a_ij x_j|
    assert np.abs(r.cpu().numpy() - r64).max() <= 1e-11 * scale.max()
