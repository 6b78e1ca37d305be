"""The allocation-free product entry point (rbf_matvec_dense_noalloc).

It exists for callers that cannot allocate device memory when they call in (a
host that reserves its device memory up front, code inside another
framework's pool or a real-time loop).  Its scratch is a file-scope device
array shared by every call, so the test calls it twice in a row with different
inputs and compares each result with the plan-based rbf_matvec (k = 0), within
the 1e-5 relative tolerance of the other product tests.  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _centers(n, seed):
    cl = synth.sphere(n // 3 + 1, seed=seed)
    C = np.zeros((n, 4), dtype=np.float32)
    pts = np.concatenate([cl.points, 1.05 * cl.points, 0.95 * cl.points])[:n]
    C[:, :3] = pts
    return torch.from_numpy(C).cuda()


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_plan_product_twice():
    import paper_1305_5179_b300 as rbf
    L = rbf.lib()
    ctx = rbf.Context(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, sigma, seed) in enumerate([(4500, 0.1, 0), (2999, 0.07, 1)]):
        C = _centers(n, seed)
        z = torch.randn(n, device="cuda", generator=torch.Generator("cuda").manual_seed(seed))
        y = torch.full((n,), float("nan"), device="cuda")
        st = L.rbf_matvec_dense_noalloc(ctx._h, ctypes.c_void_p(C.data_ptr()), n, ctypes.c_float(sigma),
                                        ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)
        assert st == 0, rbf.lib().rbf_last_error(ctx._h)
        plan = rbf.Plan(ctx, C, sigma=sigma, k=0.0)
        ref = plan.matvec(z)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert _rel(y, ref) <= 1e-5, (call, _rel(y, ref))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1305_5179_b300 as rbf
    ctx = rbf.Context(0)
    n = rbf.NOALLOC_MAX_N + 1
    C = torch.zeros((n, 4), device="cuda")
    z = torch.zeros(n, device="cuda")
    y = torch.zeros(n, device="cuda")
    with pytest.raises(rbf.RbfError) as e:
        rbf.matvec_dense_noalloc(ctx, C, 0.1, z, y)
    assert e.value.status == 8 and "32768" in str(e.value)
