"""The allocation-free product entry point (rbf_matvec_dense_noalloc).

It exists for callers that cannot allocate device memory when they call in (a
host that reserves its device memory up front, code inside another
framework's pool or a real-time loop).  Its scratch is a file-scope device
array shared by every call, resolved when the context is created.  The tests
call it twice in a row with different inputs on a fresh context, check that
free device memory does not change across the calls, and compare each result
with the float64 oracle's dense product and with the plan-based rbf_matvec
(k = 0), within the 1e-5 relative tolerance of the other product tests.  This
file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _centers(n, seed):
    cl = synth.sphere(n // 3 + 1, seed=seed)
    C = np.zeros((n, 4), dtype=np.float32)
    pts = np.concatenate([cl.points, 1.05 * cl.points, 0.95 * cl.points])[:n]
    C[:, :3] = pts
    return C


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_the_oracle_twice_without_allocating():
    import paper_1305_5179_b300 as rbf
    L = rbf.lib()
    cases = [(4500, 0.1, 0), (2999, 0.07, 1)]
    inputs = []
    for n, sigma, seed in cases:                  # every buffer exists before the calls
        C = _centers(n, seed)
        z = np.random.default_rng(seed).standard_normal(n).astype(np.float32)
        inputs.append((C, z, torch.from_numpy(C).cuda(), torch.from_numpy(z).cuda(),
                       torch.full((n,), float("nan"), device="cuda")))
    ctx = rbf.Context(0)                          # fresh context: the scratch is resolved here
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for (n, sigma, _), (_, _, Cd, zd, yd) in zip(cases, inputs):
        st = L.rbf_matvec_dense_noalloc(ctx._h, ctypes.c_void_p(Cd.data_ptr()), n, ctypes.c_float(sigma),
                                        ctypes.c_void_p(zd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), stream)
        assert st == 0, L.rbf_last_error(ctx._h)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for call, ((n, sigma, _), (C, z, Cd, zd, yd)) in enumerate(zip(cases, inputs)):
        y = yd.cpu().numpy()
        assert np.isfinite(y).all()
        y64, _ = oracle.kernel_rows(C[:, :3].astype(np.float64), z.astype(np.float64),
                                    float(np.float32(sigma)), 0.0)
        assert _rel(y, y64) <= 1e-5, (call, _rel(y, y64))
        ref = rbf.Plan(ctx, Cd, sigma=sigma, k=0.0).matvec(zd).cpu().numpy()
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
