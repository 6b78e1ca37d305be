"""Python binding of ``librbf.so`` (the C ABI in ``include/rbf.h``).

Argument marshalling only: torch supplies device memory and the current CUDA
stream; every step of the computation runs in the library's CUDA kernels.
There is no fallback: if the shared library is missing or no CUDA device is
present, calls raise.

Typical use (Algorithm 1 of the paper, steps 1-3)::

    import torch, paper_1305_5179_b300 as rbf
    ctx = rbf.Context(0)
    C, b, delta = rbf.build_centers(ctx, pts, nrm, delta=0.01)     # step 1
    plan = rbf.Plan(ctx, C, sigma=0.02, k=6.0)                     # binning
    x, rep = plan.solve(b, precond="schwarz", core=96, block=128)  # step 2
    f = plan.eval_grid(x, lo, hi, dims)                            # step 3
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "librbf.so")

RBF_OK = 0
STATUS = {0: "RBF_OK", 1: "RBF_ERR_INVALID", 2: "RBF_ERR_OOM", 3: "RBF_ERR_CUDA", 4: "RBF_ERR_NOT_CONVERGED",
          5: "RBF_ERR_BREAKDOWN", 6: "RBF_ERR_TIMEOUT", 7: "RBF_ERR_NOT_SPD", 8: "RBF_ERR_UNSUPPORTED",
          9: "RBF_ERR_RANGE"}
PRECOND = {"none": 0, "schwarz": 1, "mlp": 2}
RESIDUAL = {"df": 0, "f64": 1}

# every entry point declared in include/rbf.h
EXPORTS = (
    "rbf_version", "rbf_launch_count", "rbf_probe_peaks", "rbf_probe_wait_expiry", "rbf_status_string", "rbf_ctx_create", "rbf_ctx_destroy", "rbf_last_error",
    "rbf_build_centers", "rbf_plan_create", "rbf_plan_destroy", "rbf_plan_get_info", "rbf_plan_export_binning",
    "rbf_matvec", "rbf_count_pairs", "rbf_count_candidate_pairs", "rbf_residual",
    "rbf_plan_assemble", "rbf_plan_release_csr", "rbf_plan_export_csr", "rbf_spmv",
    "rbf_schwarz_setup", "rbf_schwarz_apply",
    "rbf_plan_solve", "rbf_solve", "rbf_plan_eval_grid", "rbf_count_grid_pairs", "rbf_count_grid_candidate_pairs",
    "rbf_eval_grid",
    "rbf_density_measures", "rbf_isosurface",
    "rbf_matvec_dense_noalloc",
    "rbf_batch_create", "rbf_batch_destroy", "rbf_batch_size", "rbf_batch_matvec", "rbf_batch_solve",
    "rbf_batch_autotune",
    "rbf_mlp_create", "rbf_mlp_destroy", "rbf_mlp_get_params", "rbf_mlp_make_data", "rbf_mlp_forward",
    "rbf_mlp_loss_grad", "rbf_mlp_train",
)
MLP_NPARAMS = 148032


class RbfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanParams(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_float), ("k", ctypes.c_float), ("cells_per_cutoff", ctypes.c_int),
                ("levels", ctypes.c_int), ("product", ctypes.c_int), ("kernel", ctypes.c_int),
                ("beta", ctypes.c_float), ("cell_edge", ctypes.c_float)]


KERNELS = {"gaussian": 0, "imq": 1}


def _plan_params(sigma, k, cells_per_cutoff=1, levels=3, product="tc", kernel="gaussian", beta=0.0,
                 cell_edge=0.0):
    return PlanParams(float(sigma), float(k), int(cells_per_cutoff), int(levels), PRODUCTS[product],
                      KERNELS[kernel], float(beta), float(cell_edge))


PRODUCTS = {"tc": 0, "simt": 1}


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ncells", ctypes.c_int64), ("nblocks", ctypes.c_int64),
                ("nchunks", ctypes.c_int64), ("pairlist_len", ctypes.c_int64), ("nsegments", ctypes.c_int64),
                ("nbits", ctypes.c_int), ("levels", ctypes.c_int), ("lo", ctypes.c_float * 3),
                ("inv", ctypes.c_float), ("sigma", ctypes.c_float), ("k", ctypes.c_float),
                ("cell_edge", ctypes.c_double), ("symmetric", ctypes.c_int)]


class SchwarzParams(ctypes.Structure):
    _fields_ = [("core", ctypes.c_int), ("block", ctypes.c_int), ("shift", ctypes.c_float),
                ("restricted", ctypes.c_int), ("escalate", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("max_it", ctypes.c_int), ("tol", ctypes.c_double), ("precond", ctypes.c_int),
                ("schwarz", SchwarzParams), ("fixed_iterations", ctypes.c_int),
                ("true_residual_each_restart", ctypes.c_int), ("residual_mode", ctypes.c_int),
                ("mlp", ctypes.c_void_p), ("mlp_lambda", ctypes.c_float), ("mlp_initial_guess", ctypes.c_int),
                ("assembled", ctypes.c_int)]


class TrainParams(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float)]


class Report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
                ("precond_failed_blocks", ctypes.c_int), ("residual_estimate", ctypes.c_double),
                ("residual_true", ctypes.c_double), ("ms_setup", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("matvec_pairs", ctypes.c_int64), ("matvec_launches", ctypes.c_int),
                ("residual_launches", ctypes.c_int), ("ms_matvec", ctypes.c_double), ("ms_residual", ctypes.c_double),
                ("ms_precond", ctypes.c_double), ("guess_scale", ctypes.c_double), ("guess_residual", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ProbeResult(ctypes.Structure):
    _fields_ = [("num_sms", ctypes.c_int), ("sm_mhz", ctypes.c_double), ("ex2_per_clk_sm", ctypes.c_double),
                ("ffma_per_clk_sm", ctypes.c_double), ("ffma2_lanes_per_clk_sm", ctypes.c_double),
                ("mma_commit_cycles", ctypes.c_double), ("mma_commit4_cycles", ctypes.c_double),
                ("dfma_per_clk_sm", ctypes.c_double)]


class Density(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("h_max", ctypes.c_double), ("mean_nn", ctypes.c_double),
                ("fill", ctypes.c_double), ("sigma_q", ctypes.c_double), ("sigma_fill", ctypes.c_double),
                ("sigma_hmax", ctypes.c_double), ("cell", ctypes.c_float)]


class BatchStats(ctypes.Structure):
    _fields_ = [("ms_setup", ctypes.c_double), ("ms_solve", ctypes.c_double), ("graph_nodes", ctypes.c_int64),
                ("recaptured", ctypes.c_int), ("persistent_ctas", ctypes.c_int), ("work_items", ctypes.c_int64),
                ("converged", ctypes.c_int), ("worst_residual", ctypes.c_double),
                ("precond_failed_blocks", ctypes.c_int)]


class Grid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("dims", ctypes.c_int64 * 3)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load ``librbf.so`` (built by ``paper_1305_5179_b300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise ImportError(f"{LIBPATH} is missing: run `python -m paper_1305_5179_b300.build`")
    L = ctypes.CDLL(LIBPATH)
    P, I64, I, F, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double
    sig = {
        "rbf_version": ([], I),
        "rbf_launch_count": ([], I64),
        "rbf_probe_peaks": ([I, ctypes.POINTER(ProbeResult)], I),
        "rbf_density_measures": ([P, P, I64, P, I64, F, P, ctypes.POINTER(Density), P], I),
        "rbf_isosurface": ([P, P, ctypes.POINTER(Grid), F, P, I64, F, P, I64, ctypes.POINTER(I64), P], I),
        "rbf_status_string": ([I], ctypes.c_char_p),
        "rbf_ctx_create": ([ctypes.POINTER(P), I], I),
        "rbf_ctx_destroy": ([P], I),
        "rbf_last_error": ([P], ctypes.c_char_p),
        "rbf_build_centers": ([P, P, P, I64, F, F, P, P, ctypes.POINTER(F), P], I),
        "rbf_plan_create": ([P, P, I64, ctypes.POINTER(PlanParams), ctypes.POINTER(P), P], I),
        "rbf_plan_destroy": ([P], I),
        "rbf_plan_get_info": ([P, ctypes.POINTER(PlanInfo)], I),
        "rbf_plan_export_binning": ([P, P, P, P, P, P], I),
        "rbf_matvec": ([P, P, P, P], I),
        "rbf_count_pairs": ([P, ctypes.POINTER(I64), P], I),
        "rbf_residual": ([P, P, P, P, ctypes.POINTER(D), I, P], I),
        "rbf_schwarz_setup": ([P, ctypes.POINTER(SchwarzParams), ctypes.POINTER(I64), P], I),
        "rbf_schwarz_apply": ([P, P, P, P], I),
        "rbf_plan_solve": ([P, P, ctypes.POINTER(SolveParams), P, ctypes.POINTER(Report), P], I),
        "rbf_solve": ([P, P, P, I64, ctypes.POINTER(PlanParams), ctypes.POINTER(SolveParams), P,
                       ctypes.POINTER(Report), P], I),
        "rbf_plan_eval_grid": ([P, P, ctypes.POINTER(Grid), P, P], I),
        "rbf_count_grid_pairs": ([P, ctypes.POINTER(Grid), ctypes.POINTER(I64), P], I),
        "rbf_count_grid_candidate_pairs": ([P, ctypes.POINTER(Grid), ctypes.POINTER(I64), P], I),
        "rbf_matvec_dense_noalloc": ([P, P, I64, F, P, P, P], I),
        "rbf_mlp_create": ([P, P, ctypes.POINTER(P)], I),
        "rbf_mlp_destroy": ([P], I),
        "rbf_mlp_get_params": ([P, P], I),
        "rbf_mlp_make_data": ([P, F, P, P, I64, P, P, ctypes.POINTER(I64), P], I),
        "rbf_mlp_forward": ([P, P, I64, P, I, P], I),
        "rbf_mlp_loss_grad": ([P, P, P, I64, ctypes.POINTER(D), P, P], I),
        "rbf_mlp_train": ([P, P, P, I64, ctypes.POINTER(TrainParams), P, P], I),
        "rbf_batch_create": ([P, ctypes.POINTER(P), I, ctypes.POINTER(P), P], I),
        "rbf_batch_destroy": ([P], I),
        "rbf_batch_size": ([P], I64),
        "rbf_batch_matvec": ([P, P, P, P], I),
        "rbf_batch_solve": ([P, P, ctypes.POINTER(SolveParams), P, P, ctypes.POINTER(BatchStats), P], I),
        "rbf_batch_autotune": ([P, P, ctypes.POINTER(SolveParams), P, I, ctypes.POINTER(I), P, P], I),
        "rbf_eval_grid": ([P, P, P, I64, ctypes.POINTER(PlanParams), ctypes.POINTER(Grid), P, P], I),
        "rbf_plan_assemble": ([P, I64, ctypes.POINTER(I64), ctypes.POINTER(I64), P], I),
        "rbf_count_candidate_pairs": ([P, ctypes.POINTER(I64), P], I),
        "rbf_probe_wait_expiry": ([P, ctypes.c_uint64, P], I),
        "rbf_plan_release_csr": ([P], I),
        "rbf_plan_export_csr": ([P, P, P, P, P], I),
        "rbf_spmv": ([P, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _req(t, dtype, name, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return t


class Context:
    """A library context bound to one CUDA device."""

    def __init__(self, device: int = 0):
        import weakref
        self._h = ctypes.c_void_p()
        self._dependents = weakref.WeakSet()    # plans, batches, networks: closed before the context
        st = lib().rbf_ctx_create(ctypes.byref(self._h), int(device))
        if st != RBF_OK:
            raise RbfError(st, f"rbf_ctx_create(device={device}) failed")
        self.device = int(device)

    def check(self, st: int, what: str, allow=()):
        if st != RBF_OK and st not in allow:
            msg = lib().rbf_last_error(self._h)
            raise RbfError(st, f"{what}: {msg.decode() if msg else ''}")
        return st

    def close(self):
        if self._h:
            for d in list(getattr(self, "_dependents", ())):
                d.close()
            lib().rbf_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().rbf_launch_count())


def probe_peaks(device: int = 0) -> dict:
    """Measured MUFU.EX2 / FFMA / FFMA2 rates per SM per clock and the SM clock."""
    r = ProbeResult()
    st = lib().rbf_probe_peaks(int(device), ctypes.byref(r))
    if st != RBF_OK:
        raise RbfError(st, "rbf_probe_peaks")
    return {f: getattr(r, f) for f, _ in r._fields_}


def isosurface(ctx: Context, f, lo, hi, iso: float = 0.0, points=None, band: float = 0.0, stream=None):
    """Step 4 without rendering: the triangles (ntri, 3, 3) of {f = iso} on the grid
    field f of shape (Gz, Gy, Gx) with nodes lo + i (hi - lo)/(G - 1); with data
    points (n, 4) and band > 0, only cells whose centre is within band of a point."""
    import torch
    _req(f, torch.float32, "f")
    if f.dim() != 3:
        raise ValueError("f must be (Gz, Gy, Gx)")
    npts = 0
    if points is not None:
        _req(points, torch.float32, "points")
        if points.dim() != 2 or points.shape[1] != 4:
            raise ValueError("points must be (n, 4) float32")
        npts = int(points.shape[0])
    pp = _ptr(points) if npts else None
    dims = (int(f.shape[2]), int(f.shape[1]), int(f.shape[0]))
    g = _grid(lo, hi, dims)
    n = ctypes.c_int64(0)
    ctx.check(lib().rbf_isosurface(ctx._h, _ptr(f), ctypes.byref(g), float(iso), pp, npts, float(band), None, 0,
                                   ctypes.byref(n), _stream(stream)), "rbf_isosurface")
    tri = torch.empty((max(1, n.value), 3, 3), dtype=torch.float32, device=f.device)
    if n.value:
        ctx.check(lib().rbf_isosurface(ctx._h, _ptr(f), ctypes.byref(g), float(iso), pp, npts, float(band),
                                       _ptr(tri), n.value, ctypes.byref(n), _stream(stream)), "rbf_isosurface")
    return tri[:n.value]


def density_measures(ctx: Context, points, probes=None, cell: float = 0.0, return_nn: bool = False, stream=None):
    """Density measures of Sec. IV on device float4 points (n, 4): separation distance,
    h_max, mean nearest-neighbour distance, fill distance over probe points (m, 4),
    and the paper's sigma rules.  Returns a dict (and the nearest-neighbour
    distances when return_nn)."""
    import torch
    _req(points, torch.float32, "points")
    if points.dim() != 2 or points.shape[1] != 4:
        raise ValueError("points must be (n, 4) float32")
    n = int(points.shape[0])
    m = 0
    if probes is not None:
        _req(probes, torch.float32, "probes")
        if probes.dim() != 2 or probes.shape[1] != 4:
            raise ValueError("probes must be (m, 4) float32")
        m = int(probes.shape[0])
    nn = torch.empty(n, dtype=torch.float32, device=points.device) if return_nn else None
    d = Density()
    ctx.check(lib().rbf_density_measures(ctx._h, _ptr(points), n, _ptr(probes) if m else None, m, float(cell),
                                         _ptr(nn) if return_nn else None, ctypes.byref(d), _stream(stream)),
              "rbf_density_measures")
    out = {f: getattr(d, f) for f, _ in d._fields_}
    return (out, nn) if return_nn else out


def build_centers(ctx: Context, pts, nrm, delta: float = 0.0, target: float = 0.0, stream=None):
    """Step 1: extended set [X; X + delta n; X - delta n] (float4) and targets."""
    import torch
    _req(pts, torch.float32, "pts")
    _req(nrm, torch.float32, "nrm", pts.numel())
    N = pts.numel() // 3
    C = torch.empty((3 * N, 4), dtype=torch.float32, device=pts.device)
    b = torch.empty(3 * N, dtype=torch.float32, device=pts.device)
    d = ctypes.c_float(0)
    ctx.check(lib().rbf_build_centers(ctx._h, _ptr(pts), _ptr(nrm), N, float(delta), float(target), _ptr(C), _ptr(b),
                                      ctypes.byref(d), _stream(stream)), "rbf_build_centers")
    return C, b, float(d.value)


def _grid(lo, hi, dims) -> Grid:
    g = Grid()
    for i in range(3):
        g.lo[i] = float(lo[i])
        g.hi[i] = float(hi[i])
        g.dims[i] = int(dims[i])
    return g


def _solve_params(m=50, max_it=500, tol=1e-6, precond="none", core=96, block=128, shift=1e-4, restricted=True,
                  escalate=True, fixed_iterations=False, true_residual_each_restart=True,
                  residual="df", mlp=None, mlp_lambda=1e-2, mlp_initial_guess=False,
                  assembled=False) -> SolveParams:
    sp = SolveParams()
    sp.m, sp.max_it, sp.tol = int(m), int(max_it), float(tol)
    sp.precond = PRECOND[precond] if isinstance(precond, str) else int(precond)
    sp.schwarz = SchwarzParams(int(core), int(block), float(shift), int(bool(restricted)), int(bool(escalate)))
    sp.fixed_iterations = int(bool(fixed_iterations))
    sp.true_residual_each_restart = int(bool(true_residual_each_restart))
    sp.residual_mode = RESIDUAL[residual]
    sp.mlp = mlp._h.value if mlp is not None else None
    sp.mlp_lambda = float(mlp_lambda)
    sp.mlp_initial_guess = int(bool(mlp_initial_guess))
    sp.assembled = int(bool(assembled))
    return sp


class Plan:
    """The matrix-free truncated Gaussian operator over a fixed set of centres."""

    def __init__(self, ctx: Context, centers, sigma: float, k: float = 0.0, cells_per_cutoff: int = 1,
                 levels: int = 3, product: str = "tc", kernel: str = "gaussian", beta: float = 0.0,
                 cell_edge: float = 0.0, stream=None):
        """kernel "gaussian" (exp(-r^2/(2 sigma^2))) or "imq" ((1 + r^2/sigma^2)^-beta, Table I);
        cell_edge > 0 fixes the binning's cell edge (0: the default rule)."""
        import torch
        _req(centers, torch.float32, "centers")
        if centers.dim() != 2 or centers.shape[1] != 4:
            raise ValueError("centers must be (n, 4) float32")
        self.ctx = ctx
        self.n = int(centers.shape[0])
        self.device = centers.device
        self.params = _plan_params(sigma, k, cells_per_cutoff, levels, product, kernel, beta, cell_edge)
        self._h = ctypes.c_void_p()
        ctx.check(lib().rbf_plan_create(ctx._h, _ptr(centers), self.n, ctypes.byref(self.params),
                                        ctypes.byref(self._h), _stream(stream)), "rbf_plan_create")
        ctx._dependents.add(self)

    def close(self):
        if self._h:
            lib().rbf_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        pi = PlanInfo()
        self.ctx.check(lib().rbf_plan_get_info(self._h, ctypes.byref(pi)), "rbf_plan_get_info")
        d = {f: getattr(pi, f) for f, _ in pi._fields_}
        d["lo"] = [pi.lo[i] for i in range(3)]
        return d

    def export_binning(self, stream=None):
        import torch
        info = self.info()
        perm = torch.empty(self.n, dtype=torch.int32, device=self.device)
        keys = torch.empty(self.n, dtype=torch.int32, device=self.device)
        cs = torch.empty(info["ncells"], dtype=torch.int32, device=self.device)
        ce = torch.empty(info["ncells"], dtype=torch.int32, device=self.device)
        self.ctx.check(lib().rbf_plan_export_binning(self._h, _ptr(perm), _ptr(keys), _ptr(cs), _ptr(ce),
                                                     _stream(stream)), "rbf_plan_export_binning")
        return perm, keys, cs, ce

    def matvec(self, z, out=None, stream=None):
        import torch
        _req(z, torch.float32, "z", self.n)
        y = torch.empty_like(z) if out is None else _req(out, torch.float32, "out", self.n)
        self.ctx.check(lib().rbf_matvec(self._h, _ptr(z), _ptr(y), _stream(stream)), "rbf_matvec")
        return y

    def count_pairs(self, stream=None) -> int:
        c = ctypes.c_int64(0)
        self.ctx.check(lib().rbf_count_pairs(self._h, ctypes.byref(c), _stream(stream)), "rbf_count_pairs")
        return int(c.value)

    def assemble(self, max_bytes: int = 0, stream=None):
        """Build the assembled matrix (Algorithm 2, CSR in binned order, kept by the plan).
        Returns (nnz, stored); raises RbfError (RBF_ERR_OOM) when it would not fit, with
        ``.nnz`` / ``.stored`` set on the exception."""
        nnz, stored = ctypes.c_int64(0), ctypes.c_int64(0)
        st = lib().rbf_plan_assemble(self._h, int(max_bytes), ctypes.byref(nnz), ctypes.byref(stored),
                                     _stream(stream))
        try:
            self.ctx.check(st, "rbf_plan_assemble")
        except RbfError as e:
            e.nnz, e.stored = int(nnz.value), int(stored.value)
            raise
        self.csr_stored = int(stored.value)
        return int(nnz.value), int(stored.value)

    def release_csr(self):
        self.ctx.check(lib().rbf_plan_release_csr(self._h), "rbf_plan_release_csr")

    def export_csr(self, stream=None):
        """(row_ptr int64 n+1, col int32, val float32) of the assembled matrix, binned order."""
        import torch
        stored = getattr(self, "csr_stored", None)
        if stored is None:
            raise RbfError(1, "the plan has no assembled matrix")
        rp = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        col = torch.empty(stored, dtype=torch.int32, device=self.device)
        val = torch.empty(stored, dtype=torch.float32, device=self.device)
        self.ctx.check(lib().rbf_plan_export_csr(self._h, _ptr(rp), _ptr(col), _ptr(val), _stream(stream)),
                       "rbf_plan_export_csr")
        return rp, col, val

    def spmv(self, z, out=None, stream=None):
        """y = A~ z through the assembled matrix (caller order)."""
        import torch
        _req(z, torch.float32, "z", self.n)
        y = torch.empty_like(z) if out is None else _req(out, torch.float32, "out", self.n)
        self.ctx.check(lib().rbf_spmv(self._h, _ptr(z), _ptr(y), _stream(stream)), "rbf_spmv")
        return y

    def count_candidate_pairs(self, stream=None) -> int:
        """Pairs the tensor-core product evaluates (the waste ratio's numerator)."""
        c = ctypes.c_int64(0)
        self.ctx.check(lib().rbf_count_candidate_pairs(self._h, ctypes.byref(c), _stream(stream)),
                       "rbf_count_candidate_pairs")
        return int(c.value)

    def residual(self, b, x, mode="df", stream=None):
        """True residual b - A~ x (float64); mode "df" (double-float) or "f64" (native)."""
        import torch
        _req(b, torch.float32, "b", self.n)
        _req(x, torch.float64, "x", self.n)
        r = torch.empty(self.n, dtype=torch.float64, device=self.device)
        norms = (ctypes.c_double * 2)()
        self.ctx.check(lib().rbf_residual(self._h, _ptr(b), _ptr(x), _ptr(r), norms, RESIDUAL[mode],
                                          _stream(stream)), "rbf_residual")
        return r, (norms[0], norms[1])

    def schwarz_setup(self, core=96, block=128, shift=1e-4, restricted=True, escalate=False, stream=None) -> int:
        p = SchwarzParams(int(core), int(block), float(shift), int(bool(restricted)), int(bool(escalate)))
        f = ctypes.c_int64(0)
        self.ctx.check(lib().rbf_schwarz_setup(self._h, ctypes.byref(p), ctypes.byref(f), _stream(stream)),
                       "rbf_schwarz_setup", allow=(7,))
        return int(f.value)

    def schwarz_apply(self, v, stream=None):
        import torch
        _req(v, torch.float32, "v", self.n)
        z = torch.empty_like(v)
        self.ctx.check(lib().rbf_schwarz_apply(self._h, _ptr(v), _ptr(z), _stream(stream)), "rbf_schwarz_apply")
        return z

    def solve(self, b, x=None, stream=None, **kw):
        """Step 2: FGMRES on A~ x = b.  Keyword arguments as ``_solve_params``.
        Returns (x float64, report dict); does not raise on NOT_CONVERGED."""
        import torch
        _req(b, torch.float32, "b", self.n)
        x = torch.empty(self.n, dtype=torch.float64, device=self.device) if x is None else x
        rep = Report()
        sp = _solve_params(**kw)
        st = lib().rbf_plan_solve(self._h, _ptr(b), ctypes.byref(sp), _ptr(x), ctypes.byref(rep), _stream(stream))
        self.ctx.check(st, "rbf_plan_solve", allow=(4,))
        d = rep.as_dict()
        d["status"] = STATUS[st]
        return x, d

    def count_grid_pairs(self, lo, hi, dims, stream=None) -> int:
        g = _grid(lo, hi, dims)
        c = ctypes.c_int64(0)
        self.ctx.check(lib().rbf_count_grid_pairs(self._h, ctypes.byref(g), ctypes.byref(c), _stream(stream)),
                       "rbf_count_grid_pairs")
        return int(c.value)

    def count_grid_candidate_pairs(self, lo, hi, dims, stream=None) -> int:
        """(node slot, centre) pairs the grid evaluation evaluates (its waste ratio's numerator)."""
        g = _grid(lo, hi, dims)
        c = ctypes.c_int64(0)
        self.ctx.check(lib().rbf_count_grid_candidate_pairs(self._h, ctypes.byref(g), ctypes.byref(c),
                                                            _stream(stream)), "rbf_count_grid_candidate_pairs")
        return int(c.value)

    def eval_grid(self, weights, lo, hi, dims, out=None, stream=None):
        """Step 3: P_f on the grid, shape (dims[2], dims[1], dims[0]) float32."""
        import torch
        _req(weights, torch.float64, "weights", self.n)
        f = torch.empty((int(dims[2]), int(dims[1]), int(dims[0])), dtype=torch.float32,
                        device=self.device) if out is None else out
        g = _grid(lo, hi, dims)
        self.ctx.check(lib().rbf_plan_eval_grid(self._h, _ptr(weights), ctypes.byref(g), _ptr(f), _stream(stream)),
                       "rbf_plan_eval_grid")
        return f


def solve(ctx: Context, centers, targets, sigma: float, k: float = 0.0, product: str = "tc", kernel: str = "gaussian",
          beta: float = 0.0, stream=None, **kw):
    """One-shot step 2 (plan + FGMRES + free)."""
    import torch
    _req(centers, torch.float32, "centers")
    n = centers.shape[0]
    _req(targets, torch.float32, "targets", n)
    pp = _plan_params(sigma, k, product=product, kernel=kernel, beta=beta)
    x = torch.empty(n, dtype=torch.float64, device=centers.device)
    rep = Report()
    sp = _solve_params(**kw)
    st = lib().rbf_solve(ctx._h, _ptr(centers), _ptr(targets), n, ctypes.byref(pp), ctypes.byref(sp), _ptr(x),
                         ctypes.byref(rep), _stream(stream))
    ctx.check(st, "rbf_solve", allow=(4,))
    d = rep.as_dict()
    d["status"] = STATUS[st]
    return x, d


def eval_grid(ctx: Context, centers, weights, sigma: float, k: float, lo, hi, dims, product: str = "tc",
              kernel: str = "gaussian", beta: float = 0.0, stream=None):
    """One-shot step 3."""
    import torch
    _req(centers, torch.float32, "centers")
    n = centers.shape[0]
    _req(weights, torch.float64, "weights", n)
    pp = _plan_params(sigma, k, product=product, kernel=kernel, beta=beta)
    f = torch.empty((int(dims[2]), int(dims[1]), int(dims[0])), dtype=torch.float32, device=centers.device)
    g = _grid(lo, hi, dims)
    ctx.check(lib().rbf_eval_grid(ctx._h, _ptr(centers), _ptr(weights), n, ctypes.byref(pp), ctypes.byref(g), _ptr(f),
                                  _stream(stream)), "rbf_eval_grid")
    return f


NOALLOC_MAX_N = 32768


def matvec_dense_noalloc(ctx: Context, centers, sigma: float, z, out, stream=None):
    """Untruncated y = A z through the allocation-free entry point; the caller
    supplies every buffer (``out`` included), the library allocates nothing."""
    import torch
    _req(centers, torch.float32, "centers")
    n = centers.shape[0]
    _req(z, torch.float32, "z", n)
    _req(out, torch.float32, "out", n)
    ctx.check(lib().rbf_matvec_dense_noalloc(ctx._h, _ptr(centers), n, float(sigma), _ptr(z), _ptr(out),
                                             _stream(stream)), "rbf_matvec_dense_noalloc")
    return out


class Batch:
    """Many independent problems (one Plan each) solved together: a persistent
    product kernel over all problems and a lockstep FGMRES captured as one CUDA
    graph (include/rbf.h, rbf_batch_*).  Keeps references to its plans."""

    def __init__(self, ctx: Context, plans, stream=None):
        self.ctx = ctx
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        self._h = ctypes.c_void_p()
        ctx.check(lib().rbf_batch_create(ctx._h, arr, len(self.plans), ctypes.byref(self._h), _stream(stream)),
                  "rbf_batch_create")
        ctx._dependents.add(self)
        self.n = int(lib().rbf_batch_size(self._h))
        self.device = self.plans[0].device

    def close(self):
        if self._h:
            lib().rbf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def matvec(self, z, stream=None):
        import torch
        _req(z, torch.float32, "z", self.n)
        y = torch.empty_like(z)
        self.ctx.check(lib().rbf_batch_matvec(self._h, _ptr(z), _ptr(y), _stream(stream)), "rbf_batch_matvec")
        return y

    def solve(self, b, stream=None, **kw):
        """Solve every problem: with fixed_iterations=True each takes max_it steps, else
        each stops at tol.  Returns (x float64, reports, stats)."""
        import torch
        _req(b, torch.float32, "b", self.n)
        x = torch.empty(self.n, dtype=torch.float64, device=self.device)
        reps = (Report * len(self.plans))()
        st = BatchStats()
        sp = _solve_params(**kw)
        self.ctx.check(lib().rbf_batch_solve(self._h, _ptr(b), ctypes.byref(sp), _ptr(x), reps, ctypes.byref(st),
                                             _stream(stream)), "rbf_batch_solve")
        return x, [r.as_dict() for r in reps], {f: getattr(st, f) for f, _ in st._fields_}

    def autotune(self, b, candidates=(32, 64, 96, 128), stream=None, **kw):
        import torch
        _req(b, torch.float32, "b", self.n)
        cand = (ctypes.c_int * len(candidates))(*candidates)
        scores = (ctypes.c_double * len(candidates))()
        best = ctypes.c_int(0)
        sp = _solve_params(**kw)
        self.ctx.check(lib().rbf_batch_autotune(self._h, _ptr(b), ctypes.byref(sp), cand, len(candidates),
                                                ctypes.byref(best), scores, _stream(stream)), "rbf_batch_autotune")
        return int(best.value), list(scores)


class MLP:
    """The learned block preconditioner's network on the device (rbf_mlp_*)."""

    def __init__(self, ctx: Context, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_NPARAMS:
            raise ValueError(f"expected {MLP_NPARAMS} parameters, got {p.size}")
        self.ctx = ctx
        self._h = ctypes.c_void_p()
        ctx.check(lib().rbf_mlp_create(ctx._h, p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self._h)),
                  "rbf_mlp_create")
        ctx._dependents.add(self)

    def close(self):
        if self._h:
            lib().rbf_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        import numpy as np
        out = np.empty(MLP_NPARAMS, dtype=np.float32)
        self.ctx.check(lib().rbf_mlp_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)), "rbf_mlp_get_params")
        return out

    def forward(self, X, bf16=True, stream=None):
        import torch
        _req(X, torch.float32, "X")
        rows = X.numel() // 256
        Y = torch.empty((rows, 64), dtype=torch.float32, device=X.device)
        self.ctx.check(lib().rbf_mlp_forward(self._h, _ptr(X), rows, _ptr(Y), int(bool(bf16)), _stream(stream)),
                       "rbf_mlp_forward")
        return Y

    def loss_grad(self, X, T, grad=True, stream=None):
        import numpy as np
        import torch
        _req(X, torch.float32, "X")
        _req(T, torch.float32, "T")
        rows = X.numel() // 256
        loss = ctypes.c_double(0)
        g = np.empty(MLP_NPARAMS, dtype=np.float32) if grad else None
        self.ctx.check(lib().rbf_mlp_loss_grad(self._h, _ptr(X), _ptr(T), rows, ctypes.byref(loss),
                                               g.ctypes.data_as(ctypes.c_void_p) if grad else None, _stream(stream)),
                       "rbf_mlp_loss_grad")
        return loss.value, g

    def train(self, X, T, epochs=10, batch=1024, lr=1e-3, stream=None):
        import numpy as np
        import torch
        _req(X, torch.float32, "X")
        _req(T, torch.float32, "T")
        ns = X.numel() // 256
        hist = np.zeros(epochs)
        tp = TrainParams(int(epochs), int(batch), float(lr))
        self.ctx.check(lib().rbf_mlp_train(self._h, _ptr(X), _ptr(T), ns, ctypes.byref(tp),
                                           hist.ctypes.data_as(ctypes.c_void_p), _stream(stream)), "rbf_mlp_train")
        return hist


def mlp_make_data(plan: Plan, lam: float, block_ids, R, stream=None):
    """Features X (ns x 256) and exact targets Y (ns x 64) on the plan's 64-centre blocks."""
    import torch
    _req(block_ids, torch.int32, "block_ids")
    _req(R, torch.float32, "R")
    ns = block_ids.numel()
    X = torch.empty((ns, 256), dtype=torch.float32, device=R.device)
    Y = torch.empty((ns, 64), dtype=torch.float32, device=R.device)
    f = ctypes.c_int64(0)
    plan.ctx.check(lib().rbf_mlp_make_data(plan._h, ctypes.c_float(lam), _ptr(block_ids), _ptr(R), ns, _ptr(X),
                                           _ptr(Y), ctypes.byref(f), _stream(stream)), "rbf_mlp_make_data")
    return X, Y, int(f.value)
