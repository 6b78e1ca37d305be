"""FP64 CPU oracle for the Gaussian-RBF reconstruction path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with ``paper_1305_5179_b300`` (neither imports the
other); the seeded input generators in ``synth`` are the only common module.

Each function states the passage of the paper it restates.  Heavy loops are in
``rbf_oracle.c`` (plain C, double precision, compiled by ``build()``); the rest
is numpy.  Library primitives used as single steps: ``numpy.argsort`` (stable
sort), ``numpy`` elementwise arithmetic.  Parity is pinned in
``tests/test_oracle_*.py`` against closed forms, brute force and library
routines, see each function's docstring.

Conventions shared with the library (these are *definitions*, stated in the
library header as well, not shared code):
  * centres are the extended set [X; X+; X-] (Section II.A.1), targets
    0 / +t / -t with t = delta by default (t = 1 reproduces the paper's +-1);
  * the kernel is exp(-r^2 / (2 sigma^2)) without the 1/(sqrt(2 pi) sigma)
    prefactor of Eq. matrixEntries (it rescales c, leaves P_f unchanged);
  * truncation keeps pairs with |x_i - x_j| < k sigma (strict), k = 0 keeps all;
  * grid nodes are xi_i = lo + i (hi - lo)/(G - 1) (inclusive ends), x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbf_oracle.c")
_LIB = os.path.join(_HERE, "librbf_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``rbf_oracle.c`` into ``librbf_oracle.so`` beside it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        lib.or_build_centers.argtypes = [P, P, I64, D, D, P, P]
        lib.or_dense_matrix.argtypes = [P, I64, D, D, P]
        lib.or_cholesky.argtypes = [P, I64]
        lib.or_cholesky.restype = ctypes.c_int
        lib.or_chol_solve.argtypes = [P, I64, P, P]
        lib.or_kernel_rows.argtypes = [P, I64, D, D, P, P, I64, P, P]
        lib.or_kernel_rows.restype = ctypes.c_int
        lib.or_eval_points.argtypes = [P, I64, P, D, D, P, I64, P]
        lib.or_eval_points.restype = ctypes.c_int
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_threads(t: int) -> None:
    _load().or_set_threads(int(t))


# --------------------------------------------------------------------------
# Section II.A.1-2: extended data set
# --------------------------------------------------------------------------
def build_centers(points: np.ndarray, normals: np.ndarray, delta: float, tval: float | None = None):
    """Extended set [X; X + delta n; X - delta n] and targets [0; +t; -t].

    Section II.A.1 (off-surface points) and II.A.2 (targets).  ``tval`` defaults
    to ``delta``.  Returns C (3N x 3 float64) and b (3N float64)."""
    pts = np.ascontiguousarray(points, dtype=np.float32)
    nrm = np.ascontiguousarray(normals, dtype=np.float32)
    N = pts.shape[0]
    C = np.empty((3 * N, 3))
    b = np.empty(3 * N)
    _load().or_build_centers(_p(pts), _p(nrm), N, float(delta),
                             float(delta if tval is None else tval), _p(C), _p(b))
    return C, b


def default_delta(points: np.ndarray) -> float:
    """Section II.A.1: delta = 1% of the bounding box (read: of its diagonal)."""
    p = np.asarray(points, dtype=np.float64)
    return 0.01 * float(np.linalg.norm(p.max(0) - p.min(0)))


# --------------------------------------------------------------------------
# Eq. matrixEntries / RBFsys: dense matrix, Cholesky, solve
# --------------------------------------------------------------------------
def dense_matrix(C: np.ndarray, sigma: float, k: float = 0.0) -> np.ndarray:
    """A_ij = exp(-|c_i - c_j|^2/(2 sigma^2)), zero where |c_i - c_j| >= k sigma (k > 0)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    n = C.shape[0]
    A = np.empty((n, n))
    _load().or_dense_matrix(_p(C), n, float(sigma), float(k), _p(A))
    return A


def cholesky(A: np.ndarray) -> np.ndarray:
    """Unpivoted right-looking Cholesky A = L L^T (own code, Section II.B: A is SPD).

    Raises ``np.linalg.LinAlgError`` when a pivot is not positive."""
    L = np.array(A, dtype=np.float64, order="C", copy=True)
    info = _load().or_cholesky(_p(L), L.shape[0])
    if info != 0:
        raise np.linalg.LinAlgError(f"non-positive pivot at column {info - 1}")
    return L


def chol_solve(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    _load().or_chol_solve(_p(np.ascontiguousarray(L)), L.shape[0], _p(b), _p(x))
    return x


def solve_dense(C: np.ndarray, b: np.ndarray, sigma: float, k: float = 0.0, refine_tol: float = 1e-12):
    """Solve A c = b (Eq. RBFsys) by Cholesky, with one step of FP64 iterative
    refinement when the relative residual exceeds ``refine_tol``.

    Returns (c, relative residual)."""
    A = dense_matrix(C, sigma, k)
    L = cholesky(A)
    x = chol_solve(L, b)
    r = b - A @ x
    nb = np.linalg.norm(b)
    if nb > 0 and np.linalg.norm(r) / nb > refine_tol:
        x = x + chol_solve(L, r)
        r = b - A @ x
    return x, (float(np.linalg.norm(r) / nb) if nb > 0 else 0.0)


# --------------------------------------------------------------------------
# Section III.A: truncated matrix-vector product on selected rows
# --------------------------------------------------------------------------
def kernel_rows(C: np.ndarray, z: np.ndarray, sigma: float, k: float, rows=None):
    """y_r = sum_{j : |c_r - c_j| < k sigma} z_j exp(-|c_r - c_j|^2/(2 sigma^2)).

    ``k <= 0`` keeps every pair.  Returns (y, number of pairs with i = j
    included, summed over the rows)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    n = C.shape[0]
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(len(rows))
    cnt = ctypes.c_int64(0)
    rc = _load().or_kernel_rows(_p(C), n, float(sigma), float(k), _p(z), _p(rows), len(rows),
                                _p(y), ctypes.byref(cnt))
    if rc != 0:
        raise MemoryError("oracle bucket list allocation failed")
    return y, int(cnt.value)


def truncated_entries(C: np.ndarray, sigma: float, k: float, rows, radius_sigmas: float = 0.0):
    """Nonzero entries of the chosen rows of the truncated matrix (Algorithm 2: for
    each point, each point of its truncation area, A_ij = phi(|x_i - x_j|)).

    Row r holds every j with |c_r - c_j| < k sigma (``k <= 0``: every j, or every j
    closer than ``radius_sigmas`` sigma when that is > 0), value
    exp(-|c_r - c_j|^2 / (2 sigma^2)).  Brute force over all centres, float64.
    Returns a list of (columns ascending int64, values float64), one per row."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    s2 = float(sigma) * float(sigma)
    if k > 0:
        lim = (float(k) * float(sigma)) ** 2
    elif radius_sigmas > 0:
        lim = (float(radius_sigmas) * float(sigma)) ** 2
    else:
        lim = np.inf
    out = []
    for r in np.asarray(rows, dtype=np.int64):
        d = C - C[r]
        d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        cols = np.nonzero(d2 < lim)[0]
        out.append((cols.astype(np.int64), np.exp(-d2[cols] / (2.0 * s2))))
    return out


# --------------------------------------------------------------------------
# Table I: the inverse multiquadric (1 + |x - x_j|^2)^(-beta), here with the
# length scale sigma: phi(r) = (1 + r^2 / sigma^2)^(-beta) (Table I is sigma = 1).
# Dense numpy, for the small systems this variant is used on.
# --------------------------------------------------------------------------
def imq_phi(r2, sigma: float, beta: float):
    """(1 + r^2/sigma^2)^(-beta) for squared distances r2."""
    return (1.0 + np.asarray(r2, dtype=np.float64) / (float(sigma) ** 2)) ** (-float(beta))


def _imq_block(Ci: np.ndarray, Cj: np.ndarray, sigma: float, beta: float, k: float) -> np.ndarray:
    d2 = ((Ci[:, None, :] - Cj[None, :, :]) ** 2).sum(-1)
    A = imq_phi(d2, sigma, beta)
    if k > 0:
        A[~(d2 < (float(k) * float(sigma)) ** 2)] = 0.0
    return A


def imq_matrix(C: np.ndarray, sigma: float, beta: float, k: float = 0.0) -> np.ndarray:
    """A_ij = phi(|c_i - c_j|), zero where |c_i - c_j| >= k sigma (k > 0)."""
    C = np.ascontiguousarray(C, dtype=np.float64)[:, :3]
    return _imq_block(C, C, sigma, beta, k)


def imq_rows(C: np.ndarray, z: np.ndarray, sigma: float, beta: float, k: float = 0.0, rows=None) -> np.ndarray:
    """y_r = sum_j A_rj z_j on the chosen rows (all by default), 256 rows at a time."""
    C = np.ascontiguousarray(C, dtype=np.float64)[:, :3]
    z = np.asarray(z, dtype=np.float64)
    rows = np.arange(len(C)) if rows is None else np.asarray(rows, dtype=np.int64)
    y = np.empty(len(rows))
    for a in range(0, len(rows), 256):
        y[a:a + 256] = _imq_block(C[rows[a:a + 256]], C, sigma, beta, k) @ z
    return y


def imq_eval_points(C: np.ndarray, w: np.ndarray, sigma: float, beta: float, k: float, P: np.ndarray) -> np.ndarray:
    """P_f(p) = sum_j w_j phi(|p - c_j|) at the rows of P."""
    C = np.ascontiguousarray(C, dtype=np.float64)[:, :3]
    P = np.ascontiguousarray(P, dtype=np.float64)[:, :3]
    w = np.asarray(w, dtype=np.float64)
    f = np.empty(len(P))
    for a in range(0, len(P), 256):
        f[a:a + 256] = _imq_block(P[a:a + 256], C, sigma, beta, k) @ w
    return f


def imq_solve_dense(C: np.ndarray, b: np.ndarray, sigma: float, beta: float):
    """Solve A c = b for the untruncated IMQ matrix by the oracle's Cholesky (A is
    positive definite for every beta > 0: phi is completely monotone in r^2).
    Returns (c, relative residual)."""
    A = imq_matrix(C, sigma, beta)
    L = cholesky(A)
    x = chol_solve(L, np.asarray(b, dtype=np.float64))
    r = np.asarray(b, dtype=np.float64) - A @ x
    return x, float(np.linalg.norm(r) / np.linalg.norm(b))


def residual_rows(C, b, x, sigma, k, rows=None):
    """r_i = b_i - (A~ x)_i on ``rows`` (all rows by default)."""
    y, _ = kernel_rows(C, x, sigma, k, rows)
    bb = np.asarray(b, dtype=np.float64)
    return (bb if rows is None else bb[np.asarray(rows)]) - y


# --------------------------------------------------------------------------
# Eq. matxvet: evaluation of P_f
# --------------------------------------------------------------------------
def eval_points(C: np.ndarray, w: np.ndarray, sigma: float, k: float, P: np.ndarray) -> np.ndarray:
    """P_f(p) = sum_j w_j phi(|p - c_j|) at the rows of P (m x 3)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    f = np.empty(P.shape[0])
    rc = _load().or_eval_points(_p(C), C.shape[0], _p(w), float(sigma), float(k), _p(P), P.shape[0], _p(f))
    if rc != 0:
        raise MemoryError("oracle bucket list allocation failed")
    return f


def grid_nodes(lo, hi, dims, flat_index=None) -> np.ndarray:
    """Nodes xi = lo + i (hi - lo)/(G - 1) per axis (G = 1 puts the node at lo),
    ordered x fastest; ``flat_index`` selects nodes by their flat position."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    dims = np.asarray(dims, dtype=np.int64)
    if flat_index is None:
        flat_index = np.arange(int(np.prod(dims)), dtype=np.int64)
    flat_index = np.asarray(flat_index, dtype=np.int64)
    ix = flat_index % dims[0]
    iy = (flat_index // dims[0]) % dims[1]
    iz = flat_index // (dims[0] * dims[1])
    step = np.where(dims > 1, (hi - lo) / np.maximum(dims - 1, 1), 0.0)
    return np.stack([lo[0] + ix * step[0], lo[1] + iy * step[1], lo[2] + iz * step[2]], axis=1)


# --------------------------------------------------------------------------
# Cell binning (the "truncation area" of Algorithm 2 made concrete)
# --------------------------------------------------------------------------
def part1by2(v: np.ndarray) -> np.ndarray:
    """Spread the low 10 bits of v so that bit b moves to bit 3b."""
    v = np.asarray(v, dtype=np.uint64)
    out = np.zeros_like(v)
    for b in range(10):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def morton3(qx, qy, qz) -> np.ndarray:
    """Interleave three 10-bit integers: bit b of qx -> 3b, qy -> 3b+1, qz -> 3b+2."""
    return (part1by2(qx) | (part1by2(qy) << np.uint64(1)) | (part1by2(qz) << np.uint64(2))).astype(np.uint32)


def truncation_cell_edge(sigma: float, k: float, cells_per_cutoff: int = 1) -> float:
    """Cell edge r_c / s with r_c = k sigma (the truncation area of Algorithm 2,
    Sec. III.A), from float32 sigma and k, in double."""
    return float(np.float32(k)) * float(np.float32(sigma)) / float(cells_per_cutoff)


def binning(C32: np.ndarray, cell_edge: float, levels: int = 3):
    """Cell binning of the centres in FP32, as a definition (the truncation area
    of Algorithm 2 made concrete: centres are grouped by cells of edge
    ``cell_edge``, each subdivided into 2^levels fine cells per axis).

    * lo = componentwise minimum of the centres; ext = hi - lo (FP32);
    * inv = float32(2^L / cell_edge) computed in double;
    * q_d = floor((c_d - lo_d) * inv) in float32 arithmetic;
    * nbits = max(L, bit length of max_d floor(ext_d * inv)) (must be <= 10);
    * key = Morton interleave of (q_x, q_y, q_z); cell = key >> 3L;
    * stable sort of the centres by key; cell start/end over the sorted order.
    The cell edge is a parameter (``truncation_cell_edge`` gives r_c / s).
    Returns dict(perm, keys_sorted, key (per input centre), cell_of_sorted,
    cell_start, cell_end (dense tables over 2^(3(nbits-L)) cell codes), nbits,
    inv, lo)."""
    c = np.ascontiguousarray(C32[:, :3], dtype=np.float32)
    lo = c.min(0)
    hi = c.max(0)
    ext = (hi - lo).astype(np.float32)
    L = int(levels)
    inv = np.float32((2.0 ** L) / float(cell_edge))
    qmax = int(np.floor(ext * inv).max()) if len(c) else 0
    nbits = max(L, int(qmax).bit_length())
    if nbits > 10:
        raise ValueError("domain spans more than 1024 fine cells per axis")
    q = np.floor((c - lo).astype(np.float32) * inv).astype(np.int64)
    q = np.clip(q, 0, (1 << nbits) - 1)
    key = morton3(q[:, 0], q[:, 1], q[:, 2])
    perm = np.argsort(key, kind="stable")
    ks = key[perm]
    cell = (ks >> np.uint32(3 * L)).astype(np.int64)
    ncell = 1 << (3 * (nbits - L))
    start = np.zeros(ncell, dtype=np.int64)
    end = np.zeros(ncell, dtype=np.int64)
    if len(cell):
        first = np.ones(len(cell), dtype=bool)
        first[1:] = cell[1:] != cell[:-1]
        last = np.ones(len(cell), dtype=bool)
        last[:-1] = cell[1:] != cell[:-1]
        start[cell[first]] = np.nonzero(first)[0]
        end[cell[last]] = np.nonzero(last)[0] + 1
    return dict(perm=perm.astype(np.int64), keys_sorted=ks, key=key, cell_of_sorted=cell,
                cell_start=start, cell_end=end, nbits=nbits, inv=inv, lo=lo)


# --------------------------------------------------------------------------
# Section III.A: restricted additive Schwarz preconditioner
# --------------------------------------------------------------------------
def schwarz_partition(n: int, core: int, block: int):
    """Cores are consecutive runs of ``core`` positions of the binned order; the
    overlapping subdomain Omega_i is the run of exactly min(block, n) positions
    starting at clamp(s - (block - core)//2, 0, n - block).

    Returns a list of (dom_start, dom_len, core_start, core_len) in binned order."""
    out = []
    o = block - core
    for s in range(0, n, core):
        e = min(s + core, n)
        if n >= block:
            d0 = min(max(s - o // 2, 0), n - block)
            dl = block
        else:
            d0, dl = 0, n
        out.append((d0, dl, s, e - s))
    return out


def schwarz_apply(Cs: np.ndarray, v: np.ndarray, sigma: float, parts, shift: float,
                  restricted: bool = True) -> np.ndarray:
    """z = sum_i Rt_i^T (A_i + shift I)^{-1} R_i v  (restricted, the paper's RASM)
    or sum_i R_i^T (A_i + shift I)^{-1} R_i v (additive), Section III.A.

    ``Cs`` are the centres in binned order, A_i is the untruncated Gaussian
    matrix of subdomain i (a principal submatrix of the SPD matrix A), each block
    solved with the own Cholesky of this module."""
    z = np.zeros(len(v))
    for d0, dl, c0, cl in parts:
        idx = slice(d0, d0 + dl)
        Ai = dense_matrix(Cs[idx], sigma, 0.0) + shift * np.eye(dl)
        si = chol_solve(cholesky(Ai), v[idx])
        if restricted:
            z[c0:c0 + cl] = si[c0 - d0:c0 - d0 + cl]
        else:
            z[idx] += si
    return z


# --------------------------------------------------------------------------
# Section III.A: GMRES (flexible, right-preconditioned) as the Krylov method
# --------------------------------------------------------------------------
def fgmres(matvec, b: np.ndarray, precond=None, m: int = 50, tol: float = 1e-6, max_it: int = 500,
           x0: np.ndarray | None = None):
    """Flexible GMRES(m) (Saad 1993) with classical Gram-Schmidt applied twice
    and Givens rotations, all in FP64.  Stops when the rotated residual estimate
    |g_{j+1}| <= tol * |b| or after ``max_it`` inner iterations; each restart
    recomputes the true residual b - A x.  Returns (x, iterations, history of
    the residual estimate relative to |b|)."""
    b = np.asarray(b, dtype=np.float64)
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    M = (lambda v: v.copy()) if precond is None else precond
    nb = np.linalg.norm(b)
    hist = []
    it = 0
    if nb == 0:
        return x, 0, hist
    while it < max_it:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= tol * nb:
            break
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        V[0] = r / beta
        g[0] = beta
        j = -1
        for j in range(m):
            Z[j] = M(V[j])
            w = matvec(Z[j])
            for _ in range(2):
                h = V[:j + 1] @ w
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / rho
            sn[j] = H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            hist.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) <= tol * nb or it >= max_it or H[j + 1, j] == 0 and rho == 0:
                break
        k = j + 1
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        if hist and hist[-1] <= tol:
            break
    return x, it, hist


# --------------------------------------------------------------------------
# Learned block preconditioner (not in the paper): FP64 reference of the MLP,
# its gradient (manual back-propagation) and the training targets.
# --------------------------------------------------------------------------
def _mlp_unpack(params, sizes):
    out, o = [], 0
    for fin, fout in zip(sizes[:-1], sizes[1:]):
        W = np.asarray(params[o:o + fin * fout], dtype=np.float64).reshape(fout, fin)
        o += fin * fout
        b = np.asarray(params[o:o + fout], dtype=np.float64)
        o += fout
        out.append((W, b))
    return out


def mlp_forward(params, X, sizes=(256, 256, 256, 64), skip=True):
    """ReLU MLP: a_{l+1} = relu(a_l W_l^T + b_l) for hidden layers, linear output,
    plus (skip) the last ``sizes[-1]`` inputs added to the output."""
    X = np.asarray(X, dtype=np.float64)
    a = X
    layers = _mlp_unpack(params, sizes)
    for li, (W, b) in enumerate(layers):
        a = a @ W.T + b
        if li < len(layers) - 1:
            a = np.maximum(a, 0.0)
    if skip:
        a = a + X[:, -sizes[-1]:]
    return a


def mlp_loss_grad(params, X, T, sizes=(256, 256, 256, 64), skip=True):
    """Mean squared error over all outputs and its gradient, packed like params
    (the skip connection has no parameters)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    layers = _mlp_unpack(params, sizes)
    acts = [X]
    a = X
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        acts.append(a)
    Y = acts[-1] + (X[:, -sizes[-1]:] if skip else 0.0)
    diff = Y - T
    loss = float(np.mean(diff * diff))
    d = 2.0 * diff / diff.size
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        grads[li] = (d.T @ acts[li], d.sum(0))
        if li > 0:
            d = (d @ W) * (acts[li] > 0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def mlp_block_data(Cs, sigma, lam, block_ids, R, block=64):
    """Features and targets of the learned preconditioner on binned centres Cs:
    block i covers Cs[64 i : 64 i + 64] (clamped to the end);
    X = [(c - mean)/sigma (x y z per centre), 8 r/|r|],
    Y = 8 lam (A_i + lam I)^-1 r/|r| with A_i the untruncated Gaussian block,
    solved by this module's Cholesky."""
    Cs = np.asarray(Cs, dtype=np.float64)
    n = len(Cs)
    X = np.zeros((len(block_ids), 256))
    Y = np.zeros((len(block_ids), 64))
    for row, (bi, r) in enumerate(zip(block_ids, R)):
        d0 = min(max(int(bi) * block, 0), n - block)
        P = Cs[d0:d0 + block]
        r = np.asarray(r, dtype=np.float64)
        nr = np.linalg.norm(r)
        rh = r / nr if nr > 0 else np.zeros_like(r)
        X[row, :192] = ((P - P.mean(0)) / sigma).ravel()
        X[row, 192:] = 8.0 * rh
        A = dense_matrix(P, sigma) + lam * np.eye(block)
        Y[row] = 8.0 * lam * chol_solve(cholesky(A), rh)
    return X, Y


# ---------------------------------------------------------------- density measures
def nn_distances(X: np.ndarray, rows=None, chunk: int = 0) -> np.ndarray:
    """Distance from each point (or each point of `rows`) to its nearest other point
    of X, by brute force over all points (the min over i != j in the separation
    distance of Eq. sepDist and in h_max of Sec. IV).  A duplicate point has
    distance 0."""
    X = np.asarray(X, dtype=np.float64)
    idx = np.arange(len(X)) if rows is None else np.asarray(rows)
    chunk = chunk or max(1, (1 << 24) // max(1, len(X)))   # rows per pass: about 400 MB of temporaries
    out = np.empty(len(idx))
    for s in range(0, len(idx), chunk):
        r = idx[s:s + chunk]
        d2 = ((X[r, None, :] - X[None, :, :]) ** 2).sum(-1)
        d2[np.arange(len(r)), r] = np.inf
        out[s:s + chunk] = np.sqrt(d2.min(1))
    return out


def fill_distance(X: np.ndarray, probes: np.ndarray, chunk: int = 0) -> float:
    """Eq. fillDist with the sup over the domain replaced by a max over the given
    probe points of the domain: max_p min_j |p - x_j| (brute force)."""
    X = np.asarray(X, dtype=np.float64)
    P = np.asarray(probes, dtype=np.float64)
    chunk = chunk or max(1, (1 << 24) // max(1, len(X)))
    h = 0.0
    for s in range(0, len(P), chunk):
        d2 = ((P[s:s + chunk, None, :] - X[None, :, :]) ** 2).sum(-1)
        h = max(h, float(np.sqrt(d2.min(1)).max()))
    return h


def density_measures(X: np.ndarray, probes=None) -> dict:
    """Density measures of Sec. IV: separation distance q = 1/2 min_{i!=j} |x_i - x_j|
    (Eq. sepDist), h_max = max_j min_{i!=j} |x_i - x_j|, the mean nearest-neighbour
    distance, and, with probe points of the domain, the fill distance (Eq. fillDist);
    with the sigma rules sigma ~ 2 q (Eq. h1), sigma ~ h sqrt(2) (Eq. h2) and
    h ~ h_max sqrt(2) (Eq. hmax)."""
    d = nn_distances(X)
    out = {"q": 0.5 * float(d.min()), "h_max": float(d.max()), "mean_nn": float(d.mean())}
    out["fill"] = fill_distance(X, probes) if probes is not None and len(probes) else float("nan")
    out["sigma_q"] = 2.0 * out["q"]
    out["sigma_fill"] = out["fill"] * np.sqrt(2.0)
    out["sigma_hmax"] = out["h_max"] * np.sqrt(2.0)
    return out


# ---------------------------------------------------------------- isosurface (Algorithm 1, step 4)
# The paper renders P_f = 0 with MATLAB's isosurface (marching cubes).  The oracle
# extracts the same level set by marching tetrahedra: every grid cell is cut into
# the 6 tetrahedra around its diagonal from corner (0,0,0) to (1,1,1) (the same cut
# in every cell, so neighbouring cells' faces match), and every tetrahedron whose
# corners straddle the level contributes 1 or 2 triangles with corners on its edges.
_CUBE = np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])   # corner bit c -> (x, y, z)


def _kuhn_tets():
    """The 6 tetrahedra (corner indices) 0 -> 0 + e_a -> 0 + e_a + e_b -> 7 for the
    orders (a, b, c) of the axes, each listed with positive orientation."""
    import itertools
    tets = []
    for a, b, _ in itertools.permutations((1, 2, 4)):
        t = [0, a, a | b, 7]
        v = _CUBE[t].astype(np.float64)
        if np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]])) < 0:
            t[2], t[3] = t[3], t[2]
        tets.append(t)
    return tets


# even permutations putting a given corner (or pair of corners) first
_FIRST = {0: (0, 1, 2, 3), 1: (1, 0, 3, 2), 2: (2, 3, 0, 1), 3: (3, 2, 1, 0)}
_PAIR = {(0, 1): (0, 1, 2, 3), (0, 2): (0, 2, 3, 1), (0, 3): (0, 3, 1, 2),
         (1, 2): (1, 2, 0, 3), (1, 3): (1, 3, 2, 0), (2, 3): (2, 3, 0, 1)}


def isosurface(f: np.ndarray, lo, hi, iso: float = 0.0, points=None, band: float = 0.0):
    """Triangles (ntri, 3, 3) of the level set {f = iso} of the grid field f
    (shape (Gz, Gy, Gx), x fastest, nodes lo + i (hi - lo)/(G - 1)), in the order
    (cell in x-fastest order, tetrahedron, triangle); a corner is inside when
    f < iso; an edge point is p_a + (iso - f_a)/(f_b - f_a) (p_b - p_a) with a the
    edge's corner of smaller node index; every
    triangle's normal (v1 - v0) x (v2 - v0) points from inside to outside (a
    corner exactly at the level counts as outside and can give zero-area triangles;
    a cell with a NaN node gives none).  With data points and band > 0 only cells
    whose centre lies within `band` of a data point contribute: the surrounding
    volume M_ext^eps = {x : d(x, M) <= eps} of Sec. II.A.3, with d(x, M) read as the
    distance to the nearest data point.
    Returns (triangles, per-cell triangle counts of shape (Gz-1, Gy-1, Gx-1))."""
    f = np.asarray(f, dtype=np.float64)
    Gz, Gy, Gx = f.shape
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    dims = np.array([Gx, Gy, Gz])
    step = np.where(dims > 1, (hi - lo) / np.maximum(dims - 1, 1), 0.0)
    tets = _kuhn_tets()
    pts = np.asarray(points, dtype=np.float64)[:, :3] if band > 0 else None
    counts = np.zeros((Gz - 1, Gy - 1, Gx - 1), dtype=np.int64)
    per_cell = {}
    for kz in range(Gz - 1):
        for ky in range(Gy - 1):
            for kx in range(Gx - 1):
                vals = np.array([f[kz + _CUBE[c, 2], ky + _CUBE[c, 1], kx + _CUBE[c, 0]] for c in range(8)])
                if np.isnan(vals).any():          # a node left out of the evaluation
                    continue
                inside = vals < iso
                if inside.all() or not inside.any():
                    continue
                pos = lo + (np.array([kx, ky, kz]) + _CUBE) * step
                if band > 0:
                    centre = lo + (np.array([kx, ky, kz]) + 0.5) * step
                    if ((pts - centre) ** 2).sum(1).min() > band * band:
                        continue
                tris = []
                for t in tets:
                    vin = inside[t]
                    nin = int(vin.sum())
                    if nin == 0 or nin == 4:
                        continue

                    def cut(i, j):
                        # interpolated from the corner with the smaller node index, so that
                        # an edge shared by several tetrahedra or cells yields one point
                        a, b = min(t[i], t[j]), max(t[i], t[j])
                        s = (iso - vals[a]) / (vals[b] - vals[a])
                        return pos[a] + s * (pos[b] - pos[a])
                    if nin in (1, 3):
                        lone = [i for i in range(4) if vin[i] == (nin == 1)][0]
                        p = _FIRST[lone]
                        tri = [cut(p[0], p[1]), cut(p[0], p[2]), cut(p[0], p[3])]
                        if nin == 3:          # the lone corner is outside: the normal must point to it
                            tri = [tri[0], tri[2], tri[1]]
                        tris.append(tri)
                    else:
                        pair = tuple(i for i in range(4) if vin[i])
                        p = _PAIR[pair]
                        e_ac, e_ad, e_bd, e_bc = cut(p[0], p[2]), cut(p[0], p[3]), cut(p[1], p[3]), cut(p[1], p[2])
                        tris.append([e_ac, e_ad, e_bd])
                        tris.append([e_ac, e_bd, e_bc])
                counts[kz, ky, kx] = len(tris)
                per_cell[(kz, ky, kx)] = tris
    out = [tri for key in sorted(per_cell) for tri in per_cell[key]]
    T = np.array(out, dtype=np.float64).reshape(-1, 3, 3)
    return T, counts
