"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-derive a value with the oracle's own formula: each compares
against a closed form, a library routine, a geometric invariant or brute force
organised differently, chosen so that a dropped term, a wrong sign or index, a
transposed operand or a wrong constant in the oracle fails at least one test.
"""
import math

import numpy as np
import pytest

import oracle
import synth


# ---------------------------------------------------------------- Section II.A.1
def test_offsurface_points_on_parallel_spheres():
    """On the unit sphere with n = x, the points x +- delta n lie on the spheres
    of radius 1 +- delta (a geometric invariant of Section II.A.1)."""
    cl = synth.sphere(300, seed=3)
    d = 0.07
    C, b = oracle.build_centers(cl.points, cl.normals, d)
    N = 300
    r = np.linalg.norm(C, axis=1)
    assert np.allclose(r[:N], 1.0, atol=1e-6)
    assert np.allclose(r[N:2 * N], 1.0 + d, atol=1e-6)
    assert np.allclose(r[2 * N:], 1.0 - d, atol=1e-6)
    assert np.all(b[:N] == 0) and np.all(b[N:2 * N] == d) and np.all(b[2 * N:] == -d)
    C1, b1 = oracle.build_centers(cl.points, cl.normals, d, tval=1.0)
    assert np.all(b1[N:2 * N] == 1.0) and np.all(b1[2 * N:] == -1.0)


def test_default_delta_is_one_percent_of_bbox_diagonal():
    p = np.array([[0, 0, 0], [3, 4, 12]], dtype=np.float32)
    assert oracle.default_delta(p) == pytest.approx(0.13)


# ------------------------------------------------------- Eq. matrixEntries, RBFsys
def test_entry_half_value_distance():
    """exp(-r^2/(2 sigma^2)) = 1/2 exactly at r = sigma sqrt(2 ln 2)."""
    s = 0.37
    r = s * math.sqrt(2 * math.log(2.0))
    C = np.array([[0.1, 0.2, 0.3], [0.1 + r, 0.2, 0.3]])
    A = oracle.dense_matrix(C, s)
    assert A[0, 0] == 1.0 and A[1, 1] == 1.0
    assert A[0, 1] == pytest.approx(0.5, rel=1e-14)
    assert A[1, 0] == pytest.approx(0.5, rel=1e-14)
    # same distance split over the three axes
    C2 = np.array([[0, 0, 0], [r / math.sqrt(3)] * 3])
    assert oracle.dense_matrix(C2, s)[0, 1] == pytest.approx(0.5, rel=1e-14)


def test_lattice_row_sum_is_separable():
    """On an m^3 lattice of spacing h with z = 1 the untruncated row sum at node
    (a, b, c) is the product of three 1-D sums of exp(-(i-a)^2 h^2/(2 sigma^2))."""
    m, h, s = 7, 0.13, 0.21
    P = synth.lattice(m, h, origin=(0.4, -0.2, 1.0))
    z = np.ones(len(P))
    row = (2 * m + 4) * m + 1          # node (x=1, y=4, z=2)
    y, cnt = oracle.kernel_rows(P, z, s, 0.0, rows=[row])
    one_d = [sum(math.exp(-((i - a) * h) ** 2 / (2 * s * s)) for i in range(m)) for a in (1, 4, 2)]
    assert cnt == m ** 3
    assert y[0] == pytest.approx(one_d[0] * one_d[1] * one_d[2], rel=1e-13)


def test_lattice_row_sum_truncated_counts_ball_nodes():
    """With cut-off k sigma, the row keeps exactly the lattice nodes strictly inside
    the ball of radius k sigma (counted by integer arithmetic)."""
    m, h, s, k = 13, 0.1, 0.1, 3.5
    P = synth.lattice(m, h)
    c = (6, 6, 6)
    row = (c[2] * m + c[1]) * m + c[0]
    y, cnt = oracle.kernel_rows(P, np.ones(len(P)), s, k, rows=[row])
    # |d|^2 < (k sigma / h)^2 = 12.25 in lattice units
    inside = [(i, j, l) for i in range(-6, 7) for j in range(-6, 7) for l in range(-6, 7)
              if i * i + j * j + l * l < 12.25]
    assert cnt == len(inside)
    expect = sum(math.exp(-(i * i + j * j + l * l) * h * h / (2 * s * s)) for i, j, l in inside)
    assert y[0] == pytest.approx(expect, rel=1e-13)


def test_matrix_symmetric_positive_definite(sphere_c1):
    """Section II.B: the Gaussian gives a symmetric positive definite matrix
    (checked with LAPACK's symmetric eigensolver, a library routine)."""
    cl = synth.sphere(60, seed=1)
    C, _ = oracle.build_centers(cl.points, cl.normals, 0.05)
    A = oracle.dense_matrix(C, 0.3)
    assert np.array_equal(A, A.T)
    lam = np.linalg.eigvalsh(A)
    assert lam[0] > 0


def test_truncation_bound():
    """|(A~ z - A z)_i| <= exp(-k^2/2) * sum_{|c_i - c_j| >= k sigma} |z_j|."""
    rng = np.random.default_rng(7)
    C = rng.uniform(-1, 1, (400, 3))
    z = rng.standard_normal(400)
    s, k = 0.25, 2.5
    yt, _ = oracle.kernel_rows(C, z, s, k)
    yf, _ = oracle.kernel_rows(C, z, s, 0.0)
    D = np.sqrt(((C[:, None, :] - C[None, :, :]) ** 2).sum(-1))
    far = D >= k * s
    bound = math.exp(-k * k / 2) * (far * np.abs(z)[None, :]).sum(1)
    assert np.all(np.abs(yt - yf) <= bound * (1 + 1e-12) + 1e-300)
    assert np.any(far)


def test_kernel_rows_match_brute_force_loops():
    """The bucket list only skips far pairs: compare with plain Python loops."""
    rng = np.random.default_rng(11)
    C = rng.uniform(0, 1, (50, 3))
    z = rng.standard_normal(50)
    s, k = 0.1, 3.0
    y, cnt = oracle.kernel_rows(C, z, s, k)
    ref = np.zeros(50)
    ref_cnt = 0
    for i in range(50):
        for j in range(50):
            d2 = sum((C[i, t] - C[j, t]) ** 2 for t in range(3))
            if math.sqrt(d2) < k * s:
                ref[i] += z[j] * math.exp(-d2 / (2 * s * s))
                ref_cnt += 1
    assert cnt == ref_cnt
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------- Cholesky / solve
def test_truncated_entries_on_a_lattice_count_ball_offsets():
    """Algorithm 2 on the 7^3 unit lattice, sigma 0.5, k 3 (cut-off 1.5): a row keeps the
    integer offsets (a, b, c) with a^2 + b^2 + c^2 < 2.25 that stay on the lattice,
    value exp(-2 (a^2 + b^2 + c^2)); counted here by enumerating the offsets."""
    m = 7
    C = synth.lattice(m, 1.0)
    idx = lambda x, y, z: x + m * (y + m * z)
    for (x, y, z) in [(3, 3, 3), (0, 0, 0), (6, 3, 0), (1, 5, 6)]:
        want = {}
        for a in range(-2, 3):
            for b in range(-2, 3):
                for c in range(-2, 3):
                    q = a * a + b * b + c * c
                    if q < 2.25 and 0 <= x + a < m and 0 <= y + b < m and 0 <= z + c < m:
                        want[idx(x + a, y + b, z + c)] = math.exp(-2.0 * q)
        cols, vals = oracle.truncated_entries(C, 0.5, 3.0, [idx(x, y, z)])[0]
        assert sorted(want) == list(cols)
        np.testing.assert_allclose(vals, [want[j] for j in cols], rtol=1e-15)
    # interior row: 1 + 6 + 12 offsets of squared length 0, 1, 2
    assert len(oracle.truncated_entries(C, 0.5, 3.0, [idx(3, 3, 3)])[0][0]) == 19


def test_truncated_entries_agree_with_the_c_product_and_are_symmetric():
    """Rows of the numpy entry list against the C row product (an independent code):
    sum_j A_rj z_j and the pair count; and A_rj = A_jr."""
    cl = synth.torus(3000, noise=1e-3, seed=5)
    C = oracle.build_centers(cl.points, cl.normals, 0.02)[0]
    sigma, k = 0.05, 4.0
    rng = np.random.default_rng(1)
    z = rng.standard_normal(len(C))
    rows = rng.choice(len(C), 40, replace=False)
    ent = oracle.truncated_entries(C, sigma, k, rows)
    y, pairs = oracle.kernel_rows(C, z, sigma, k, rows)
    np.testing.assert_allclose([v @ z[c] for c, v in ent], y, rtol=1e-12, atol=1e-13)
    assert sum(len(c) for c, _ in ent) == pairs
    for r, (cols, vals) in zip(rows, ent):
        for j, v in zip(cols[:5], vals[:5]):
            cj, vj = oracle.truncated_entries(C, sigma, k, [j])[0]
            assert v == vj[np.searchsorted(cj, r)] and r in cj
    # k = 0 with a radius: the full dense rows less the entries beyond it
    A = oracle.dense_matrix(C[:500], sigma)
    e0 = oracle.truncated_entries(C[:500], sigma, 0.0, [7], radius_sigmas=13.0)[0]
    d = np.linalg.norm(C[:500] - C[7], axis=1)
    assert list(e0[0]) == list(np.nonzero(d < 13 * sigma)[0])
    np.testing.assert_allclose(e0[1], A[7, e0[0]], rtol=1e-13)   # exponents up to 84.5: 84.5 x 2^-52 x a few


def test_imq_interpolant_matches_scipy():
    """Table I's inverse multiquadric with beta = 1/2 is SciPy's 'inverse_multiquadric'
    kernel 1/sqrt(1 + (eps r)^2) with eps = 1/sigma; with no polynomial part the two
    interpolants of the same data agree (an independent library routine)."""
    from scipy.interpolate import RBFInterpolator
    cl = synth.sphere(150, seed=11)
    C, b = oracle.build_centers(cl.points, cl.normals, 0.05)
    sigma = 0.3
    x, res = oracle.imq_solve_dense(C, b, sigma, 0.5)
    assert res < 1e-10
    P = np.random.default_rng(4).uniform(-1.2, 1.2, (500, 3))
    ours = oracle.imq_eval_points(C, x, sigma, 0.5, 0.0, P)
    ref = RBFInterpolator(C, b, kernel="inverse_multiquadric", epsilon=1.0 / sigma, degree=-1)(P)
    assert np.abs(ours - ref).max() <= 1e-8 * np.abs(ref).max()


def test_imq_matrix_positive_definite_truncation_bound_and_rows():
    cl = synth.sphere(200, seed=12)
    C, _ = oracle.build_centers(cl.points, cl.normals, 0.05)
    for beta in (0.5, 1.5, 2.5):
        assert np.linalg.eigvalsh(oracle.imq_matrix(C, 0.2, beta)).min() > 0
    A = oracle.imq_matrix(C, 0.1, 2.0)
    At = oracle.imq_matrix(C, 0.1, 2.0, k=6.0)
    assert np.abs(A - At).max() <= (1 + 36.0) ** -2.0
    assert A[0, 0] == 1.0 and np.allclose(np.diag(A), 1.0)
    d2 = ((C[3] - C[17]) ** 2).sum()
    assert A[3, 17] == pytest.approx(1.0 / (1.0 + d2 / 0.01) ** 2, rel=1e-14)
    z = np.random.default_rng(5).standard_normal(len(C))
    np.testing.assert_allclose(oracle.imq_rows(C, z, 0.1, 2.0, 6.0, [3, 17, 500]), (At @ z)[[3, 17, 500]],
                               rtol=1e-12)


def test_cholesky_reconstructs_and_matches_lapack():
    cl = synth.sphere(80, seed=2)
    C, _ = oracle.build_centers(cl.points, cl.normals, 0.05)
    A = oracle.dense_matrix(C, 0.04)      # well conditioned, so the factors compare
    assert np.linalg.cond(A) < 1e4
    L = oracle.cholesky(A)
    assert np.all(np.triu(L, 1) == 0)
    assert np.abs(L @ L.T - A).max() <= 1e-14 * np.abs(A).max() * 10
    assert np.allclose(L, np.linalg.cholesky(A), rtol=1e-10, atol=1e-12)


def test_cholesky_rejects_indefinite():
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_solve_one_and_two_points():
    """n = 1: c = b.  n = 2: [[1, g], [g, 1]] c = b with g = exp(-r^2/(2 s^2))."""
    c, res = oracle.solve_dense(np.array([[0.3, 0.1, -0.2]]), np.array([0.7]), 0.2)
    assert c[0] == pytest.approx(0.7, rel=1e-15)
    r, s = 0.15, 0.2
    C = np.array([[0, 0, 0], [0, r, 0]])
    b = np.array([0.3, -0.9])
    g = math.exp(-r * r / (2 * s * s))
    c, _ = oracle.solve_dense(C, b, s)
    det = 1 - g * g
    assert c[0] == pytest.approx((b[0] - g * b[1]) / det, rel=1e-12)
    assert c[1] == pytest.approx((b[1] - g * b[0]) / det, rel=1e-12)


@pytest.fixture(scope="module")
def c1_solution(sphere_c1):
    C, b = oracle.build_centers(sphere_c1.points, sphere_c1.normals, 0.05)
    x, res = oracle.solve_dense(C, b, 0.1)
    return C, b, x, res


@pytest.mark.slow
def test_c1_interpolation_residual(c1_solution):
    """Interpolation conditions hold at every centre to 1e-12 (absolute, b ~ 0.05)."""
    C, b, x, res = c1_solution
    y, _ = oracle.kernel_rows(C, x, 0.1, 0.0)
    assert np.abs(y - b).max() <= 1e-12
    assert res <= 1e-12


@pytest.mark.slow
def test_c1_zero_set_near_unit_sphere(c1_solution):
    """The zero set of P_f along 2,000 seeded rays lies within delta/2 of the unit
    sphere (mean within delta/10); f < 0 just inside and f > 0 just outside."""
    C, b, x, _ = c1_solution
    rng = np.random.default_rng(123)
    g = rng.standard_normal((2000, 3))
    u = g / np.linalg.norm(g, axis=1, keepdims=True)
    lo = np.full(2000, 0.9)
    hi = np.full(2000, 1.1)
    flo = oracle.eval_points(C, x, 0.1, 0.0, lo[:, None] * u)
    fhi = oracle.eval_points(C, x, 0.1, 0.0, hi[:, None] * u)
    assert np.all(flo < 0) and np.all(fhi > 0)
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        fm = oracle.eval_points(C, x, 0.1, 0.0, mid[:, None] * u)
        neg = fm < 0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
    rstar = 0.5 * (lo + hi)
    assert np.abs(rstar - 1).max() <= 0.025
    assert np.abs(rstar - 1).mean() <= 0.005


# ----------------------------------------------------------------- Eq. matxvet
def test_eval_single_centre_closed_form():
    s = 0.2
    r = s * math.sqrt(2 * math.log(2.0))
    C = np.array([[1.0, -1.0, 0.5]])
    P = np.array([[1.0 + r, -1.0, 0.5], [1.0, -1.0, 0.5], [1.0, -1.0 + 3 * s, 0.5]])
    f = oracle.eval_points(C, np.array([2.0]), s, 0.0, P)
    assert f[0] == pytest.approx(1.0, rel=1e-14)
    assert f[1] == pytest.approx(2.0, rel=1e-15)
    assert f[2] == pytest.approx(2.0 * math.exp(-4.5), rel=1e-14)
    ft = oracle.eval_points(C, np.array([2.0]), s, 2.0, P)   # cut-off 2 sigma drops the third
    assert ft[2] == 0.0 and ft[0] == pytest.approx(1.0, rel=1e-14)


def test_eval_far_points_are_zero_when_truncated():
    rng = np.random.default_rng(1)
    C = rng.uniform(0, 1, (100, 3))
    P = np.array([[5.0, 5.0, 5.0], [-3.0, 0.5, 0.5], [0.5, 0.5, 1.0 + 0.31]])
    f = oracle.eval_points(C, np.ones(100), 0.05, 6.0, P)
    assert f[0] == 0.0 and f[1] == 0.0 and f[2] == 0.0


def test_grid_nodes_inclusive_x_fastest():
    P = oracle.grid_nodes((-1, 0, 2), (1, 1, 2), (3, 2, 1))
    assert P.shape == (6, 3)
    assert np.allclose(P[:, 0], [-1, 0, 1, -1, 0, 1])
    assert np.allclose(P[:, 1], [0, 0, 0, 1, 1, 1])
    assert np.allclose(P[:, 2], 2)
    Q = oracle.grid_nodes((-1.2,) * 3, (1.2,) * 3, (64,) * 3, flat_index=[64 ** 3 - 1, 0])
    assert np.allclose(Q[0], 1.2) and np.allclose(Q[1], -1.2)


# ------------------------------------------------------------------- binning
def test_morton_known_codes():
    m = oracle.morton3(np.array([1, 0, 0, 7, 1023, 5]), np.array([0, 1, 0, 7, 0, 3]),
                       np.array([0, 0, 1, 7, 0, 6]))
    # (5,3,6): x=101 y=011 z=110 -> bits z2y2x2 z1y1x1 z0y0x0 = 101 110 011
    assert list(m) == [1, 2, 4, 511, int("001" * 10, 2), int("101110011", 2)]


def test_binning_permutation_sorted_stable():
    rng = np.random.default_rng(4)
    C = rng.uniform(-1, 2, (5000, 3)).astype(np.float32)
    C[100:110] = C[7]                          # duplicates: equal keys
    B = oracle.binning(C, oracle.truncation_cell_edge(0.05, 3.0))
    perm = B["perm"]
    assert np.array_equal(np.sort(perm), np.arange(5000))
    ks = B["keys_sorted"].astype(np.int64)
    assert np.all(np.diff(ks) >= 0)
    eq = np.diff(ks) == 0
    assert np.all(np.diff(perm)[eq] > 0)       # stable: equal keys keep input order
    assert np.array_equal(B["key"][perm], B["keys_sorted"])
    # every centre lies in the fine cell its key names
    inv, lo = B["inv"], B["lo"]
    q = np.floor((C[perm] - lo).astype(np.float32) * inv)
    hf = 1.0 / float(inv)
    assert np.all(q >= 0)
    assert np.all((C[perm] - lo) >= q * hf * (1 - 1e-6) - 1e-7)
    # cell table covers every sorted position exactly once
    st, en = B["cell_start"], B["cell_end"]
    covered = np.zeros(5000, dtype=int)
    for s, e in zip(st, en):
        covered[s:e] += 1
    assert np.all(covered == 1)


def test_binning_matches_a_brute_force_grouping():
    """Cells by brute force: integer cell coordinates from float64 division (away
    from cell faces the float32 rule agrees), grouped by a dictionary."""
    rng = np.random.default_rng(8)
    hc = 0.25
    cells = rng.integers(0, 6, (400, 3))
    C = ((cells + rng.uniform(0.05, 0.95, (400, 3))) * hc).astype(np.float32)
    C[0] = 0.0                                  # pins lo at the origin
    B = oracle.binning(C, hc, levels=2)
    groups = {}
    for i, c in enumerate(C.astype(np.float64)):
        groups.setdefault(tuple(np.floor(c / hc).astype(int)), []).append(i)
    cs, ce, perm = B["cell_start"], B["cell_end"], B["perm"]
    nonempty = [(s, e) for s, e in zip(cs, ce) if e > s]
    assert len(nonempty) == len(groups)
    found = {tuple(sorted(perm[s:e])) for s, e in nonempty}
    assert found == {tuple(sorted(g)) for g in groups.values()}


def test_binning_cell_edge():
    """Fine cells are hc/2^L; cells are 2^L fine cells; r_c / s is k sigma / s."""
    assert oracle.truncation_cell_edge(0.1, 3.0, 1) == float(np.float32(3.0)) * float(np.float32(0.1))
    C = np.array([[0, 0, 0], [0.299, 0, 0], [0.301, 0, 0], [0.61, 0.0, 0.0]], dtype=np.float32)
    B = oracle.binning(C, oracle.truncation_cell_edge(0.1, 3.0, 1), levels=3)   # hc = 0.3
    cell = B["cell_of_sorted"][np.argsort(B["perm"])]
    assert cell[0] == cell[1] and cell[2] != cell[1]
    assert cell[2] == 1 and cell[3] == 8   # Morton codes of cell x = 1 and x = 2


# ------------------------------------------------------------ Schwarz / FGMRES
def test_schwarz_partition_covers_and_contains_cores():
    for n, core, block in [(1000, 96, 128), (130, 96, 128), (100, 96, 128), (500, 128, 128), (7, 3, 5)]:
        parts = oracle.schwarz_partition(n, core, block)
        cov = np.zeros(n, dtype=int)
        for d0, dl, c0, cl in parts:
            assert dl == min(block, n)
            assert d0 <= c0 and c0 + cl <= d0 + dl and 0 <= d0 and d0 + dl <= n
            cov[c0:c0 + cl] += 1
        assert np.all(cov == 1)


def test_schwarz_single_block_is_exact_inverse():
    cl = synth.sphere(40, seed=5)
    C, b = oracle.build_centers(cl.points, cl.normals, 0.05)
    s = 0.3
    parts = oracle.schwarz_partition(len(C), len(C), len(C))
    z = oracle.schwarz_apply(C, b, s, parts, 0.0)
    A = oracle.dense_matrix(C, s)
    assert np.allclose(z, np.linalg.solve(A, b), rtol=1e-8, atol=1e-10)
    x, it, hist = oracle.fgmres(lambda v: A @ v, b, lambda v: oracle.schwarz_apply(C, v, s, parts, 0.0))
    assert it == 1 and hist[-1] < 1e-8


def test_schwarz_block_jacobi_and_additive():
    """Zero overlap: restricted == additive == block-diagonal solve (LAPACK)."""
    rng = np.random.default_rng(9)
    C = rng.uniform(0, 1, (90, 3))
    v = rng.standard_normal(90)
    s, lam = 0.2, 1e-3
    parts = oracle.schwarz_partition(90, 30, 30)
    zr = oracle.schwarz_apply(C, v, s, parts, lam, restricted=True)
    za = oracle.schwarz_apply(C, v, s, parts, lam, restricted=False)
    ref = np.concatenate([np.linalg.solve(oracle.dense_matrix(C[i:i + 30], s) + lam * np.eye(30), v[i:i + 30])
                          for i in (0, 30, 60)])
    assert np.allclose(zr, ref, rtol=1e-9, atol=1e-12)
    assert np.allclose(za, ref, rtol=1e-9, atol=1e-12)
    # with overlap the two differ, and restricted only writes cores
    parts = oracle.schwarz_partition(90, 30, 40)
    zr = oracle.schwarz_apply(C, v, s, parts, lam, restricted=True)
    za = oracle.schwarz_apply(C, v, s, parts, lam, restricted=False)
    assert not np.allclose(zr, za)


def test_fgmres_distinct_eigenvalues():
    """GMRES on a diagonal matrix with k distinct eigenvalues converges in <= k steps."""
    d = np.repeat([1.0, 2.0, 5.0, 9.0], 25)
    b = np.random.default_rng(2).standard_normal(100)
    x, it, hist = oracle.fgmres(lambda v: d * v, b, m=20, tol=1e-12)
    assert it <= 4
    assert np.allclose(x, b / d, rtol=1e-10)


def test_fgmres_matches_scipy_gmres_history():
    """Unrestarted residual history equals SciPy's GMRES (library) on an SPD system."""
    from scipy.sparse.linalg import gmres
    cl = synth.sphere(60, seed=8)
    C, b = oracle.build_centers(cl.points, cl.normals, 0.05)
    A = oracle.dense_matrix(C, 0.2)
    x, it, hist = oracle.fgmres(lambda v: A @ v, b, m=30, tol=1e-30, max_it=30)
    ref = []
    gmres(A, b, rtol=1e-30, restart=30, maxiter=1, callback=lambda r: ref.append(r), callback_type="pr_norm")
    assert it == 30
    assert np.allclose(hist[:20], ref[:20], rtol=1e-6)
    y = A @ x
    assert np.linalg.norm(b - y) / np.linalg.norm(b) == pytest.approx(hist[-1], rel=1e-4)


def test_fgmres_flexible_preconditioner_changes_nothing_at_convergence():
    """A variable (flexible) preconditioner still gives the solution of A x = b."""
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((40, 40))
    A = Q @ Q.T + 40 * np.eye(40)
    b = rng.standard_normal(40)
    cnt = [0]

    def prec(v):
        cnt[0] += 1
        return v / np.diag(A) * (1.0 + 0.1 * (cnt[0] % 3))
    x, it, hist = oracle.fgmres(lambda v: A @ v, b, prec, m=40, tol=1e-12)
    assert np.allclose(A @ x, b, rtol=1e-9, atol=1e-9)


# ------------------------------------------------------- learned preconditioner
def test_mlp_forward_hand_computed():
    """A 2-3-2-1 network with chosen weights, evaluated by hand."""
    sizes = (2, 3, 2, 1)
    W1 = np.array([[1.0, -1.0], [0.5, 0.5], [-2.0, 0.0]]); b1 = np.array([0.0, 1.0, 0.5])
    W2 = np.array([[1.0, 1.0, 1.0], [0.0, -1.0, 2.0]]); b2 = np.array([-1.0, 0.0])
    W3 = np.array([[3.0, -1.0]]); b3 = np.array([0.25])
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    x = np.array([[2.0, 1.0]])
    # h1 = relu([1, 2.5, -3.5]) = [1, 2.5, 0]; h2 = relu([2.5, -2.5]) = [2.5, 0]; y = 7.5 + 0.25
    assert oracle.mlp_forward(p, x, sizes, skip=False)[0, 0] == pytest.approx(7.75)
    # the skip connection adds the last input to the (single) output
    assert oracle.mlp_forward(p, x, sizes, skip=True)[0, 0] == pytest.approx(8.75)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    sizes = (6, 5, 4, 3)
    p = synth.mlp_init(seed=4, sizes=sizes).astype(np.float64) + 0.05 * rng.standard_normal(
        sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:])))
    X = rng.standard_normal((7, 6))
    T = rng.standard_normal((7, 3))
    loss, g = oracle.mlp_loss_grad(p, X, T, sizes)
    assert loss == pytest.approx(np.mean((oracle.mlp_forward(p, X, sizes) - T) ** 2))
    assert not np.allclose(oracle.mlp_forward(p, X, sizes), oracle.mlp_forward(p, X, sizes, skip=False))
    for idx in rng.choice(len(p), 25, replace=False):
        e = np.zeros_like(p)
        e[idx] = 1e-6
        fd = (oracle.mlp_loss_grad(p + e, X, T, sizes)[0] - oracle.mlp_loss_grad(p - e, X, T, sizes)[0]) / 2e-6
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_mlp_block_targets_solve_the_shifted_block():
    """(A_i + lam I) Y / lam = r/|r| with A_i rebuilt by the dense-matrix routine."""
    rng = np.random.default_rng(5)
    Cs = rng.uniform(0, 0.3, (200, 3))
    R = rng.standard_normal((3, 64))
    X, Y = oracle.mlp_block_data(Cs, 0.05, 1e-3, [0, 2, 3], R)
    for row, (bi, r) in enumerate(zip([0, 2, 3], R)):
        d0 = min(bi * 64, 200 - 64)
        A = oracle.dense_matrix(Cs[d0:d0 + 64], 0.05) + 1e-3 * np.eye(64)
        assert np.allclose(A @ Y[row] / 8e-3, r / np.linalg.norm(r), atol=1e-9)
        assert np.allclose(X[row, 192:], 8 * r / np.linalg.norm(r))
        assert np.allclose(X[row, :192].reshape(64, 3).mean(0), 0, atol=1e-12)


# ---------------------------------------------------------------- Section IV: density measures
def test_density_halton_example_of_the_paper():
    """The worked example of Fig. filDist: 25 Halton points on [0,1]^2 have
    q ~ 0.0597 and fill distance ~ 0.2667 (tests/golden/density_halton25.json)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "density_halton25.json")))
    P = synth.halton(25, bases=(2, 3), start=1)
    X = np.c_[P, np.zeros(25)]
    m = 1201
    u = np.linspace(0.0, 1.0, m)
    gx, gy = np.meshgrid(u, u, indexing="ij")
    probes = np.c_[gx.ravel(), gy.ravel(), np.zeros(m * m)]
    d = oracle.density_measures(X, probes)
    half = 0.5 * 10.0 ** -(g["printed_digits"])
    assert abs(d["q"] - g["q"]) <= half
    # the max over a probe grid of spacing 1/1200 is within 1/1200 of the sup
    assert abs(d["fill"] - g["fill"]) <= half + 1.0 / (m - 1)
    assert d["sigma_q"] == pytest.approx(2 * d["q"]) and d["sigma_fill"] == pytest.approx(d["fill"] * math.sqrt(2))


def test_density_square_lattice_closed_forms():
    """Square lattice of spacing s: every nearest neighbour is at s, so q = s/2,
    h_max = mean = s; the farthest domain points from the lattice are the cell
    centres, at s / sqrt(2)."""
    s = 0.37
    g = np.arange(7) * s
    gx, gy = np.meshgrid(g, g, indexing="ij")
    X = np.c_[gx.ravel(), gy.ravel(), np.zeros(49)]
    cx, cy = np.meshgrid(g[:-1] + s / 2, g[:-1] + s / 2, indexing="ij")
    probes = np.c_[cx.ravel(), cy.ravel(), np.zeros(36)]
    d = oracle.density_measures(X, probes)
    assert d["q"] == pytest.approx(s / 2, rel=1e-12)
    assert d["h_max"] == pytest.approx(s, rel=1e-12) and d["mean_nn"] == pytest.approx(s, rel=1e-12)
    assert d["fill"] == pytest.approx(s / math.sqrt(2), rel=1e-12)


def test_density_nearest_neighbours_match_a_kd_tree():
    """Brute-force nearest-neighbour distances equal SciPy's k-d tree query (an
    independent algorithm) on a 3-D torus sample with duplicates."""
    from scipy.spatial import cKDTree
    cl = synth.torus(3000, noise=1e-3, seed=4)
    X = np.concatenate([cl.points.astype(np.float64), cl.points[:5].astype(np.float64)])   # 5 duplicates
    d = oracle.nn_distances(X)
    dd, _ = cKDTree(X).query(X, k=2)
    assert np.allclose(d, dd[:, 1], rtol=0, atol=1e-15)
    assert oracle.density_measures(X)["q"] == 0.0
    two = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    t = oracle.density_measures(two)
    assert t["q"] == pytest.approx(0.25) and t["h_max"] == pytest.approx(0.5)


# ---------------------------------------------------------------- Algorithm 1, step 4: the level set
def test_density_hemisphere_fill_closed_form_and_subset_monotone():
    """Data on the upper unit hemisphere: the distance from the south pole to (x, y, z)
    on the sphere is sqrt(2 + 2 z), so with the pole among the probes the fill distance
    over the whole sphere is sqrt(2 + 2 z_min) (the paper's sqrt 2 when points reach the
    equator), and it cannot be below that; removing points never lowers a fill distance."""
    Xf = synth.fibonacci_sphere(1120).points.astype(np.float64)
    Xf /= np.linalg.norm(Xf, axis=1, keepdims=True)          # exactly on the sphere (up to float64)
    Xu = Xf[Xf[:, 2] >= 0]
    u = np.random.default_rng(2).standard_normal((20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pole = np.array([[0.0, 0.0, -1.0]])
    zmin = Xu[:, 2].min()
    assert oracle.fill_distance(Xu, pole) == pytest.approx(math.sqrt(2 + 2 * zmin), rel=1e-14)
    assert oracle.fill_distance(Xu, np.vstack([u, pole])) == pytest.approx(math.sqrt(2 + 2 * zmin), rel=1e-14)
    eq = np.array([[math.cos(a), math.sin(a), 0.0] for a in (0.3, 2.4, 4.5)])
    assert oracle.fill_distance(np.vstack([Xu, eq]), pole) == pytest.approx(math.sqrt(2.0), rel=1e-15)
    sub = Xf[np.random.default_rng(3).choice(len(Xf), len(Xf) // 2, replace=False)]
    assert oracle.fill_distance(sub, u) >= oracle.fill_distance(Xf, u)


def _poly_area_clip(square, keep):
    """Area of a convex polygon clipped by half-planes keep(p) >= 0 (linear in p),
    Sutherland-Hodgman, for the reference area of a plane section."""
    pts = square
    for h in keep:
        out = []
        for k in range(len(pts)):
            p, q = np.array(pts[k]), np.array(pts[(k + 1) % len(pts)])
            hp, hq = h(p), h(q)
            if hp >= 0:
                out.append(p)
            if (hp >= 0) != (hq >= 0):
                out.append(p + (hp / (hp - hq)) * (q - p))
        pts = out
    x, y = np.array(pts).T
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_isosurface_of_a_linear_field_is_its_plane():
    """For f = a.x - c the interpolation along every edge is exact: every vertex lies
    on the plane, every normal points along a, and the triangles tile the plane's
    section of the box (area from an independent polygon clip)."""
    a = np.array([0.3, -0.5, 0.8])
    c = 0.1
    lo, hi, G = np.array([-1.0, -0.7, -0.6]), np.array([0.9, 1.1, 0.8]), (13, 11, 9)
    xs = [np.linspace(lo[d], hi[d], G[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    f = a[0] * X + a[1] * Y + a[2] * Z - c
    T, counts = oracle.isosurface(f, lo, hi)
    assert len(T) == counts.sum() > 0
    assert np.abs(T @ a - c).max() <= 1e-12
    n = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
    live = np.linalg.norm(n, axis=1) > 1e-14      # nodes exactly on the plane give zero-area triangles
    assert live.sum() > 0.9 * len(T) and np.all(n[live] @ a > 0)
    area = 0.5 * np.linalg.norm(n, axis=1).sum()
    # section area = area of its projection on the xy-plane (z between lo and hi) x |a| / |a_z|
    square = [(lo[0], lo[1]), (hi[0], lo[1]), (hi[0], hi[1]), (lo[0], hi[1])]
    zof = lambda p: (c - a[0] * p[0] - a[1] * p[1]) / a[2]
    proj = _poly_area_clip(square, [lambda p: zof(p) - lo[2], lambda p: hi[2] - zof(p)])
    assert area == pytest.approx(proj * np.linalg.norm(a) / abs(a[2]), rel=1e-12)


def _mesh_topology(T, digits=9):
    key = {}
    V = np.round(T.reshape(-1, 3), digits)
    ids = np.array([key.setdefault(tuple(v), len(key)) for v in V]).reshape(-1, 3)
    edges = {}
    for t in ids:
        for i in range(3):
            e = (min(t[i], t[(i + 1) % 3]), max(t[i], t[(i + 1) % 3]))
            edges[e] = edges.get(e, 0) + 1
    return len(key), edges, len(ids)


@pytest.mark.parametrize("shape,chi", [("sphere", 2), ("torus", 0)])
def test_isosurface_is_a_closed_surface(shape, chi):
    """The level set of a signed distance to a sphere or a torus is a closed
    2-manifold: every edge borders exactly two triangles, and the Euler
    characteristic V - E + F is 2 for the sphere and 0 for the torus."""
    g = np.linspace(-1.0, 1.0, 23)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    if shape == "sphere":
        f = np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 0.63
    else:
        f = np.sqrt((np.sqrt(X ** 2 + Y ** 2) - 0.55) ** 2 + Z ** 2) - 0.23
    T, _ = oracle.isosurface(f, (-1.0,) * 3, (1.0,) * 3)
    V, E, F = _mesh_topology(T)
    assert all(c == 2 for c in E.values())
    assert V - len(E) + F == chi


def test_isosurface_band_keeps_only_cells_near_the_data():
    """With a band, a cell contributes only when its centre is within the band of a
    data point: a plane's level set restricted to a disc of data points keeps
    exactly the cells whose centres are within the band, and the full level set's
    cells are kept when the band exceeds the box diagonal."""
    lo, hi, G = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0]), 17
    g = np.linspace(-1, 1, G)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    f = Z - 0.03
    T_all, c_all = oracle.isosurface(f, lo, hi)
    pts = np.array([[0.0, 0.0, 0.03]])                     # one data point on the plane
    T_b, c_b = oracle.isosurface(f, lo, hi, points=pts, band=0.3)
    step = (hi - lo) / (G - 1)
    kz, ky, kx = np.nonzero(c_all)
    centres = lo + (np.stack([kx, ky, kz], 1) + 0.5) * step
    near = ((centres - pts[0]) ** 2).sum(1) <= 0.09
    assert np.array_equal(c_b[kz, ky, kx] > 0, near) and 0 < near.sum() < len(near)
    T_w, c_w = oracle.isosurface(f, lo, hi, points=pts, band=4.0)
    assert np.array_equal(c_w, c_all)
