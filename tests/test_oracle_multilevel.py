"""Pins of the oracle's transfer operators, Galerkin products, colouring, smoothers."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import bmg, fem, mesh, multilevel
from paper_1511_07042_gb300 import inputs


@pytest.fixture(scope="module")
def H4():
    v, t = inputs.icosahedron()
    return bmg.build_hierarchy(v, t, 4)


def test_prolongation_entries_and_constants(H4):
    for l in range(2, 5):
        P = H4.P[l]
        assert np.allclose(P @ np.ones(P.shape[1]), 1.0, rtol=0, atol=0)  # P 1 = 1 exactly
        vals = np.unique(P.data)
        assert set(vals.tolist()) <= {0.5, 1.0}
        nnz = P.getnnz(axis=1)
        nc = P.shape[1]
        assert np.all(nnz[:nc] == 1) and np.all(nnz[nc:] == 2)
        assert P.nnz == 2 * P.shape[0] - nc


def test_prolongation_matches_definition_pointwise(H4):
    """Eq. proj-1: value copied at old vertices, mean of the two ends at midpoints."""
    rng = np.random.default_rng(3)
    v, t = inputs.icosahedron()
    fv, ft, par = mesh.surface_hierarchy(v, t, 2)[2]
    w = rng.standard_normal(42)
    x = H4.P[2] @ w
    for i in range(fv.shape[0]):
        a, b = par[i]
        assert x[i] == (w[a] if a == b else (w[a] + w[b]) / 2)


def test_galerkin_pattern_is_coarse_mesh_pattern(H4):
    for f in range(2, 5):
        for j in range(1, f):
            G = H4.GA[f][j]
            A = H4.A[j]
            assert np.array_equal(G.indptr, A.indptr) and np.array_equal(G.indices, A.indices)
            Gm = H4.GM[f][j]
            assert np.array_equal(Gm.indptr, A.indptr) and np.array_equal(Gm.indices, A.indices)


def test_galerkin_rayleigh_quotient_identity(H4):
    """Eq. evalapprox: RQ of x on level j (Galerkin pair) = RQ of P x on level f."""
    rng = np.random.default_rng(4)
    f = 4
    for j in (1, 2, 3):
        x = rng.standard_normal(H4.A[j].shape[0])
        y = bmg.prolong_chain(H4, x, j, f)
        rq_c = (x @ (H4.GA[f][j] @ x)) / (x @ (H4.GM[f][j] @ x))
        rq_f = (y @ (H4.A[f] @ y)) / (y @ (H4.M[f] @ y))
        assert abs(rq_c - rq_f) < 1e-13 * abs(rq_f)
        assert abs(H4.GA[f][j] @ np.ones(x.shape[0])).max() < 1e-12  # kernel kept


def test_splitmix64_reference_value():
    # published first output of SplitMix64 seeded with 0
    assert multilevel.splitmix64(0) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("r", [1, 3])
def test_colouring_is_proper_and_greedy(r):
    v, t = inputs.icosahedron()
    fv, ft, _ = mesh.surface_hierarchy(v, t, r)[r]
    rp, col = mesh.csr_pattern(fv.shape[0], ft)
    c = multilevel.greedy_colouring(rp, col)
    n = fv.shape[0]
    prio = [(multilevel.splitmix64(i), i) for i in range(n)]
    for i in range(n):
        nb = [int(j) for j in col[rp[i]:rp[i + 1]] if j != i]
        assert all(c[j] != c[i] for j in nb)
        higher = {int(c[j]) for j in nb if prio[j] > prio[i]}
        assert int(c[i]) == min(set(range(len(nb) + 2)) - higher)   # smallest free colour
    assert c.max() + 1 <= 7


@pytest.mark.parametrize("sym", [False, True])
def test_multicolour_gs_equals_sequential_gs(H4, sym):
    A, M = H4.A[2], H4.M[2]
    rng = np.random.default_rng(7)
    x = rng.standard_normal(A.shape[0])
    b = rng.standard_normal(A.shape[0])
    s = 3.5
    seq = multilevel.gauss_seidel_sequential(A, M, x, b, s, H4.colour[2], symmetric=sym)
    mc = multilevel.mc_gauss_seidel(A, M, x[:, None], b[:, None], [s], H4.colour[2], 1,
                                    symmetric=sym)[:, 0]
    assert np.max(np.abs(seq - mc)) < 1e-13 * np.max(np.abs(seq))


def test_smoothers_fix_exact_solution_and_reduce_error(H4):
    A, M = H4.A[3], H4.M[3]
    rng = np.random.default_rng(8)
    xs = rng.standard_normal((A.shape[0], 2))
    s = [0.5, 2.5]
    b = multilevel.shifted_apply(A, M, xs, s)
    for fn in (lambda x: multilevel.jacobi(A, M, x, b, s, 2 / 3, 3),
               lambda x: multilevel.mc_gauss_seidel(A, M, x, b, s, H4.colour[3], 2)):
        assert np.max(np.abs(fn(xs) - xs)) < 1e-12
        x0 = xs + rng.standard_normal(xs.shape)
        e0 = np.linalg.norm(x0 - xs)
        assert np.linalg.norm(fn(x0) - xs) < 0.9 * e0


def test_jacobi_on_diagonal_system_is_exact_with_unit_damping():
    A = sp.diags([2.0, 3.0, 5.0]).tocsr()
    M = sp.diags([1.0, 1.0, 1.0]).tocsr()
    b = np.array([[1.0], [2.0], [3.0]])
    x = multilevel.jacobi(A, M, np.zeros((3, 1)), b, [1.0], 1.0, 1)
    assert np.allclose(x[:, 0], [1.0, 1.0, 0.75])


# ---- Kaczmarz relaxation (Sec. 5.3, Table 2) ------------------------------------
def _k_level(R=3):
    from oracle import bmg as _b
    from paper_1511_07042_gb300 import inputs as _in
    v, t = _in.icosahedron()
    H = _b.build_hierarchy(v, t, R, colour2=True)
    return H.A[R].tocsr(), H.M[R].tocsr(), H.colour2[R]


def test_distance2_colouring_is_proper():
    A, M, c2 = _k_level(2)
    G = (A != 0).astype(np.int64).toarray()
    near = (G @ G) > 0                                 # within two edges, brute force
    np.fill_diagonal(near, False)
    i, j = np.nonzero(near)
    assert np.all(c2[i] != c2[j])


def test_kaczmarz_multicolour_equals_sequential():
    A, M, c2 = _k_level(3)
    rng = np.random.default_rng(21)
    x0, b = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    s = 20.0                                           # indefinite: A - 20 M has negative eigenvalues
    seq = multilevel.kaczmarz_sequential(A, M, x0, b, s, c2, omega=0.9)
    par = multilevel.kaczmarz(A, M, x0[:, None], b[:, None], np.array([s]), c2, 1, 0.9)[:, 0]
    assert np.max(np.abs(par - seq)) <= 1e-12 * np.max(np.abs(seq))


def test_kaczmarz_is_sor_on_the_normal_equations():
    """Textbook identity: a Kaczmarz sweep from x0 is x0 + K^T y, y one SOR sweep from 0
    on (K K^T) y = b - K x0 in the same row order (dense, independent arithmetic)."""
    A, M, c2 = _k_level(2)
    s, omega = 7.5, 0.8
    K = (A - s * M).toarray()
    rng = np.random.default_rng(22)
    x0, b = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    KK = K @ K.T
    rhs = b - K @ x0
    y = np.zeros_like(b)
    for i in sorted(range(A.shape[0]), key=lambda v: (int(c2[v]), v)):
        y[i] += omega * (rhs[i] - KK[i] @ y) / KK[i, i]
    want = x0 + K.T @ y
    got = multilevel.kaczmarz(A, M, x0[:, None], b[:, None], np.array([s]), c2, 1, omega)[:, 0]
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))


def test_kaczmarz_error_never_grows_on_an_indefinite_system():
    """Each row step is an orthogonal projection onto a hyperplane through the
    solution, so the 2-norm of the error cannot grow (omega = 1), for any shift."""
    A, M, c2 = _k_level(3)
    s = 20.0
    K = (A - s * M).toarray()
    assert np.min(np.linalg.eigvalsh(0.5 * (K + K.T))) < 0
    rng = np.random.default_rng(23)
    b = rng.standard_normal(A.shape[0])
    xs = np.linalg.solve(K, b)
    x = np.zeros((A.shape[0], 1))
    errs = [np.linalg.norm(x[:, 0] - xs)]
    for _ in range(10):
        x = multilevel.kaczmarz(A, M, x, b[:, None], np.array([s]), c2, 1, 1.0)
        errs.append(np.linalg.norm(x[:, 0] - xs))
    assert all(e1 <= e0 * (1 + 1e-12) for e0, e1 in zip(errs, errs[1:])) and errs[-1] < errs[0]
