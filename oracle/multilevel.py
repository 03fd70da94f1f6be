"""Prolongation, restriction, Galerkin operators, colouring and smoothers.

Oracle (test infrastructure only).

Eq. (proj-1): the geometric prolongation keeps the value at an old vertex and takes
the mean of the two parent values at a projected midpoint, so P_h has entries 1 and
1/2 (Sec. 3, the matrix P_h after Eq. proj-1).  The restriction is P_H = P_h^T.
Composite operators (Sec. 1.1, Eq. evalapprox): P_l = P_1^0 ... P_l^{l-1} and the
Galerkin coarse matrices A_l = P_l^T A_0 P_l, for which the Rayleigh quotient of a
coarse vector equals the fine Rayleigh quotient of its prolongation.

Smoothers for the shifted source problems (A - s_i M) x_i = b_i (Eq. pb-f-aux-mat,
Eq. pb-m-s; Remark on smoothers after Alg. 1; Sec. 5.3, symmetric Gauss-Seidel):
  * damped Jacobi: x <- x + omega D^{-1} (b - (A - s M) x), D = diag(A) - s diag(M)
  * multicolour Gauss-Seidel: the same update applied colour by colour (ascending),
    using the newest values; symmetric variant = ascending then descending colours.
Rows of one colour are not adjacent, so updating a colour at once equals the
sequential Gauss-Seidel sweep over that colour's rows.
Colouring: sequential greedy in descending priority; priority(v) = (splitmix64(v), v);
each vertex takes the smallest colour unused by its already coloured neighbours.

Kaczmarz relaxation (Sec. 5.3, Table 2: the paper's smoother for the shifted indefinite
source problems): row r of K = A - s M projects x onto the hyperplane of its equation,
x <- x + omega (b_r - k_r^T x) / ||k_r||^2 k_r, which changes every x_j with k_rj != 0.
Two rows can be projected at once when no column carries a nonzero of both, i.e.
when their vertices are more than two edges apart; a greedy colouring of the
distance-2 graph (same priorities) groups such rows, and projecting the rows of one
colour at once equals the sequential sweep in (colour, index) order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MASK64 = (1 << 64) - 1


def prolongation(parents: np.ndarray, n_coarse: int) -> sp.csr_matrix:
    """P [N_fine, N_coarse]: 1 at (v, v) for old vertices, 1/2 at both parents."""
    nf = parents.shape[0]
    rows, cols, vals = [], [], []
    for v in range(nf):
        i, j = int(parents[v, 0]), int(parents[v, 1])
        if i == j:
            rows.append(v); cols.append(i); vals.append(1.0)
        else:
            rows += [v, v]; cols += [i, j]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, n_coarse))


def galerkin(P: sp.csr_matrix, A: sp.csr_matrix) -> sp.csr_matrix:
    """P^T A P with sorted indices."""
    G = (P.T @ A @ P).tocsr()
    G.sort_indices()
    return G


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood 2014) of the integer x."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def greedy_colouring(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Greedy colouring in descending (splitmix64(v), v) priority; int32 colours."""
    n = row_ptr.shape[0] - 1
    order = sorted(range(n), key=lambda v: (splitmix64(v), v), reverse=True)
    colour = np.full(n, -1, dtype=np.int64)
    for v in order:
        used = set()
        for p in range(row_ptr[v], row_ptr[v + 1]):
            u = col[p]
            if u != v and colour[u] >= 0:
                used.add(int(colour[u]))
        c = 0
        while c in used:
            c += 1
        colour[v] = c
    return colour.astype(np.int32)


def shifted_diag(A, M, s):
    """D[:, i] = diag(A) - s_i diag(M), [N, k]."""
    return A.diagonal()[:, None] - M.diagonal()[:, None] * np.asarray(s)[None, :]


def shifted_apply(A, M, X, s):
    """(A - s_i M) x_i for every column i."""
    return A @ X - (M @ X) * np.asarray(s)[None, :]


def jacobi(A, M, X, B, s, omega: float, nu: int):
    """nu damped-Jacobi sweeps on (A - s_i M) x_i = b_i, columnwise shifts s."""
    D = shifted_diag(A, M, s)
    X = X.copy()
    for _ in range(nu):
        R = B - shifted_apply(A, M, X, s)
        X = X + omega * R / D
    return X


def mc_gauss_seidel(A, M, X, B, s, colour, nu: int, symmetric: bool = True):
    """nu multicolour (symmetric) Gauss-Seidel sweeps on (A - s_i M) x_i = b_i."""
    D = shifted_diag(A, M, s)
    X = X.copy()
    ncol = int(colour.max()) + 1
    rows_of = [np.nonzero(colour == c)[0] for c in range(ncol)]
    order = list(range(ncol))
    if symmetric:
        order = order + order[::-1]
    s = np.asarray(s)[None, :]
    for _ in range(nu):
        for c in order:
            r = rows_of[c]
            Ar, Mr = A[r], M[r]
            R = B[r] - (Ar @ X - (Mr @ X) * s)
            X[r] = X[r] + R / D[r]
    return X


def gauss_seidel_sequential(A, M, x, b, s: float, colour, symmetric: bool = True):
    """One sequential Gauss-Seidel sweep over rows ordered by (colour, index).

    Pure-Python definition used to pin the multicolour form on small meshes.
    """
    A = A.tocsr(); M = M.tocsr()
    x = x.copy()
    n = x.shape[0]
    rows = sorted(range(n), key=lambda v: (int(colour[v]), v))
    if symmetric:
        rows = rows + sorted(range(n), key=lambda v: (-int(colour[v]), v))
    for i in rows:
        acc = 0.0
        for p in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[p]
            acc += (A.data[p] - s * M.data[p]) * x[j]
        d = A[i, i] - s * M[i, i]
        x[i] = x[i] + (b[i] - acc) / d
    return x


def distance2_pattern(row_ptr: np.ndarray, col: np.ndarray):
    """CSR (row_ptr, col) of the vertices within two edges of each vertex (itself
    included), ascending columns."""
    n = row_ptr.shape[0] - 1
    G = sp.csr_matrix((np.ones(col.shape[0]), col, row_ptr), shape=(n, n))
    G2 = (G @ G).tocsr()
    G2.sort_indices()
    return G2.indptr.astype(np.int64), G2.indices.astype(np.int64)


def row_norms(A, M):
    """Per row: sum_j a_rj^2, sum_j a_rj m_rj, sum_j m_rj^2 (shared pattern), so that
    ||a_r - s m_r||^2 = na - 2 s nam + s^2 nm."""
    A = A.tocsr(); M = M.tocsr()
    na = np.asarray(A.multiply(A).sum(axis=1)).ravel()
    nam = np.asarray(A.multiply(M).sum(axis=1)).ravel()
    nm = np.asarray(M.multiply(M).sum(axis=1)).ravel()
    return na, nam, nm


def kaczmarz(A, M, X, B, s, colour2, nu: int, omega: float = 1.0):
    """nu multicolour Kaczmarz sweeps on (A - s_i M) x_i = b_i, colours ascending,
    colour2 a distance-2 colouring."""
    A = A.tocsr(); M = M.tocsr()
    X = X.copy()
    s = np.asarray(s)[None, :]
    na, nam, nm = row_norms(A, M)
    ncol = int(colour2.max()) + 1
    rows_of = [np.nonzero(colour2 == c)[0] for c in range(ncol)]
    for _ in range(nu):
        for c in range(ncol):
            r = rows_of[c]
            Ar, Mr = A[r], M[r]
            R = B[r] - (Ar @ X - (Mr @ X) * s)
            nrm = na[r][:, None] - 2.0 * s * nam[r][:, None] + s * s * nm[r][:, None]
            Cf = omega * R / nrm
            X = X + (Ar.T @ Cf) - (Mr.T @ Cf) * s
    return X


def kaczmarz_sequential(A, M, x, b, s: float, colour2, omega: float = 1.0):
    """One sequential Kaczmarz sweep over the rows in (colour, index) order.

    Pure-Python definition used to pin the multicolour form on small meshes.
    """
    A = A.tocsr(); M = M.tocsr()
    x = x.copy()
    n = x.shape[0]
    for i in sorted(range(n), key=lambda v: (int(colour2[v]), v)):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        k = A.data[A.indptr[i]:A.indptr[i + 1]] - s * M.data[M.indptr[i]:M.indptr[i + 1]]
        res = b[i] - float(np.dot(k, x[cols]))
        x[cols] = x[cols] + omega * res / float(np.dot(k, k)) * k
    return x
