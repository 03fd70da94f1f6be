"""Surface meshes: uniform refinement with projection of new vertices onto the surface.

Oracle (test infrastructure only).

Sec. 3 (two-grid section, first paragraphs, and the figure on the octahedral
prolongation): the fine mesh is the uniform refinement of the coarse one; the new
vertices are the edge midpoints, projected onto the continuous surface.  Sec. 2.1:
every vertex lies on the surface.

Readings fixed here:
  * numbering: old vertices keep their indices; the midpoint of edge (i<j) gets index
    N_coarse + rank of (i,j) in the lexicographically sorted list of unique edges.
  * child triangles of t=(a,b,c), in this order, at indices 4t..4t+3:
        (a, m_ab, m_ca), (b, m_bc, m_ab), (c, m_ca, m_bc), (m_ab, m_bc, m_ca)
  * projection: radial.  Unit sphere: m / |m| (the closest point, Eq. lift).
    Star-shaped perturbed sphere: r(n) n with n = m / |m| and
        r(n) = 1 + a * sum_{l<=4, |m|<=l} c_lm Y_lm(n),
    Y_lm the real orthonormal spherical harmonics as Cartesian polynomials.
  * |m| = sqrt((x*x + y*y) + z*z), evaluated left to right; m = (v_i + v_j) * 0.5.
"""
from __future__ import annotations

import math

import numpy as np


def unique_edges(tris: np.ndarray) -> np.ndarray:
    """All edges (i<j) of a triangle list, lexicographically sorted, [E,2] int64."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]], axis=0)
    e = np.sort(e.astype(np.int64), axis=1)
    return np.unique(e, axis=0)  # np.unique on rows sorts lexicographically


def _norm3(m: np.ndarray) -> np.ndarray:
    return np.sqrt(m[:, 0] * m[:, 0] + m[:, 1] * m[:, 1] + m[:, 2] * m[:, 2])


def sh_basis(n: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics Y_lm, l<=4, at unit vectors n [P,3].

    Columns ordered l=0..4, m=-l..l (25 columns).  Standard Cartesian forms of the
    real harmonics (x, y, z on the unit sphere).
    """
    x, y, z = n[:, 0], n[:, 1], n[:, 2]
    pi = math.pi
    c00 = 0.5 * math.sqrt(1.0 / pi)
    c1 = math.sqrt(3.0 / (4.0 * pi))
    c2a = 0.5 * math.sqrt(15.0 / pi)
    c20 = 0.25 * math.sqrt(5.0 / pi)
    c22 = 0.25 * math.sqrt(15.0 / pi)
    c3a = 0.25 * math.sqrt(35.0 / (2.0 * pi))
    c3b = 0.5 * math.sqrt(105.0 / pi)
    c3c = 0.25 * math.sqrt(21.0 / (2.0 * pi))
    c30 = 0.25 * math.sqrt(7.0 / pi)
    c32 = 0.25 * math.sqrt(105.0 / pi)
    c4a = 0.75 * math.sqrt(35.0 / pi)
    c4b = 0.75 * math.sqrt(35.0 / (2.0 * pi))
    c4c = 0.75 * math.sqrt(5.0 / pi)
    c4d = 0.75 * math.sqrt(5.0 / (2.0 * pi))
    c40 = (3.0 / 16.0) * math.sqrt(1.0 / pi)
    c42 = (3.0 / 8.0) * math.sqrt(5.0 / pi)
    c44 = (3.0 / 16.0) * math.sqrt(35.0 / pi)
    one = np.ones_like(x)
    z4 = z * z * z * z
    cols = [
        c00 * one,
        c1 * y, c1 * z, c1 * x,
        c2a * x * y, c2a * y * z, c20 * (3.0 * z * z - 1.0), c2a * x * z,
        c22 * (x * x - y * y),
        c3a * y * (3.0 * x * x - y * y), c3b * x * y * z,
        c3c * y * (5.0 * z * z - 1.0), c30 * z * (5.0 * z * z - 3.0),
        c3c * x * (5.0 * z * z - 1.0), c32 * z * (x * x - y * y),
        c3a * x * (x * x - 3.0 * y * y),
        c4a * x * y * (x * x - y * y), c4b * y * z * (3.0 * x * x - y * y),
        c4c * x * y * (7.0 * z * z - 1.0), c4d * y * z * (7.0 * z * z - 3.0),
        c40 * (35.0 * z4 - 30.0 * z * z + 3.0),
        c4d * x * z * (7.0 * z * z - 3.0), c42 * (x * x - y * y) * (7.0 * z * z - 1.0),
        c4b * x * z * (x * x - 3.0 * y * y),
        c44 * (x * x * (x * x - 3.0 * y * y) - y * y * (3.0 * x * x - y * y)),
    ]
    return np.stack(cols, axis=1)


def radius(n: np.ndarray, amplitude: float, coefs) -> np.ndarray:
    """r(n) = 1 + a * sum c_lm Y_lm(n) for unit vectors n.

    The sum runs in the column order of sh_basis, one term at a time, so that its
    rounding is fixed (products and sums evaluated left to right, no fused
    multiply-add).
    """
    if amplitude == 0.0:
        return np.ones(n.shape[0])
    Y = sh_basis(n)
    c = np.asarray(coefs, dtype=np.float64)
    acc = Y[:, 0] * c[0]
    for q in range(1, 25):
        acc = acc + Y[:, q] * c[q]
    return 1.0 + amplitude * acc


def project(m: np.ndarray, amplitude: float = 0.0, coefs=None) -> np.ndarray:
    """Radial projection of points onto the (perturbed) sphere."""
    nrm = _norm3(m)
    n = m / nrm[:, None]
    if amplitude == 0.0:
        return n
    return radius(n, amplitude, coefs)[:, None] * n


def refine(verts: np.ndarray, tris: np.ndarray, amplitude: float = 0.0, coefs=None,
           project_new: bool = True):
    """One uniform refinement with projection (project_new=False keeps the flat
    midpoints, which makes the P1 spaces nested).

    Returns (fine_verts [N+E,3], fine_tris [4F,3] int32, parents [N+E,2] int32).
    parents[v] = (v, v) for an old vertex, (i, j) for the midpoint of edge (i<j).
    """
    n = verts.shape[0]
    edges = unique_edges(tris)
    ne = edges.shape[0]
    mid = (verts[edges[:, 0]] + verts[edges[:, 1]]) * 0.5
    newv = project(mid, amplitude, coefs) if project_new else mid
    fverts = np.concatenate([verts, newv], axis=0)

    # edge id lookup: key i*n + j for i<j
    keys = edges[:, 0] * n + edges[:, 1]

    def eid(a, b):
        lo = np.minimum(a, b).astype(np.int64)
        hi = np.maximum(a, b).astype(np.int64)
        return np.searchsorted(keys, lo * n + hi) + n

    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    mab, mbc, mca = eid(a, b), eid(b, c), eid(c, a)
    ch = np.stack([
        np.stack([a, mab, mca], 1), np.stack([b, mbc, mab], 1),
        np.stack([c, mca, mbc], 1), np.stack([mab, mbc, mca], 1)], axis=1)
    ftris = ch.reshape(-1, 3).astype(np.int32)

    parents = np.empty((n + ne, 2), dtype=np.int32)
    parents[:n, 0] = np.arange(n)
    parents[:n, 1] = np.arange(n)
    parents[n:] = edges
    return fverts, ftris, parents


def surface_hierarchy(coarse_verts, coarse_tris, refinements: int,
                      amplitude: float = 0.0, coefs=None):
    """Refine the input mesh `refinements` times.

    The input vertices are first projected onto the surface (every vertex lies on
    the surface, Sec. 2.1).  Returns a list of (verts, tris, parents) for
    refinement 0..refinements; parents is None at refinement 0.
    """
    v = project(np.asarray(coarse_verts, dtype=np.float64), amplitude, coefs)
    t = np.asarray(coarse_tris, dtype=np.int32)
    out = [(v, t, None)]
    for _ in range(refinements):
        v, t, p = refine(v, t, amplitude, coefs)
        out.append((v, t, p))
    return out


def csr_pattern(n: int, tris: np.ndarray):
    """Vertex adjacency (self included) as CSR: row_ptr [n+1], col [nnz] int32.

    Columns ascending within a row.
    """
    e = unique_edges(tris)
    rows = np.concatenate([e[:, 0], e[:, 1], np.arange(n)])
    cols = np.concatenate([e[:, 1], e[:, 0], np.arange(n)])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr.astype(np.int32), cols.astype(np.int32)
