"""P1 surface finite elements: stiffness A and mass M on flat triangles.

Oracle (test infrastructure only).

Eq. (bl-dis): a_h(u,v) = int_{Gamma_h} grad_G u . grad_G v,  b_h(u,v) = int u v, on
the piecewise-flat surface; Eq. (sp-fe): continuous piecewise-linear space; the
matrix form of the pencil is (A_h, M_h) (Sec. 4.1, matrix form of Alg. 2).

On one flat triangle with vertices (a,b,c) the surface gradient is the planar
gradient in the triangle's plane (Sec. 2.1, constant normal n_T), which gives the
cotangent formula (textbook P1 Laplacian):
    A^T_ab = -1/2 cot(theta_c)          theta_c = angle at c, opposite edge ab
    A^T_aa = 1/2 (cot theta_b + cot theta_c)
and the consistent P1 mass
    M^T = |T|/12 [[2,1,1],[1,2,1],[1,1,2]].
cot(theta_c) = (pa-pc).(pb-pc) / |(pa-pc) x (pb-pc)|,  |T| = 1/2 |(pb-pa) x (pc-pa)|.
Global matrices are accumulated element by element in triangle order into the CSR
pattern of the vertex adjacency.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import csr_pattern


def _cross(u, v):
    return np.stack([u[:, 1] * v[:, 2] - u[:, 2] * v[:, 1],
                     u[:, 2] * v[:, 0] - u[:, 0] * v[:, 2],
                     u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]], axis=1)


def _dot(u, v):
    return u[:, 0] * v[:, 0] + u[:, 1] * v[:, 1] + u[:, 2] * v[:, 2]


def _norm(u):
    return np.sqrt(_dot(u, u))


def element_matrices(verts: np.ndarray, tris: np.ndarray):
    """Per-triangle 3x3 stiffness and mass blocks, [F,3,3] each."""
    pa, pb, pc = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]

    def cot(p, q, apex):  # cot of the angle at `apex` between edges to p and q
        u, v = p - apex, q - apex
        return _dot(u, v) / _norm(_cross(u, v))

    cot_a = cot(pb, pc, pa)
    cot_b = cot(pc, pa, pb)
    cot_c = cot(pa, pb, pc)
    area = 0.5 * _norm(_cross(pb - pa, pc - pa))
    F = tris.shape[0]
    K = np.empty((F, 3, 3))
    K[:, 0, 1] = K[:, 1, 0] = -0.5 * cot_c
    K[:, 1, 2] = K[:, 2, 1] = -0.5 * cot_a
    K[:, 0, 2] = K[:, 2, 0] = -0.5 * cot_b
    K[:, 0, 0] = 0.5 * (cot_b + cot_c)
    K[:, 1, 1] = 0.5 * (cot_c + cot_a)
    K[:, 2, 2] = 0.5 * (cot_a + cot_b)
    M = np.empty((F, 3, 3))
    off = area / 12.0
    dia = area / 6.0
    for i in range(3):
        for j in range(3):
            M[:, i, j] = dia if i == j else off
    return K, M, area


def assemble(verts: np.ndarray, tris: np.ndarray):
    """Global P1 stiffness A and mass M as scipy CSR (sorted columns), float64."""
    n = verts.shape[0]
    row_ptr, col = csr_pattern(n, tris)
    K, Me, _ = element_matrices(verts, tris)
    # CSR slot of every (tri, i, j) local entry
    r = np.repeat(tris, 3, axis=1).reshape(-1, 3, 3)        # r[t,i,j] = tris[t,i]
    c = np.tile(tris, (1, 3)).reshape(-1, 3, 3)             # c[t,i,j] = tris[t,j]
    r = r.reshape(-1).astype(np.int64)
    c = c.reshape(-1).astype(np.int64)
    # CSR entries sorted by (row, col) => key row*n+col is globally ascending
    slot_row = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    keys = slot_row * n + col.astype(np.int64)
    slot = np.searchsorted(keys, r * n + c)
    a_val = np.zeros(col.shape[0])
    m_val = np.zeros(col.shape[0])
    np.add.at(a_val, slot, K.reshape(-1))  # unbuffered: triangle order
    np.add.at(m_val, slot, Me.reshape(-1))
    A = sp.csr_matrix((a_val, col, row_ptr), shape=(n, n))
    M = sp.csr_matrix((m_val, col, row_ptr), shape=(n, n))
    return A, M
