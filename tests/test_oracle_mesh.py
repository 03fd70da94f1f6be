"""Pins of the oracle's surface meshes against facts the paper and geometry fix."""
import math
import os

import numpy as np
import pytest

from oracle import mesh
from paper_1511_07042_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def test_icosahedron_input_is_regular_and_outward():
    v, t = inputs.icosahedron()
    assert v.shape == (12, 3) and t.shape == (20, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    e = mesh.unique_edges(t)
    assert e.shape[0] == 30
    el = np.linalg.norm(v[e[:, 0]] - v[e[:, 1]], axis=1)
    assert np.ptp(el) < 1e-14                       # all 30 edges equal
    c = v[t].mean(axis=1)
    nrm = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    assert np.all(np.sum(nrm * c, axis=1) > 0)      # outward orientation


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_counts_euler_degrees(r):
    v, t = inputs.icosahedron()
    H = mesh.surface_hierarchy(v, t, r)
    fv, ft, par = H[r]
    N = inputs.n_vertices(r)
    E = mesh.unique_edges(ft).shape[0]
    F = ft.shape[0]
    assert fv.shape[0] == N and E == 3 * N - 6 and F == 2 * N - 4
    assert N - E + F == 2                           # Euler characteristic of S^2
    deg = np.bincount(mesh.unique_edges(ft).ravel(), minlength=N)
    assert np.sum(deg == 5) == 12 and np.sum(deg == 6) == N - 12
    row_ptr, col = mesh.csr_pattern(N, ft)
    assert row_ptr[-1] == 7 * N - 12               # nnz = N + 2E
    # every vertex on the unit sphere to rounding (Sec. 2.1: vertices lie on Gamma)
    assert np.max(np.abs(np.linalg.norm(fv, axis=1) - 1.0)) < 4e-16


def test_dof_counts_golden():
    for nc, r, nf in load("dof_counts.txt"):
        n = int(nc)
        for _ in range(int(r)):
            n = 4 * n - 6
        assert n == int(nf)


def test_refinement_numbering_and_children():
    v, t = inputs.icosahedron()
    fv, ft, par = mesh.refine(v, t)
    e = mesh.unique_edges(t)
    # midpoint of the lexicographically first edge gets index 12
    assert tuple(par[12]) == tuple(e[0]) and tuple(par[11]) == (11, 11)
    # children of triangle 0 = (a, m_ab, m_ca), (b, m_bc, m_ab), (c, m_ca, m_bc), (m_ab, m_bc, m_ca)
    a, b, c = t[0]

    def m(i, j):
        i, j = min(i, j), max(i, j)
        return 12 + int(np.nonzero((e[:, 0] == i) & (e[:, 1] == j))[0][0])
    want = [[a, m(a, b), m(c, a)], [b, m(b, c), m(a, b)], [c, m(c, a), m(b, c)],
            [m(a, b), m(b, c), m(c, a)]]
    assert np.array_equal(ft[:4], np.array(want))
    # new vertex = normalised midpoint of its parents
    mid = 0.5 * (v[par[12, 0]] + v[par[12, 1]])
    assert np.allclose(fv[12], mid / np.linalg.norm(mid), atol=1e-16)
    # children keep the parent's orientation
    for q in range(4):
        p = fv[ft[q]]
        nq = np.cross(p[1] - p[0], p[2] - p[0])
        assert np.dot(nq, p.mean(axis=0)) > 0


def _rotation(axis, ang):
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_icosahedral_symmetry_of_refined_mesh():
    """A 72-degree rotation about a vertex maps the refined vertex set onto itself."""
    v, t = inputs.icosahedron()
    fv = mesh.surface_hierarchy(v, t, 3)[3][0]
    R = _rotation(v[0], 2 * math.pi / 5)
    rv = fv @ R.T
    # nearest-neighbour match
    d = np.linalg.norm(rv[:, None, :] - fv[None, :, :], axis=2).min(axis=1)
    assert d.max() < 1e-13


def test_spherical_harmonics_orthonormal_on_fine_mesh():
    """Y_lm from the radius model are L2-orthonormal on S^2 (quadrature by centroids)."""
    v, t = inputs.icosahedron()
    fv, ft, _ = mesh.surface_hierarchy(v, t, 6)[6]
    c = fv[ft].mean(axis=1)
    c = c / np.linalg.norm(c, axis=1)[:, None]
    area = 0.5 * np.linalg.norm(np.cross(fv[ft[:, 1]] - fv[ft[:, 0]], fv[ft[:, 2]] - fv[ft[:, 0]]), axis=1)
    w = area * (4 * math.pi / area.sum())
    Y = mesh.sh_basis(c)
    G = Y.T @ (Y * w[:, None])
    assert np.max(np.abs(G - np.eye(25))) < 2e-3


def test_perturbed_projection_is_radial():
    v, t = inputs.icosahedron()
    coefs = inputs.sh_coefficients(1003)
    H = mesh.surface_hierarchy(v, t, 2, amplitude=0.1, coefs=coefs)
    fv = H[2][0]
    n = fv / np.linalg.norm(fv, axis=1)[:, None]
    r = mesh.radius(n, 0.1, coefs)
    assert np.allclose(np.linalg.norm(fv, axis=1), r, rtol=1e-14)
    # the coarse input vertices are projected too
    assert np.allclose(H[0][0], mesh.radius(v, 0.1, coefs)[:, None] * v)
