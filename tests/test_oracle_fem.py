"""Pins of the oracle's P1 assembly (Eq. bl-dis, sp-fe) and spectrum (Lemma apriori)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import certify, fem, mesh, multilevel
from paper_1511_07042_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def level(r, amplitude=0.0, coefs=None):
    v, t = inputs.icosahedron()
    fv, ft, _ = mesh.surface_hierarchy(v, t, r, amplitude, coefs)[r]
    A, M = fem.assemble(fv, ft)
    return fv, ft, A, M


def test_element_matrices_right_triangle():
    """Unit right triangle: textbook P1 stiffness 1/2[[2,-1,-1],[-1,1,0],[-1,0,1]],
    mass |T|/12 [[2,1,1],[1,2,1],[1,1,2]] with |T| = 1/2."""
    v = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    t = np.array([[0, 1, 2]])
    K, M, area = fem.element_matrices(v, t)
    Kw = 0.5 * np.array([[2.0, -1, -1], [-1, 1, 0], [-1, 0, 1]])
    Mw = (0.5 / 12.0) * np.array([[2.0, 1, 1], [1, 2, 1], [1, 1, 2]])
    assert np.allclose(K[0], Kw, atol=1e-15) and np.allclose(M[0], Mw, atol=1e-16)
    assert area[0] == 0.5


def test_element_stiffness_rotation_invariant_and_matches_gradient_formula():
    """K^T_ij = |T| grad(phi_i).grad(phi_j) computed from the inverse Jacobian."""
    rng = np.random.default_rng(5)
    p = rng.standard_normal((3, 3))
    K, _, area = fem.element_matrices(p, np.array([[0, 1, 2]]))
    e1, e2 = p[1] - p[0], p[2] - p[0]
    J = np.stack([e1, e2], axis=1)                      # 3x2
    G = np.linalg.pinv(J)                               # rows: grads of bary 1, 2
    g = np.vstack([-G[0] - G[1], G[0], G[1]])
    Kg = area[0] * g @ g.T
    assert np.allclose(K[0], Kg, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("r", [1, 3, 5])
def test_assembly_invariants(r):
    fv, ft, A, M = level(r)
    one = np.ones(A.shape[0])
    scale = abs(A).max()
    assert np.max(np.abs(A @ one)) < 1e-13 * scale          # constants in the kernel
    assert abs(A - A.T).max() < 1e-15 * scale
    assert abs(M - M.T).max() == 0.0
    area = 0.5 * np.linalg.norm(np.cross(fv[ft[:, 1]] - fv[ft[:, 0]], fv[ft[:, 2]] - fv[ft[:, 0]]), axis=1).sum()
    assert abs(one @ (M @ one) - area) < 1e-13 * area        # 1^T M 1 = sum |T|
    assert np.array_equal(A.indptr, M.indptr) and np.array_equal(A.indices, M.indices)
    if r <= 3:
        w = np.linalg.eigvalsh(M.toarray())
        assert w.min() > 0                                   # M SPD


def test_area_converges_to_4pi_at_second_order():
    errs = []
    for r in (2, 3, 4, 5):
        _, _, _, M = level(r)
        one = np.ones(M.shape[0])
        errs.append(4 * math.pi - one @ (M @ one))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4.0) < 0.1)               # O(h^2) = O(DoF^-1)


def test_flat_refinement_gives_nested_galerkin_identity():
    """Refining without projection keeps flat midpoints: P1 spaces are nested and
    P^T A_h P = A_H, P^T M_h P = M_H (variational property)."""
    v, t = inputs.icosahedron()
    A0, M0 = fem.assemble(v, t)
    fv, ft, par = mesh.refine(v, t, project_new=False)
    A1, M1 = fem.assemble(fv, ft)
    P = multilevel.prolongation(par, 12)
    assert abs(P.T @ A1 @ P - A0).max() < 1e-14 * abs(A0).max()
    assert abs(P.T @ M1 @ P - M0).max() < 1e-15 * abs(M0).max()


def test_spectrum_structure_and_rate():
    """Dense eigensolves: lambda_0 = 0, multiplets near l(l+1), O(DoF^-1) convergence
    (Lemma apriori; Sec. 5 intro; Table 1's r ~= 1)."""
    gold = np.loadtxt(os.path.join(GOLDEN, "sphere_spectrum.txt"), comments="#")
    errs = {}
    for r in (2, 3, 4):
        _, _, A, M = level(r)
        w = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True)
        assert abs(w[0]) < 1e-14 * w[-1]                   # rounding of lambda_max scale
        for l, lam, mult, j0, j1 in gold[:4]:
            blk = w[int(j0):int(j1) + 1]
            assert np.all(np.abs(blk - lam) < 0.6 * max(lam, 1) * 4.0 ** (2 - r) + 1e-12)
            errs.setdefault(int(l), []).append(np.max(np.abs(blk - lam)))
    for l in (1, 2, 3):
        e = np.array(errs[l])
        rate = np.log(e[:-1] / e[1:]) / np.log(4.0)
        assert np.all(np.abs(rate - 1.0) < 0.1), (l, rate)


def test_icosahedral_multiplets():
    """On the icosahedral mesh, l=0,1,2 stay degenerate (irreps of size 1,3,5) and
    l=3 splits 3+4."""
    _, _, A, M = level(3)
    w = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True)
    groups = certify.cluster_groups(w[:16], rel_gap=1e-9)
    assert [len(g) for g in groups] == [1, 3, 5, 3, 4] or [len(g) for g in groups] == [1, 3, 5, 4, 3]


def test_eigen_identity_lemma():
    """Lemma eigenid: RQ(w) - lambda = [a(w-u,w-u) - lambda b(w-u,w-u)] / b(w,w)."""
    _, _, A, M = level(2)
    w, V = sla.eigh(A.toarray(), M.toarray())
    u, lam = V[:, 5], w[5]
    x = u + 0.1 * np.random.default_rng(1).standard_normal(u.shape)
    lhs = (x @ (A @ x)) / (x @ (M @ x)) - lam
    d = x - u
    rhs = (d @ (A @ d) - lam * (d @ (M @ d))) / (x @ (M @ x))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_perturbed_sphere_weyl_count():
    """Weyl's law: N(lambda) ~ Area * lambda / (4 pi) on a closed surface."""
    coefs = inputs.sh_coefficients(1003)
    fv, ft, A, M = level(4, 0.1, coefs)
    area = np.ones(A.shape[0]) @ (M @ np.ones(A.shape[0]))
    cnt = certify.inertia_below(A, M, 110.0)
    assert abs(cnt - area * 110.0 / (4 * math.pi)) < 0.15 * cnt
