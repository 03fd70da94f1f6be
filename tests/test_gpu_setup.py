"""GPU set-up parity: meshes, CSR patterns, P, colouring bit-exact; matrices and
Galerkin operators against the FP64 oracle."""
import numpy as np
import pytest

from oracle import bmg as obmg, fem, mesh as omesh, multilevel
from paper_1511_07042_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[(0.0, None), (0.1, 1003)], ids=["sphere", "bumpy"])
def pair(request, gpu_bmg):
    amp, seed = request.param
    coefs = None if seed is None else inputs.sh_coefficients(seed)
    v, t = inputs.icosahedron()
    R = 5
    prob = gpu_bmg.Problem(v, t, R, amp, coefs)
    prob.hierarchy(R)
    H = obmg.build_hierarchy(v, t, R, amp, coefs)
    meshes = omesh.surface_hierarchy(v, t, R, amp, coefs)
    return prob, H, meshes, R


def test_meshes_bit_exact(pair):
    prob, H, meshes, R = pair
    for r in range(R + 1):
        gv, gt, gp = prob.mesh(r)
        ov, ot, op = meshes[r]
        assert gv.shape == ov.shape and np.array_equal(gv, ov), r   # bit-exact positions
        assert np.array_equal(gt, ot), r
        if op is not None:
            assert np.array_equal(gp, op), r


def test_csr_and_matrices(pair):
    prob, H, meshes, R = pair
    for r in range(1, R + 1):
        rp, col, a, m = prob.csr(r)
        orp, ocol = omesh.csr_pattern(meshes[r][0].shape[0], meshes[r][1])
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
        A, M = H.A[r], H.M[r]
        assert np.array_equal(A.indptr, rp) and np.array_equal(A.indices, col)
        # same element formulas, same order of accumulation: equal to the last bit
        assert np.array_equal(a, A.data), np.max(np.abs(a - A.data))
        assert np.array_equal(m, M.data), np.max(np.abs(m - M.data))


def test_colouring_bit_exact(pair):
    prob, H, meshes, R = pair
    for l in range(1, R + 1):
        c, nc = prob.colouring(l)
        assert np.array_equal(c, H.colour[l]) and nc == H.colour[l].max() + 1


def test_distance2_colouring_bit_exact(pair):
    """The Kaczmarz smoother's colouring: sequential greedy on the distance-2 graph in
    the same priority order, computed by the oracle from the square of the pattern."""
    prob, H, meshes, R = pair
    for l in range(1, R + 1):
        A = H.A[l]
        want = multilevel.greedy_colouring(*multilevel.distance2_pattern(A.indptr, A.indices))
        c, nc = prob.colouring2(l)
        assert np.array_equal(c, want) and nc == want.max() + 1, l


def test_galerkin_operators(pair):
    prob, H, meshes, R = pair
    for f in range(2, R + 1):
        for j in range(1, f):
            a, m = prob.galerkin(f, j)
            GA, GM = H.GA[f][j], H.GM[f][j]
            assert np.allclose(a, GA.data, rtol=0, atol=1e-13 * abs(GA.data).max())
            assert np.allclose(m, GM.data, rtol=0, atol=1e-13 * abs(GM.data).max())


def test_perturbed_vertices_lie_on_surface(pair):
    prob, H, meshes, R = pair
    gv, _, _ = prob.mesh(R)
    n = gv / np.linalg.norm(gv, axis=1)[:, None]
    amp = 0.0 if H.A[1] is None else None
    r = np.linalg.norm(gv, axis=1)
    # radial distance equals r(n) (1 for the unit sphere) to rounding
    coef_r = omesh.radius(n, 0.1, inputs.sh_coefficients(1003)) if not np.allclose(r, 1.0) else np.ones_like(r)
    assert np.max(np.abs(r - coef_r)) < 1e-14
