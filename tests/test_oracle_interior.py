"""The interior workload's shift, sigma = 110, on its perturbed surface
(r = 1 + 0.1 sum c_lm Y_lm, l <= 4, c_lm seed 1003), at refinement 4 (2562
vertices), where LAPACK can give the whole spectrum.

The paper shows interior eigenvalues only near lambda = 20 (Sec. 5.3), within reach of
its coarse space.  Far above the part of the spectrum that the 42-vertex coarse level
resolves, the oracle's BFMG does not reach the cluster nearest sigma: it settles on
Ritz pairs of smaller eigenvalues (near 54-74 with Jacobi), with damped Jacobi and with
symmetric multicolour Gauss-Seidel alike; the paper's smoother for interior problems,
five multicolour Kaczmarz sweeps (Sec. 5.3, Table 2), gets closer (Ritz values near
86-109) but crawls (residual 3e-4 after 200 finest cycles, 0.99 per cycle) and still
holds pairs outside the cluster; with the adaptive shift the shift drifts down to the
mean Rayleigh quotient of the block (near 65) and the pairs with it.  These
tests record that behaviour against facts fixed outside the oracle: the dense pencil
spectrum (LAPACK) and the Sylvester inertia of A - s M (sparse LU)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bmg as obmg, certify
from paper_1511_07042_gb300 import inputs

SIGMA, K, NW = 110.0, 48, 21


@pytest.fixture(scope="module")
def surface():
    v, t = inputs.icosahedron()
    H = obmg.build_hierarchy(v, t, 4, amplitude=0.1, coefs=inputs.sh_coefficients(1003), colour2=True)
    A, M = H.A[4], H.M[4]
    w = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True)
    return H, A, M, w


def test_cluster_nearest_sigma_located_by_inertia(surface):
    H, A, M, w = surface
    near = np.sort(w[np.argsort(np.abs(w - SIGMA))[:NW]])
    lo, hi = near[0] - 1e-3, near[-1] + 1e-3
    assert 99.0 < near[0] and near[-1] < 120.0
    # Sylvester: the count of eigenvalues below each end of the cluster's interval
    assert certify.inertia_below(A, M, hi) - certify.inertia_below(A, M, lo) == NW


@pytest.mark.parametrize("smoother,nu,omega", [("jacobi", 2, 2 / 3), ("mcsgs", 1, 1.0)])
def test_bfmg_does_not_reach_the_cluster(surface, smoother, nu, omega):
    H, A, M, w = surface
    near = np.sort(w[np.argsort(np.abs(w - SIGMA))[:NW]])
    X0 = inputs.gaussian_block(162, K, 1013)
    res = obmg.bfmg(H, X0, K, NW, SIGMA, 1e-10, obmg.Options(smoother=smoother, nu=nu, omega=omega,
                                                            max_cycles=30))
    assert not res.converged and res.resid[:NW].max() > 1e-5
    # the wanted Ritz values are not the cluster nearest sigma: most of them are
    # eigenvalue approximations far below it
    lam = np.sort(res.lam[:NW])
    assert np.max(np.abs(lam - near)) > 10.0
    assert np.sum(lam < near[0] - 10.0) >= NW // 2, lam


def test_kaczmarz_gets_closer_but_does_not_reach_the_cluster(surface):
    """Five Kaczmarz sweeps (Table 2's setting) with the fixed shift: the residual
    stays above 1e-4 after 30 finest cycles and some wanted Ritz values are still
    more than 10 away from the cluster; with the adaptive shift (Alg. 3 step 4) the
    shift itself leaves the cluster for the block's mean Rayleigh quotient."""
    H, A, M, w = surface
    near = np.sort(w[np.argsort(np.abs(w - SIGMA))[:NW]])
    X0 = inputs.gaussian_block(162, K, 1013)
    res = obmg.bfmg(H, X0, K, NW, SIGMA, 1e-10, obmg.Options(smoother="kaczmarz", nu=5, omega=1.0, max_cycles=30))
    assert not res.converged and res.resid[:NW].max() > 1e-4
    lam = np.sort(res.lam[:NW])
    assert lam[0] > 80.0 and np.max(np.abs(lam - near)) > 10.0, lam
    ada = obmg.bfmg(H, X0, K, NW, SIGMA, 1e-10, obmg.Options(smoother="kaczmarz", nu=5, omega=1.0, max_cycles=30,
                                                            adaptive_shift=True))
    assert not ada.converged and ada.shifts[-1] < near[0] - 20.0
    assert np.all(np.sort(ada.lam[:NW]) < near[0] - 10.0)
