"""Pins of the oracle's down-leg (Alg. 3 step 3, "from level k back to level 1";
`vleg_levels` and `source_smoothing`), by facts of multigrid that do not depend on
the oracle's own code:

* Two-level exactness.  With one coarse level and a coarse smoother run to
  convergence, the correction is the Galerkin coarse-grid correction
  x_s + P (P^T K P)^{-1} P^T (b - K x_s), K = A - sigma M, x_s the fine pre-smoothed
  iterate; P and K are taken from the hierarchy's prolongation and assembled
  matrices, not from its stored Galerkin operators.
* h-independence.  As a linear solver for (A - sigma M) x = b (sigma < 0, so K is
  positive definite), the V-leg reduces the energy-norm error by a factor that does
  not grow under refinement, while plain smoothing (vcycle_depth = 0) slows towards 1.
* Eigen cycles.  The finest-level BMG cycles to a fixed tolerance stay bounded under
  refinement with the V-leg and grow without it (the behaviour Sec. 5.3 relies on).

Planted mistakes in a copy of the down-leg (wrong restriction scale, a coarse
correction left unprolongated, the wrong sign of the residual) fail these pins.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bmg as obmg, multilevel
from paper_1511_07042_gb300 import inputs

SIGMA = -1.0   # K = A + M: symmetric positive definite on every level


def hierarchy(R):
    v, t = inputs.icosahedron()
    return obmg.build_hierarchy(v, t, R)


def run_leg(H, f, X, b, opt, leg=None):
    """source_smoothing as a linear iteration for (A - SIGMA M) x = b: with the
    shifted form, s = SIGMA and B = MU * theta, so MU = b and theta = 1."""
    leg = leg or obmg.source_smoothing
    ones = np.ones(b.shape[1])
    return leg(H, f, X, b, ones, ones, SIGMA, opt)


def test_two_level_correction_is_the_galerkin_coarse_correction():
    H = hierarchy(3)
    f = 3
    A, M, P = H.A[f], H.M[f], H.P[f]
    K = (A - SIGMA * M).tocsr()
    rng = np.random.default_rng(31)
    b = rng.standard_normal((A.shape[0], 3))
    X = rng.standard_normal((A.shape[0], 3))
    nu = 3000                                   # the 162-vertex coarse smoother converges
    opt = obmg.Options(smoother="jacobi", nu=nu, omega=2 / 3, vcycle_depth=1)
    assert obmg.vleg_levels(H, f, np.full(3, SIGMA), opt) == [2]
    got = run_leg(H, f, X, b, opt)
    xs = multilevel.jacobi(A, M, X, b, np.full(3, SIGMA), 2 / 3, nu)
    Kc = (P.T @ K @ P).tocsc()
    want = xs + P @ spla.splu(Kc).solve(P.T @ (b - K @ xs))
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def energy_rate(H, f, opt, leg=None, iters=12):
    A, M = H.A[f], H.M[f]
    K = (A - SIGMA * M).tocsc()
    b = np.random.default_rng(f).standard_normal((A.shape[0], 2))
    xs = spla.splu(K).solve(b)
    x = np.zeros_like(b)
    errs = []
    for _ in range(iters):
        x = run_leg(H, f, x, b, opt, leg)
        e = x - xs
        errs.append(np.sqrt(np.sum(e * (K @ e))))
    return (errs[-1] / errs[5]) ** (1.0 / (iters - 6))


@pytest.fixture(scope="module")
def hierarchies():
    return {R: hierarchy(R) for R in (3, 4, 5)}


def test_vleg_rate_is_h_independent(hierarchies):
    vleg = [energy_rate(hierarchies[R], R, obmg.Options()) for R in (3, 4, 5)]
    plain = [energy_rate(hierarchies[R], R, obmg.Options(vcycle_depth=0)) for R in (3, 4, 5)]
    assert max(vleg) <= 0.9 and max(vleg) - min(vleg) <= 0.03, vleg
    assert min(plain) >= 0.97 and plain[0] < plain[1] < plain[2], plain


def test_bfmg_finest_cycles_bounded_with_vleg_only(hierarchies):
    counts = {}
    for R in (3, 4, 5):
        X0 = inputs.gaussian_block(162, 20, 1001)
        for depth in (99, 0):
            res = obmg.bfmg(hierarchies[R], X0, 20, 16, 0.0, 1e-9,
                            obmg.Options(vcycle_depth=depth, max_cycles=80))
            counts[R, depth] = (res.cycles[-1], res.converged)
    assert all(counts[R, 99][1] and counts[R, 99][0] <= 25 for R in (3, 4, 5)), counts
    assert counts[3, 0][0] >= 2 * counts[3, 99][0], counts
    assert not counts[4, 0][1] and not counts[5, 0][1], counts


# ---- planted mistakes (copies of the down-leg with one error each) -------------
def _leg_with(mistake):
    def leg(H, f, U, MU, theta, lam, sigma, opt):
        s = np.full(lam.shape, sigma)
        B = MU * theta[None, :]
        A, M = H.A[f], H.M[f]
        X = obmg.smooth(A, M, U, B, s, H.colour[f], opt)
        levels = obmg.vleg_levels(H, f, s, opt)
        sign = -1.0 if mistake == "sign" else 1.0
        r = {f: sign * (B - multilevel.shifted_apply(A, M, X, s))}
        e = {}
        for idx, j in enumerate(levels):
            Ga, Gm = H.GA[f][j], H.GM[f][j]
            scale = 0.5 if mistake == "restriction" else 1.0
            rj = scale * (H.P[j + 1].T @ r[j + 1])
            e[j] = obmg.smooth(Ga, Gm, np.zeros_like(rj), rj, s, H.colour[j], opt)
            if idx + 1 < len(levels):
                r[j] = rj - multilevel.shifted_apply(Ga, Gm, e[j], s)
        if mistake != "unprolongated":
            for j in reversed(levels[1:]):
                e[j + 1] = e[j + 1] + H.P[j + 1] @ e[j]
        return X + H.P[f] @ e[levels[0]]
    return leg


def test_planted_mistakes_fail_the_pins(hierarchies):
    # the faithful copy passes: it is the oracle's down-leg
    H = hierarchies[4]
    ok = energy_rate(H, 4, obmg.Options(), _leg_with(None))
    assert abs(ok - energy_rate(H, 4, obmg.Options())) < 1e-12
    # a halved restriction no longer gives the Galerkin correction
    H3 = hierarchy(3)
    rng = np.random.default_rng(31)
    b = rng.standard_normal((H3.A[3].shape[0], 3))
    X = rng.standard_normal((H3.A[3].shape[0], 3))
    opt = obmg.Options(smoother="jacobi", nu=3000, omega=2 / 3, vcycle_depth=1)
    exact = run_leg(H3, 3, X, b, opt)
    wrong = run_leg(H3, 3, X, b, opt, _leg_with("restriction"))
    assert np.max(np.abs(wrong - exact)) > 1e-7 * np.max(np.abs(exact))    # 1e-10 holds for the oracle
    # each mistake (halved restriction, deeper corrections left out, the residual's
    # sign flipped) moves the rate out of the bound of the V-leg pin
    for mistake in ("restriction", "unprolongated", "sign"):
        rates = [energy_rate(hierarchies[R], R, obmg.Options(), _leg_with(mistake)) for R in (3, 4, 5)]
        assert not (max(rates) <= 0.9 and max(rates) - min(rates) <= 0.03), (mistake, rates)
