"""Bootstrap multigrid eigensolver: enriched Rayleigh-Ritz, BMG cycle, BFMG driver.

Oracle (test infrastructure only).

Follows Alg. 2 (two-grid bootstrap with an enriched coarse space), Alg. 3 (BMG
V-cycle between level 1 and level k) and Alg. 4 (BFMG), with the enriched block
matrices of Sec. 4.1:
    A_{H,h} = [[A_H, P_H A_h U], [U^T A_h P_h, U^T A_h U]]   (and M_{H,h} alike)
where the coarse block is the composite Galerkin matrix Q^T A Q of level 1
(Sec. 1.1, Eq. evalapprox) and Q = P_2 ... P_f is the composite prolongation from
level 1 to the current finest level f.

Readings of the paper used here (each listed in the design notes):
  * X0: a seeded Gaussian block on level 2 (instead of coarse eigenvectors), so that
    k may exceed dim V_{h_1} = 42.
  * b-orthogonalisation (Alg. 2 step 3) and the eigensolve in V_H + X_h (step 4) are
    done together by SVQB: M_hat is scaled to unit diagonal, eigendecomposed,
    directions with eigenvalue below tau*max dropped, which M-orthonormalises the
    enriched basis; then the shifted standard problem is solved.
  * Lambda (Alg. 2 step 2): the k Ritz pairs with smallest |theta| (theta = lambda -
    sigma); ties by ascending theta then index.  The first n_wanted are the
    answer, the rest guard vectors.
  * Source problem (Eq. pb-m-s): per vector i, (A - s_i M) x_i = b_i starting from
    the Ritz vector u_i.  form="shifted": s_i = sigma, b_i = theta_i M u_i (the
    paper's right-hand side); form="homogeneous": s_i = lambda_i, b_i = 0.  Both
    have the same residual at x = u_i.
  * "from level k back to level 1" (Alg. 3 step 3): after the fine sweeps, the
    residual is restricted level by level; each coarser level smooths its
    correction from zero on its Galerkin operator, passes its residual down, and
    the corrections are prolonged back and added.  Levels whose shifted diagonal is
    not safely positive are skipped (with all coarser ones).
  * shift: fixed by default (the Remark on the choice of shifts allows it), or, with
    adaptive_shift, updated before the eigensolve of every cycle after the first
    (Alg. 3 step 4; Sec. 5.3): the previous shift plus the mean of the shifted
    Rayleigh quotients of the source solutions in X, i.e. mu = mean_i x_i^T A x_i /
    x_i^T M x_i over the k columns of X; the first cycle uses the given shift.  Intermediate levels run a fixed number of cycles; the finest level
    cycles until every wanted pair has relative residual
    ||A u - lambda M u||_2 / (||A||_1 ||u||_2) <= tol.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem, mesh, multilevel

SVQB_TAU = 1e-12
DIAG_MARGIN = 0.25


@dataclass
class Options:
    smoother: str = "jacobi"        # "jacobi" | "mcgs" | "mcsgs" | "kaczmarz"
    nu: int = 2
    omega: float = 2.0 / 3.0
    form: str = "shifted"           # "shifted" (Eq. pb-m-s) | "homogeneous"
    vcycle_depth: int = 99          # coarse levels visited by the down-leg
    cycles_intermediate: int = 6     # cycle cap on levels 2..L-1
    tol_intermediate: float = -1.0   # early stop on levels 2..L-1 (negative: none)
    max_cycles: int = 200
    adaptive_shift: bool = False     # Alg. 3 step 4: shift from the Rayleigh quotients of X
    # Which Ritz pairs are kept (Sec. 5.2): "nearest" -- the k smallest |theta| in every
    # Rayleigh-Ritz (the enrichment follows the spectrum near the shift: index-updating);
    # "index" -- positions index_first .. index_first + k - 1 of the ascending Ritz
    # values in every Rayleigh-Ritz (index-fixed), the wanted ones being those of the
    # window nearest the shift.
    selection: str = "nearest"
    index_first: int = 0
    # Start block (Alg. 4 step 1): "given" -- X0 on level 2 as passed; "coarse" -- the
    # eigenvectors of the level-1 problem (the Galerkin pair of level 2 on level 1)
    # selected as above (an index window past the 42 coarse values moved down to the
    # top k of them), prolongated to level 2 (k <= 42).
    init: str = "given"


@dataclass
class Hierarchy:
    """Levels 1..L (index 0 unused): meshes, operators, prolongations, colourings."""
    verts: list = field(default_factory=list)
    tris: list = field(default_factory=list)
    A: list = field(default_factory=list)
    M: list = field(default_factory=list)
    P: list = field(default_factory=list)       # P[l]: level l-1 -> l
    colour: list = field(default_factory=list)
    colour2: list = field(default_factory=list)   # distance-2 colourings (Kaczmarz)
    GA: dict = field(default_factory=dict)      # GA[f][j]: Galerkin of A_f on level j
    GM: dict = field(default_factory=dict)

    @property
    def levels(self):
        return len(self.A) - 1


def build_hierarchy(coarse_verts, coarse_tris, levels: int, amplitude=0.0,
                    coefs=None, colour=True, colour2=False) -> Hierarchy:
    """Refine, assemble, and build prolongations and Galerkin sets (setup, a0)."""
    meshes = mesh.surface_hierarchy(coarse_verts, coarse_tris, levels, amplitude, coefs)
    H = Hierarchy()
    H.verts.append(None); H.tris.append(None); H.A.append(None); H.M.append(None)
    H.P.append(None); H.colour.append(None); H.colour2.append(None)
    for l in range(1, levels + 1):
        v, t, par = meshes[l]
        A, M = fem.assemble(v, t)
        H.verts.append(v); H.tris.append(t); H.A.append(A); H.M.append(M)
        H.P.append(None if l == 1 else multilevel.prolongation(par, meshes[l - 1][0].shape[0]))
        H.colour.append(multilevel.greedy_colouring(A.indptr, A.indices) if colour else None)
        H.colour2.append(multilevel.greedy_colouring(*multilevel.distance2_pattern(A.indptr, A.indices))
                         if colour2 else None)
    for f in range(2, levels + 1):
        ga = {f: H.A[f]}
        gm = {f: H.M[f]}
        for j in range(f, 1, -1):
            ga[j - 1] = multilevel.galerkin(H.P[j], ga[j])
            gm[j - 1] = multilevel.galerkin(H.P[j], gm[j])
        H.GA[f] = ga
        H.GM[f] = gm
    return H


def restrict_chain(H: Hierarchy, Y, f: int, to: int = 1):
    for j in range(f, to, -1):
        Y = H.P[j].T @ Y
    return Y


def prolong_chain(H: Hierarchy, Z, start: int, f: int):
    for j in range(start + 1, f + 1):
        Z = H.P[j] @ Z
    return Z


def select_order(theta: np.ndarray) -> np.ndarray:
    """Indices sorted by (|theta|, theta, index)."""
    idx = np.arange(theta.shape[0])
    return np.lexsort((idx, theta, np.abs(theta)))


def select_pairs(theta: np.ndarray, k: int, selection: str = "nearest", first: int = 0) -> np.ndarray:
    """Indices of the k kept pairs, ordered by (|theta|, theta, index).

    "nearest": the k smallest |theta|.  "index": positions first .. first + k - 1 of
    the values in ascending order (ties by index), then put in the same order; a window
    that runs past the top of the r values present is moved down to positions
    r - k .. r - 1 (a rank-deficient enriched space, or the coarse problem alone).
    """
    if selection == "nearest":
        return select_order(theta)[:k]
    if selection != "index":
        raise ValueError(selection)
    asc = np.lexsort((np.arange(theta.shape[0]), theta))
    first = min(max(first, 0), theta.shape[0] - k)
    win = asc[first:first + k]
    return win[select_order(theta[win])]


def svqb_eig(Ahat, Mhat, sigma: float, k: int, tau: float = SVQB_TAU, selection: str = "nearest",
             first: int = 0):
    """k pairs of (Ahat - sigma Mhat) y = theta Mhat y via SVQB: the smallest |theta|,
    or a window of positions of the ascending spectrum (select_pairs).

    Returns (theta [k], Y [n,k]) with Y^T Mhat Y = I.
    """
    Ahat = 0.5 * (Ahat + Ahat.T)
    Mhat = 0.5 * (Mhat + Mhat.T)
    d = 1.0 / np.sqrt(np.diag(Mhat))
    Ms = Mhat * d[:, None] * d[None, :]
    mu, V = sla.eigh(Ms)
    keep = mu > tau * mu.max()
    if int(keep.sum()) < k:
        raise np.linalg.LinAlgError("enriched space rank %d < k=%d" % (keep.sum(), k))
    B = (d[:, None] * V[:, keep]) / np.sqrt(mu[keep])[None, :]
    At = B.T @ (Ahat - sigma * Mhat) @ B
    At = 0.5 * (At + At.T)
    theta, W = sla.eigh(At)
    sel = select_pairs(theta, k, selection, first)
    return theta[sel], B @ W[:, sel]


def enriched_matrices(H: Hierarchy, f: int, X, AX, MX):
    """Block matrices of the enriched space V_{h1} + span(X) on level f (Sec. 4.1)."""
    CA = restrict_chain(H, AX, f)
    CM = restrict_chain(H, MX, f)
    GA = X.T @ AX
    GM = X.T @ MX
    AQ = H.GA[f][1].toarray()
    MQ = H.GM[f][1].toarray()
    Ahat = np.block([[AQ, CA], [CA.T, GA]])
    Mhat = np.block([[MQ, CM], [CM.T, GM]])
    return Ahat, Mhat


def norm1(A: sp.spmatrix) -> float:
    return float(abs(A).sum(axis=0).max())


def residuals(A, M, U, lam, anorm=None):
    anorm = norm1(A) if anorm is None else anorm
    R = A @ U - (M @ U) * lam[None, :]
    return np.linalg.norm(R, axis=0) / (anorm * np.linalg.norm(U, axis=0))


def smooth(A, M, X, B, s, colour, opt: Options, colour2=None):
    if opt.smoother == "kaczmarz":
        return multilevel.kaczmarz(A, M, X, B, s, colour2, opt.nu, opt.omega)
    if opt.smoother == "jacobi":
        return multilevel.jacobi(A, M, X, B, s, opt.omega, opt.nu)
    if opt.smoother in ("mcgs", "mcsgs"):
        return multilevel.mc_gauss_seidel(A, M, X, B, s, colour, opt.nu,
                                          symmetric=(opt.smoother == "mcsgs"))
    raise ValueError(opt.smoother)


def vleg_levels(H: Hierarchy, f: int, s, opt: Options):
    """Coarse levels visited by the down-leg: f-1, f-2, ... while D stays positive."""
    smax = float(np.max(s))
    out = []
    for j in range(f - 1, 0, -1):
        if len(out) >= opt.vcycle_depth:
            break
        da = H.GA[f][j].diagonal()
        dm = H.GM[f][j].diagonal()
        if not np.all(da - smax * dm > DIAG_MARGIN * da):
            break
        out.append(j)
    return out


def source_smoothing(H: Hierarchy, f: int, U, MU, theta, lam, sigma, opt: Options):
    """Approximate the source problems from the Ritz vectors (Alg. 3 step 3)."""
    if opt.form == "shifted":
        s = np.full(lam.shape, sigma)
        B = MU * theta[None, :]
    else:
        s = lam.copy()
        B = np.zeros_like(U)
    A, M = H.A[f], H.M[f]
    X = smooth(A, M, U, B, s, H.colour[f], opt, H.colour2[f])
    levels = vleg_levels(H, f, s, opt)
    if not levels:
        return X
    r = {f: B - multilevel.shifted_apply(A, M, X, s)}
    e = {}
    for idx, j in enumerate(levels):
        Ga, Gm = H.GA[f][j], H.GM[f][j]
        rj = H.P[j + 1].T @ r[j + 1]
        ej = smooth(Ga, Gm, np.zeros_like(rj), rj, s, H.colour[j], opt, H.colour2[j])
        e[j] = ej
        if idx + 1 < len(levels):
            r[j] = rj - multilevel.shifted_apply(Ga, Gm, ej, s)
    for j in reversed(levels[1:]):       # coarsest first: add into the next finer
        e[j + 1] = e[j + 1] + H.P[j + 1] @ e[j]
    return X + H.P[f] @ e[levels[0]]


@dataclass
class CycleResult:
    lam: np.ndarray
    U: np.ndarray
    resid: np.ndarray
    X_next: np.ndarray | None
    sigma: float = 0.0


def mean_rayleigh_quotient(X, AX, MX) -> float:
    """Mean over the columns of X of x^T A x / x^T M x (Sec. 5.3, the shift update)."""
    return float(np.mean(np.sum(X * AX, axis=0) / np.sum(X * MX, axis=0)))


def cycle(H: Hierarchy, f: int, X, sigma: float, k: int, n_wanted: int, tol: float,
          opt: Options, anorm=None, smooth_if_converged=False, first=True):
    """One BMG cycle on level f: enriched RR, residual check, source smoothing.
    With opt.adaptive_shift every cycle but the solve's first takes as its shift the
    mean Rayleigh quotient of X, the source solutions of the previous cycle
    (returned as CycleResult.sigma); otherwise the shift is `sigma`."""
    A, M = H.A[f], H.M[f]
    AX, MX = A @ X, M @ X
    if opt.adaptive_shift and not first:
        sigma = mean_rayleigh_quotient(X, AX, MX)
    Ahat, Mhat = enriched_matrices(H, f, X, AX, MX)
    theta, Y = svqb_eig(Ahat, Mhat, sigma, k, selection=opt.selection, first=opt.index_first)
    lam = theta + sigma
    n1 = H.A[1].shape[0]
    U = prolong_chain(H, Y[:n1], 1, f) + X @ Y[n1:]
    AU, MU = A @ U, M @ U
    anorm = norm1(A) if anorm is None else anorm
    R = AU - MU * lam[None, :]
    resid = np.linalg.norm(R, axis=0) / (anorm * np.linalg.norm(U, axis=0))
    conv = bool(np.all(resid[:n_wanted] <= tol))
    Xn = None
    if not conv or smooth_if_converged:
        Xn = source_smoothing(H, f, U, MU, theta, lam, sigma, opt)
    return CycleResult(lam, U, resid, Xn, sigma), conv


def coarse_start(H: Hierarchy, sigma: float, k: int, opt: Options):
    """Alg. 4 step 1: the level-1 eigenpairs of (A - sigma M) y = theta M y for the
    Galerkin pair of level 2 (P_2^T A_2 P_2, P_2^T M_2 P_2), k of them kept as in every
    Rayleigh-Ritz (select_pairs), prolongated to level 2."""
    A1 = H.GA[2][1].toarray()
    M1 = H.GM[2][1].toarray()
    if k > A1.shape[0]:
        raise ValueError("coarse start: k = %d > %d coarse vertices" % (k, A1.shape[0]))
    theta, V = sla.eigh(0.5 * (A1 + A1.T) - sigma * 0.5 * (M1 + M1.T), 0.5 * (M1 + M1.T))
    sel = select_pairs(theta, k, opt.selection, opt.index_first)
    return H.P[2] @ V[:, sel]


@dataclass
class SolveResult:
    lam: np.ndarray
    U: np.ndarray
    resid: np.ndarray
    cycles: list
    converged: bool
    history: list
    level_lams: list        # Ritz values at the end of each level 2..L
    shifts: list = field(default_factory=list)   # shift of every cycle


def bfmg(H: Hierarchy, X0, k: int, n_wanted: int, sigma: float, tol: float,
         opt: Options = Options(), verbose=False) -> SolveResult:
    """Alg. 4: cycles on levels 2..L, prolongating the Ritz vectors between levels."""
    L = H.levels
    if opt.init == "coarse":
        X0 = coarse_start(H, sigma, k, opt)
    X = np.array(X0, dtype=np.float64, copy=True)
    cycles, history, level_lams, shifts = [], [], [], []
    res = None
    for f in range(2, L + 1):
        if f > 2:
            X = H.P[f] @ res.U
        anorm = norm1(H.A[f])
        budget = opt.max_cycles if f == L else opt.cycles_intermediate
        ftol = tol if f == L else opt.tol_intermediate
        c = 0
        while True:
            res, conv = cycle(H, f, X, sigma, k, n_wanted, ftol, opt, anorm, first=not shifts)
            shifts.append(res.sigma)
            c += 1
            history.append((f, c, float(res.resid[:n_wanted].max())))
            if verbose:
                print(f, c, res.resid[:n_wanted].max(), res.lam[:4])
            if conv or c >= budget:
                break
            X = res.X_next
        cycles.append(c)
        level_lams.append(res.lam.copy())
    conv = bool(np.all(res.resid[:n_wanted] <= tol))
    return SolveResult(res.lam, res.U, res.resid, cycles, conv, history, level_lams, shifts)
