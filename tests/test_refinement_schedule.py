"""The refinement schedule of the enriched eigensolve, emulated in NumPy.

The CUDA eigensolve starts from FP32-accurate eigenvectors of the reduced matrix T
and refines them in FP64 by the iterative scheme of Ogita & Aishima (2018) in four
steps: two with the pair-separation floor at 1e-3 of max|lambda| (the FP32 start's
resolution), a cluster step that diagonalises the groups of nearly equal values, and
one with the floor at 1e-7.  This test replays that schedule step for step on the
enriched problems that the oracle's BFMG meets on the 642- and 2562-vertex spheres
(FP32 eigenvectors from LAPACK standing in for the FP32 start) and checks that it
reaches FP64 accuracy: the final error estimate ||S - diag||/max|lambda| + ||I - G||
and the eigenvalues against LAPACK in FP64.  The CUDA path itself is checked against
the oracle by the GPU tests."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bmg as obmg
from paper_1511_07042_gb300 import inputs

MODES = [0, 0, 1, 0]
FLOORS = [1e-3, 1e-3, 1e-3, 1e-7]
GUARD = 0.05


def enriched_problems(R, k, nw):
    cases, orig = [], obmg.svqb_eig

    def spy(Ah, Mh, sigma, kk, *a, **kw):
        cases.append((Ah.copy(), Mh.copy(), sigma))
        return orig(Ah, Mh, sigma, kk, *a, **kw)
    obmg.svqb_eig = spy
    try:
        H = obmg.build_hierarchy(*inputs.icosahedron(), R)
        obmg.bfmg(H, inputs.gaussian_block(inputs.n_vertices(2), k, 1001), k, nw, 0.0, 1e-10,
                  obmg.Options(smoother="mcsgs", nu=1, omega=1.0))
    finally:
        obmg.svqb_eig = orig
    return cases


def reduced_matrix(Ah, Mh, sigma):
    Ms = 0.5 * (Mh + Mh.T)
    d = 1.0 / np.sqrt(np.diag(Ms))
    mu, V = sla.eigh(Ms * np.outer(d, d))
    B = V[:, mu > 1e-12 * mu.max()] / np.sqrt(mu[mu > 1e-12 * mu.max()])
    T = B.T @ ((0.5 * (Ah + Ah.T) - sigma * Ms) * np.outer(d, d)) @ B
    return 0.5 * (T + T.T)


def cluster_vectors(A):
    """Eigenvectors of the cluster block as the cluster step forms them: FP32 on the
    scaled deviation from the mean, one Newton-Schulz step, FP64 polish."""
    m = A.shape[0]
    D = A - np.trace(A) / m * np.eye(m)
    V0 = np.linalg.eigh((D / np.abs(D).max()).astype(np.float32))[1].astype(np.float64)
    V1 = V0 @ (1.5 * np.eye(m) - 0.5 * (V0.T @ V0))
    Ap = V1.T @ A @ V1
    return V1 @ np.linalg.eigh(0.5 * (Ap + Ap.T))[1]


def refine(T, W):
    r = T.shape[0]

    def products(W):
        G = W.T @ W
        S = W.T @ T @ W
        G, S = 0.5 * (G + G.T), 0.5 * (S + S.T)
        lam = np.diag(S) / (2.0 - np.diag(G))
        return G, S, lam, np.sum((S - np.diag(lam)) ** 2), np.sum((np.eye(r) - G) ** 2), np.abs(lam).max()

    G, S, lam, a0, a1, amax = products(W)
    for mode, floor in zip(MODES, FLOORS):
        thr = max(2.0 * (np.sqrt(a0) + amax * np.sqrt(a1)), floor * amax)
        R = np.eye(r) - G
        if mode == 0:
            E = 0.5 * R
            D = lam[None, :] - lam[:, None]
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (S + lam[None, :] * R) / D
            sel = (np.abs(D) > thr) & (np.abs(t) < GUARD)
            np.fill_diagonal(sel, False)
            E[sel] = t[sel]
        else:
            E = np.diag(0.5 * np.diag(R))
            order = np.argsort(lam, kind="stable")
            sl = lam[order]
            cuts = [0] + [i for i in range(1, r) if not (sl[i] - sl[i - 1] <= thr)] + [r]
            for c in range(len(cuts) - 1):
                idx = order[cuts[c]:cuts[c + 1]]
                if len(idx) < 2:
                    continue
                K = 1.5 * np.eye(len(idx)) - 0.5 * G[np.ix_(idx, idx)]
                A = K @ S[np.ix_(idx, idx)] @ K
                E[np.ix_(idx, idx)] = K @ cluster_vectors(0.5 * (A + A.T)) - np.eye(len(idx))
        W = W + W @ E
        G, S, lam, a0, a1, amax = products(W)
    return W, lam, np.sqrt(a0) / amax + np.sqrt(a1)


@pytest.mark.parametrize("R,k,nw", [(3, 20, 16), (4, 32, 24)])
def test_four_step_schedule_reaches_fp64_accuracy(R, k, nw):
    cases = enriched_problems(R, k, nw)
    assert len(cases) >= 10
    for Ah, Mh, sigma in cases[::3]:
        T = reduced_matrix(Ah, Mh, sigma)
        W0 = np.linalg.eigh(T.astype(np.float32))[1].astype(np.float64)
        W, lam, quality = refine(T, W0)
        assert quality <= 1e-12
        ref = np.linalg.eigvalsh(T)
        assert np.max(np.abs(np.sort(lam) - ref)) <= 1e-13 * max(np.abs(ref).max(), 1.0)
