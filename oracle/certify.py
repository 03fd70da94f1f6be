"""Independent checks of computed eigenpairs: dense solves, residual bounds, inertia.

Oracle (test infrastructure only).

These use library routines (LAPACK through scipy.linalg.eigh, SuperLU through
scipy.sparse.linalg.splu) and textbook facts about symmetric-definite pencils, so
they pin the BMG iteration to something other than itself:
  * dense eigh(A, M): the exact discrete spectrum for small meshes;
  * residual bound: for the pencil (A, M) with M SPD and any (lam, u), some
    eigenvalue lies within ||A u - lam M u||_{M^-1} / ||u||_M of lam;
  * Sylvester inertia: the number of eigenvalues below s equals the number of
    negative pivots of an LDL^T factorisation of A - s M.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla


def dense_pencil_eigs(A, M):
    """All eigenpairs of the pencil (A, M) by LAPACK; eigenvectors M-orthonormal."""
    return sla.eigh(A.toarray(), M.toarray())


def nearest(w, V, sigma: float, count: int):
    """The `count` eigenpairs nearest sigma (ties by value then index)."""
    idx = np.lexsort((np.arange(w.shape[0]), w, np.abs(w - sigma)))[:count]
    idx = np.sort(idx)
    return w[idx], V[:, idx]


def residual_bound(A, M, lam, U):
    """||A u - lam M u||_{M^{-1}} / ||u||_M per column (sparse LU of M)."""
    R = A @ U - (M @ U) * lam[None, :]
    lu = spla.splu(sp.csc_matrix(M))
    MinvR = lu.solve(R)
    num = np.sqrt(np.maximum(np.sum(R * MinvR, axis=0), 0.0))
    den = np.sqrt(np.sum(U * (M @ U), axis=0))
    return num / den


def inertia_below(A, M, s: float) -> int:
    """Number of eigenvalues of (A, M) below s, by Sylvester's law of inertia.

    Symmetric RCM reordering, then an LU factorisation without row exchanges
    (natural column order, no pivoting threshold): U's diagonal holds the pivots of
    the LDL^T factorisation of the permuted A - s M.
    """
    K = sp.csr_matrix(A - s * M)
    perm = csg.reverse_cuthill_mckee(K, symmetric_mode=True)
    Kp = sp.csc_matrix(K[perm][:, perm])
    lu = spla.splu(Kp, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    if not (np.all(lu.perm_r == np.arange(K.shape[0]))):
        raise RuntimeError("row exchanges happened; inertia not available")
    return int(np.sum(lu.U.diagonal() < 0))


def cluster_groups(w, rel_gap: float = 1e-6):
    """Group sorted reference eigenvalues into clusters separated by a relative gap."""
    groups, cur = [], [0]
    for i in range(1, len(w)):
        if abs(w[i] - w[i - 1]) <= rel_gap * max(1.0, abs(w[i])):
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return groups


def max_principal_angle(M, U, V):
    """Largest M-principal angle between span(U) and span(V) (radians)."""
    def morth(Z):
        G = Z.T @ (M @ Z)
        L = np.linalg.cholesky(0.5 * (G + G.T))
        return np.linalg.solve(L, Z.T).T
    Qu, Qv = morth(U), morth(V)
    # sine of the largest angle = M-norm of the part of span(U) outside span(V)
    R = Qu - Qv @ (Qv.T @ (M @ Qu))
    G = R.T @ (M @ R)
    smax = np.sqrt(max(float(np.linalg.eigvalsh(0.5 * (G + G.T)).max()), 0.0))
    return float(np.arcsin(min(smax, 1.0)))


def compare_to_reference(M, lam, U, w_ref, V_ref, rel_gap=1e-6):
    """Eigenvalue relative errors and per-cluster M-subspace angles.

    lam, U: computed pairs (any order); w_ref, V_ref: reference pairs, ascending.
    Eigenvalue error uses the denominator max(|ref|, 1).  Clusters are formed on
    the reference values; a computed cluster is the same number of computed pairs
    closest to the reference cluster.
    """
    order = np.argsort(lam)
    lam, U = lam[order], U[:, order]
    err = np.abs(lam - w_ref) / np.maximum(np.abs(w_ref), 1.0)
    angles = []
    for g in cluster_groups(w_ref, rel_gap):
        angles.append(max_principal_angle(M, U[:, g], V_ref[:, g]))
    return err, np.array(angles)
