"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds only input generation: the coarse input mesh (the regular
icosahedron inscribed in the unit sphere), seeded Gaussian test-vector blocks,
seeded spherical-harmonic coefficients of a perturbed radius, and the descriptors of
the batched workload. It contains none of the method's arithmetic (no refinement,
no assembly, no smoothing, no eigensolve). Both sides receive what it returns.

The paper's experiments start from a 54-node Distmesh sphere (Sec. 5); that mesh is
not available, so the icosahedron stands in as the coarse input mesh that the
algorithm takes (Sec. 4.1: a coarse mesh, a shift and a tolerance are the inputs).
"""
from __future__ import annotations

import numpy as np

# Workload descriptors: refinement count of the finest level, block size k, wanted
# pairs, shift, tolerance, smoother, seeds.  Level 1 (refinement 1, 42 vertices) is
# the coarsest level of every hierarchy.
WORKLOADS = {
    "sphere642_k20": dict(refinements=3, k=20, n_wanted=16, sigma=0.0, tol=1e-10,
                          smoother="jacobi", nu=2, omega=2.0 / 3.0, seed=1001,
                          amplitude=0.0, coef_seed=None),
    "sphere40962_k64": dict(refinements=6, k=64, n_wanted=49, sigma=0.0, tol=1e-10,
                            smoother="mcsgs", nu=1, omega=1.0, seed=1002,
                            amplitude=0.0, coef_seed=None),
    "bumpy163842_k48_s110": dict(refinements=7, k=48, n_wanted=21, sigma=110.0,
                                 tol=1e-10, smoother="jacobi", nu=2, omega=2.0 / 3.0,
                                 seed=1013, amplitude=0.1, coef_seed=1003),
    "sphere655362_k128_mixed": dict(refinements=8, k=128, n_wanted=100, sigma=0.0,
                                    tol=1e-8, smoother="jacobi", nu=2,
                                    omega=2.0 / 3.0, seed=1004, amplitude=0.0,
                                    coef_seed=None),
}


def n_vertices(refinements: int) -> int:
    """Vertex count of the icosahedron refined r times: 10*4^r + 2."""
    return 10 * 4 ** refinements + 2


def icosahedron():
    """The regular icosahedron on the unit sphere, outward-oriented faces.

    Returns (verts float64 [12,3], tris int32 [20,3]).  Vertices are the cyclic
    permutations of (0, +-1, +-phi) scaled to unit length; the face list is fixed.
    """
    phi = (1.0 + np.sqrt(5.0)) / 2.0
    raw = np.array([
        [-1.0, phi, 0.0], [1.0, phi, 0.0], [-1.0, -phi, 0.0], [1.0, -phi, 0.0],
        [0.0, -1.0, phi], [0.0, 1.0, phi], [0.0, -1.0, -phi], [0.0, 1.0, -phi],
        [phi, 0.0, -1.0], [phi, 0.0, 1.0], [-phi, 0.0, -1.0], [-phi, 0.0, 1.0],
    ], dtype=np.float64)
    nrm = np.sqrt(raw[:, 0] * raw[:, 0] + raw[:, 1] * raw[:, 1] + raw[:, 2] * raw[:, 2])
    verts = raw / nrm[:, None]
    tris = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int32)
    return verts, tris


def gaussian_block(n: int, k: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) test-vector block, row-major [n, k] float64."""
    return np.random.default_rng(seed).standard_normal((n, k))


def sh_coefficients(seed: int) -> np.ndarray:
    """Seeded N(0,1) coefficients c_lm of the real harmonics with l <= 4.

    Ordered l = 0..4 and, within l, m = -l..l: 25 values.
    """
    return np.random.default_rng(seed).standard_normal(25)


def batch_instances(seed: int = 1005, count: int = 32):
    """Descriptors of the batched workload: perturbed spheres of uneven size.

    Each instance draws a refinement in {4,...,7}, an amplitude U(0, 0.15), 25
    harmonic coefficients and two shifts {0, U(20, 200)}.  Returns a list of dicts.
    """
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        out.append(dict(refinements=int(rng.integers(4, 8)),
                        amplitude=float(rng.uniform(0.0, 0.15)),
                        coefs=rng.standard_normal(25),
                        sigmas=(0.0, float(rng.uniform(20.0, 200.0))),
                        x0_seed=int(rng.integers(0, 2 ** 31 - 1))))
    return out
