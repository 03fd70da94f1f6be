"""Batched form: many (surface, shift) jobs solved together.

Each job's result must equal what a single bmg_solve gives for it (same kernels and
reduction orders, so the eigenvalues agree bit for bit), match dense LAPACK on
small perturbed spheres with interior shifts, and, on the workload of 32 seeded
perturbed spheres of uneven size with two shifts each, match the FP64 oracle's BFMG
on sampled jobs with residuals recomputed on the host."""
import numpy as np
import pytest

from oracle import bmg as obmg, certify
from paper_1511_07042_gb300 import inputs

pytestmark = pytest.mark.gpu


def make(bmg, desc):
    v, t = inputs.icosahedron()
    p = bmg.Problem(v, t, desc["refinements"], desc["amplitude"], desc["coefs"])
    p.hierarchy(desc["refinements"])
    return p


def small_instances(n):
    """Perturbed 642-vertex spheres with shifts {0, U(10, 25)}: interior shifts within
    the reach of the 42-vertex coarse space, where the method converges."""
    rng = np.random.default_rng(77)
    return [dict(refinements=3, amplitude=float(rng.uniform(0.0, 0.15)), coefs=rng.standard_normal(25),
                 sigmas=(0.0, float(rng.uniform(10.0, 25.0))), x0_seed=int(rng.integers(1, 10 ** 6)))
            for _ in range(n)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_equals_single_solves(gpu_bmg, precision):
    descs = small_instances(3)
    probs = [make(gpu_bmg, d) for d in descs]
    jobs = [(probs[i], s, inputs.gaussian_block(inputs.n_vertices(2), 24, descs[i]["x0_seed"] + j))
            for i, d in enumerate(descs) for j, s in enumerate(d["sigmas"])]
    opt = gpu_bmg.options(precision=precision, max_cycles=60)
    ev, _, rs, infos, code = gpu_bmg.solve_batched([j[0] for j in jobs], [j[1] for j in jobs],
                                                   [j[2] for j in jobs], 24, 12, 1e-9, opt, concurrency=4)
    assert code in (0, 5)
    for q, (p, s, X0) in enumerate(jobs):
        e1, _, r1, info1 = p.solve(X0, 24, 12, s, 1e-9, opt, evecs=False)
        assert np.array_equal(e1, ev[q]) and np.array_equal(r1, rs[q])
        assert info1.total_cycles == infos[q].total_cycles and info1.converged == infos[q].converged


def test_batched_matches_dense(gpu_bmg):
    descs = small_instances(4)
    probs = [make(gpu_bmg, d) for d in descs]
    jobs = [(i, s) for i, d in enumerate(descs) for s in d["sigmas"]]
    X0s = [inputs.gaussian_block(inputs.n_vertices(2), 24, 5 + q) for q in range(len(jobs))]
    ev, U, rs, infos, code = gpu_bmg.solve_batched([probs[i] for i, _ in jobs], [s for _, s in jobs], X0s, 24, 12,
                                                   1e-10, gpu_bmg.options(precision="fp32"), evecs=True)
    assert code == 0
    for q, (i, s) in enumerate(jobs):
        d = descs[i]
        H = obmg.build_hierarchy(*inputs.icosahedron(), 3, d["amplitude"], d["coefs"], colour=False)
        A, M = H.A[3], H.M[3]
        w, V = certify.dense_pencil_eigs(A, M)
        wr, Vr = certify.nearest(w, V, s, 12)
        err, ang = certify.compare_to_reference(M, ev[q], U[q], wr, Vr)
        assert err.max() <= 1e-10 and ang.max() <= 1e-8, (q, err.max(), ang.max())


def test_batched_workload_32_surfaces_two_shifts(gpu_bmg):
    """32 perturbed spheres (refinements 4..7), shifts {0, U(20, 200)}, k=32, 24
    wanted, tol 1e-8, precision form.  Every sigma=0 job converges, and sampled ones
    match the oracle's FP64 BFMG with residuals recomputed on the host.  Interior
    shifts this far above the reach of the 42-vertex coarse space do not converge
    with the method (the oracle stalls in the same way); those jobs must still
    return finite Ritz pairs with the cycle-cap status."""
    descs = inputs.batch_instances()
    probs = [make(gpu_bmg, d) for d in descs]
    jobs = [(i, s) for i, d in enumerate(descs) for s in d["sigmas"]]
    X0s = [inputs.gaussian_block(inputs.n_vertices(2), 32, descs[i]["x0_seed"] + (s != 0.0)) for i, s in jobs]
    opt = gpu_bmg.options(precision="fp32", max_cycles=100)
    ev, U, rs, infos, code = gpu_bmg.solve_batched([probs[i] for i, _ in jobs], [s for _, s in jobs], X0s, 32, 24,
                                                   1e-8, opt, evecs=True)
    assert code in (0, 5)
    for q, (i, s) in enumerate(jobs):
        assert np.all(np.isfinite(ev[q])) and np.all(np.isfinite(rs[q]))
        if s == 0.0:
            assert infos[q].converged == 1, q
    picks = [q for q, (i, s) in enumerate(jobs) if s == 0.0 and descs[i]["refinements"] <= 5][:3]
    assert picks
    for q in picks:
        i, s = jobs[q]
        d = descs[i]
        R = d["refinements"]
        H = obmg.build_hierarchy(*inputs.icosahedron(), R, d["amplitude"], d["coefs"], colour=False)
        A, M = H.A[R], H.M[R]
        assert np.all(obmg.residuals(A, M, U[q], ev[q]) <= 1e-8)
        ref = obmg.bfmg(H, X0s[q], 32, 24, s, 1e-10, obmg.Options())
        got, want = np.sort(ev[q]), np.sort(ref.lam[:24])
        assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1.0)) <= 1e-9, q
