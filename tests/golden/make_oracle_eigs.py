"""Writes reference eigenvalues of a named workload from the FP64 oracle.

Usage:  python tests/golden/make_oracle_eigs.py sphere655362_k128_mixed [tol]

Runs the oracle's BFMG (Alg. 4 with the cycle of Alg. 3, everything in float64) on
the workload's icosphere hierarchy with the workload's seeded X0, to the given
relative-residual tolerance (default 1e-10, tighter than the workload's own), and
writes tests/golden/<workload>_oracle_eigs.txt: one line per wanted pair with its
index, eigenvalue and relative residual.  Only the oracle and the input generators
are called; the CUDA path is not involved.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import bmg as obmg  # noqa: E402
from paper_1511_07042_gb300 import inputs  # noqa: E402


def main():
    name = sys.argv[1]
    tol = float(sys.argv[2]) if len(sys.argv) > 2 else 1e-10
    wl = inputs.WORKLOADS[name]
    R, k, nw = wl["refinements"], wl["k"], wl["n_wanted"]
    v, t = inputs.icosahedron()
    coefs = inputs.sh_coefficients(wl["coef_seed"]) if wl["coef_seed"] is not None else None
    t0 = time.time()
    H = obmg.build_hierarchy(v, t, R, amplitude=wl["amplitude"], coefs=coefs,
                             colour=wl["smoother"] != "jacobi")
    X0 = inputs.gaussian_block(inputs.n_vertices(2), k, wl["seed"])
    opt = obmg.Options(smoother=wl["smoother"], nu=wl["nu"], omega=wl["omega"])
    res = obmg.bfmg(H, X0, k, nw, wl["sigma"], tol, opt, verbose=True)
    dt = time.time() - t0
    out = os.path.join(HERE, "%s_oracle_eigs.txt" % name)
    with open(out, "w") as fh:
        fh.write("# Reference eigenvalues of workload %s (icosphere refined %d times, %d vertices)\n"
                 % (name, R, inputs.n_vertices(R)))
        fh.write("# written by tests/golden/make_oracle_eigs.py: FP64 oracle BFMG (Alg. 4), k=%d,\n" % k)
        fh.write("# sigma=%g, %s nu=%d, X0 seed %d, tol %g; cycles per level %s; converged %s;\n"
                 % (wl["sigma"], wl["smoother"], wl["nu"], wl["seed"], tol, res.cycles, res.converged))
        fh.write("# %.0f s on %d host cores.\n" % (dt, os.cpu_count()))
        fh.write("# columns: index  eigenvalue  relative_residual\n")
        for i in range(nw):
            fh.write("%d %.17g %.3e\n" % (i, res.lam[i], res.resid[i]))
    print("wrote", out, "in %.0f s" % dt)


if __name__ == "__main__":
    main()
