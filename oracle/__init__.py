"""FP64 CPU oracle of the bootstrap multigrid (BMG) eigensolver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this
package: only the tests, the smoke check and the benchmark's CPU-baseline leg use
it.  It is a plain, slow, direct transcription of the method (surface P1 finite
elements on a refined icosahedral sphere, geometric prolongation, Galerkin coarse
operators, smoothers, enriched Rayleigh-Ritz, BFMG driver) written with NumPy and
SciPy in float64.  It shares no code with the CUDA library.

Modules:
  mesh        uniform refinement with projection onto the surface (Sec. 3, Eq. proj)
  fem         P1 stiffness and mass matrices (Eq. bl-dis, sp-fe)
  multilevel  prolongation P_h, restriction P_h^T, Galerkin products, colouring,
              Jacobi / multicolour Gauss-Seidel smoothers (Sec. 3; Remark on
              smoothers; Sec. 5.3)
  bmg         enriched Rayleigh-Ritz (Alg. 2 step 4, block form of Sec. 4.1), the
              BMG cycle (Alg. 3) and the BFMG driver (Alg. 4)
  certify     brute-force dense eigensolves, residual bounds and inertia counts
"""
