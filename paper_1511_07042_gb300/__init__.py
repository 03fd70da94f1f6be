"""GB300-native bootstrap multigrid (BMG) eigensolver for the P1 surface-FEM
Laplace-Beltrami pencil A x = lambda M x (Brannick & Cao, arXiv 1511.07042).

The compute path is the C-ABI library `libbmg.so` (hand-written sm_103a CUDA) built
from `csrc/`; `bmg.py` is the thin ctypes binding over it.  Importing this package
does not load the library; `paper_1511_07042_gb300.bmg` does, and fails loudly when
it is missing.
"""
