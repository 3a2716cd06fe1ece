"""Plain FP64 CPU oracle of the Wilson-clover multigrid hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
execute anything in this package.  The product path (the C-ABI library under
``paper_1904_08678_gb300/``) shares no code with it and never calls it.

Paper: Richtmann, Boyle, Wettig, "Multigrid for Wilson Clover Fermions in Grid",
LATTICE2018 (arXiv:1904.08678).  The paper names the operators (Sec. 1, Sec. 2.1,
Sec. 2.2) but does not write the Dirac operator, the clover term, the gamma basis,
the setup or the solver parameters down; the readings used here are listed in the
module docstrings and pinned by tests/test_oracle_*.py against closed forms,
invariants and brute force:

  gamma.py        chiral Euclidean gamma basis          pinned: Clifford algebra, gamma5 diagonal
  wilson.py       Wilson-clover D, clover term          pinned: plane waves, abelian flux, gamma5-herm., gauge cov.
  aggregation.py  block orthonormalisation, P, P^dag    pinned: QR uniqueness, P^dag P = 1, adjointness, gamma5 P = P sigma3
  coarse.py       Galerkin coarse operator (9 blocks)   pinned: dense P^dag D P, sigma3-hermiticity, gauge invariance
  solvers.py      MR, GMRES, FGMRES                     pinned: MR step minimality, dense solve, lucky breakdown
  mg.py           MG cycle, initial + iterative setup   pinned: block 1^4 exact preconditioner; setup sweeps = normalised
                                                         inverse iteration (free-field spectrum) with an exact
                                                         smoother / cycle; Rayleigh quotient falls with sweeps
  sap.py          SAP smoother, even-odd block solves   pinned: red-black exact solves, dense per-block solves
  ptc.py          parallel-transport conv. network      pinned: gauge/translation equivariance, adjoint identity,
                                                         finite-difference gradients

Every array is complex128.  Internal field shape is (T, Z, Y, X, ncomp), i.e. the
external lexicographic site order s = x + Lx*(y + Ly*(z + Lz*t)) reshaped; fine
fields have ncomp = 12 = 4 spins x 3 colours (spin-major).
"""
