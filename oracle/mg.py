"""Multigrid cycle and setup (oracle; test infrastructure).

Sec. 2.1 describes the pieces but not the algorithmic parameters:
  * the solver class calls itself recursively over the levels;
  * the initial setup (from HDCR) iterates a smoother on random vectors to get
    near-null vectors, then builds the intergrid and coarse operators;
  * the iterative-refinement setup (from DDalphaAMG) then applies the whole MG
    preconditioner to the near-null vectors and rebuilds the operators;
  * MR is the smoother, GMRES the coarsest solver, FGMRES the outer solver;
    the benchmark comparison of Sec. 4 (Table 1) runs GMRES as the smoother.

Readings used here (each listed with the other readings of the paper):
  cycle  M_l(r):  e = P_l CoarseSolve_{l+1}(P_l^dag r);  e += S_k(D_l; r - D_l e);
         S_k is the smoother: MR_k, GMRES with k steps (zero initial guess, no
         restart, no tolerance), or SAP over the level's aggregates (sap.py; with
         sap_eo its block solves on the finest level are even-odd preconditioned), the
         same smoother in the setup sweeps;
         on an intermediate level (neither finest nor coarsest) CoarseSolve is one
         cycle of that level (V-cycle) or, with kcycle, FGMRES(kcycle_steps) to
         kcycle_tol right-preconditioned by that level's cycle (K-cycle);
         no pre-smoothing.  CoarseSolve is GMRES(m) with a relative tolerance at the
         coarsest level and one application of M_{l+1} (V-cycle) in between.
  initial setup on level l: for each sweep, for each i:
         v_i <- S_k(D_l; v_i) (zero initial guess), v_i <- v_i / ||v_i||;
         then P_l (block orthonormalisation) and D_{l+1} = P_l^dag D_l P_l; recurse
         with the level-(l+1) random vectors.
  iterative refinement: for each sweep: v_i <- M_0(v_i), v_i <- v_i/||v_i|| for all i
         (all using the current hierarchy), then rebuild P_0 and D_1; every coarser
         non-coarsest level then runs one warm-started initial sweep on its current
         vectors with its new operator and rebuilds its own P and D.
The outcome of the setup with the real smoother has no closed form.  Its sweeps are
pinned where they reduce to a textbook routine: with an exact smoother (GMRES with
as many steps as the free operator has distinct eigenvalues) the initial sweeps, and
with an exact cycle (one-site aggregates, Nvec 6, coarse solve to 1e-14) the refinement
sweeps, are normalised inverse iteration, checked against the free-field spectrum.
"""
from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

from .aggregation import Aggregation
from .coarse import coarsen
from .sap import parity, sap, self_solve
from .solvers import fgmres, gmres, mr, norm


@dataclass
class MGParams:
    blocks: Sequence[Sequence[int]]          # one block per coarsening, (bx, by, bz, bt)
    nvecs: Sequence[int]                     # Nvec per coarsening
    smoother_steps: int = 4
    init_sweeps: int = 3
    refine_sweeps: int = 0
    coarse_restart: int = 20
    coarse_tol: float = 0.05
    coarse_maxiter: int = 100
    outer_restart: int = 20
    outer_tol: float = 1e-10
    outer_maxiter: int = 1000
    smoother: str = "mr"                     # "mr", "gmres" or "sap"
    sap_cycles: int = 1                      # SAP: cycles; smoother_steps = MR steps per block solve
    sap_eo: bool = False                     # SAP: even-odd preconditioned block solves on the finest level
    coarse_eo: bool = False                  # coarsest solve on the odd-site Schur complement (even-odd)
    kcycle: bool = False                     # intermediate levels: FGMRES around the cycle
    kcycle_steps: int = 5
    kcycle_tol: float = 0.1


@dataclass
class Level:
    op: object
    dims: tuple
    vecs: list = field(default_factory=list)   # raw (normalised) near-null vectors
    agg: object = None


def coarse_eo_solve(op, dims, b, restart, tol, maxiter):
    """Even-odd (red-black) preconditioned coarsest solve (Sec. 4 lists red-black
    preconditioning among Grid's missing features; DDalphaAMG, its comparison, uses it on
    every level).  With coarse sites even / odd by the parity of x + y + z + t, the hops
    of the nine-block operator join sites of opposite parity and the self blocks A_0 form
    the diagonal: D_c = [[A_ee, A_eo], [A_oe, A_oo]] with A_ee, A_oo block diagonal.
      b^_o = b_o - A_oe A_ee^-1 b_e,
      GMRES(restart) on S = A_oo - A_oe A_ee^-1 A_eo to tol relative to ||b^_o||
        (reading: the coarse tolerance applies to the system GMRES solves),
      x_e = A_ee^-1 (b_e - A_eo x_o).
    Needs even coarse extents (an odd one would join equal parities across the
    boundary).  Odd-site vectors are full fields that vanish on even sites."""
    if any(L % 2 for L in dims):
        raise ValueError("even-odd coarsest solve needs even coarse extents")
    ev = (parity(dims) == 0)[..., None]
    od = ~ev
    b_hat = np.where(od, b - op(np.where(ev, self_solve(op, b), 0)), 0)

    def schur(v):
        Dv = op(v)
        return np.where(od, Dv - op(np.where(ev, self_solve(op, np.where(ev, Dv, 0)), 0)), 0)

    x_o, _ = gmres(schur, b_hat, restart=restart, tol=tol, maxiter=maxiter)
    x_e = np.where(ev, self_solve(op, b - op(x_o)), 0)
    return x_e + x_o


class Multigrid:
    def __init__(self, fine_op, params: MGParams, init_vecs: List[list], build=True):
        """init_vecs[l] is the list of Nvec random fields of level l (generator data)."""
        self.p = params
        self.levels: List[Level] = [Level(fine_op, tuple(fine_op.dims))]
        self.init_vecs = init_vecs
        if build:
            self.setup()

    @property
    def nlevels(self):
        return len(self.p.blocks) + 1

    # ---------------- setup ----------------
    def smooth(self, l, b):
        """S_k(D_l; b) from a zero initial guess."""
        op, k = self.levels[l].op, self.p.smoother_steps
        if self.p.smoother == "mr":
            return mr(op, b, k)
        if self.p.smoother == "gmres":
            return gmres(op, b, restart=k, tol=0.0, maxiter=k)[0]
        if self.p.smoother == "sap":
            return sap(op, self.levels[l].dims, self.p.blocks[l], b, k, self.p.sap_cycles,
                       eo=self.p.sap_eo and l == 0)
        raise ValueError(self.p.smoother)

    def _smooth_sweep(self, l):
        lev = self.levels[l]
        out = []
        for v in lev.vecs:
            x = self.smooth(l, v)
            out.append(x / norm(x))
        lev.vecs = out

    def _build(self, l):
        lev = self.levels[l]
        lev.agg = Aggregation(lev.dims, self.p.blocks[l], lev.vecs)
        Dc = coarsen(lev.op, lev.agg)
        if len(self.levels) > l + 1:
            self.levels[l + 1].op = Dc
        else:
            self.levels.append(Level(Dc, tuple(lev.agg.cdims)))

    def setup(self):
        for l in range(self.nlevels - 1):
            self.levels[l].vecs = [v.copy() for v in self.init_vecs[l]]
            for _ in range(self.p.init_sweeps):
                self._smooth_sweep(l)
            self._build(l)
        for _ in range(self.p.refine_sweeps):
            self.refine_sweep()

    def refine_sweep(self):
        lev = self.levels[0]
        new = []
        for v in lev.vecs:
            x = self.cycle(0, v)
            new.append(x / norm(x))
        lev.vecs = new
        self._build(0)
        for l in range(1, self.nlevels - 1):
            self._smooth_sweep(l)
            self._build(l)

    # ---------------- solve ----------------
    def coarse_solve(self, l, r):
        """Solve on level l (l >= 1): GMRES at the coarsest level, else one cycle
        (V-cycle) or a short FGMRES preconditioned by the cycle (K-cycle)."""
        if l == self.nlevels - 1:
            if self.p.coarse_eo:
                return coarse_eo_solve(self.levels[l].op, self.levels[l].dims, r, self.p.coarse_restart,
                                       self.p.coarse_tol, self.p.coarse_maxiter)
            x, _ = gmres(self.levels[l].op, r, restart=self.p.coarse_restart,
                         tol=self.p.coarse_tol, maxiter=self.p.coarse_maxiter)
            return x
        if self.p.kcycle:
            x, _ = fgmres(self.levels[l].op, r, lambda v: self.cycle(l, v), restart=self.p.kcycle_steps,
                          tol=self.p.kcycle_tol, maxiter=self.p.kcycle_steps)
            return x
        return self.cycle(l, r)

    def cycle(self, l, r):
        lev = self.levels[l]
        e = lev.agg.prolong(self.coarse_solve(l + 1, lev.agg.restrict(r)))
        return e + self.smooth(l, r - lev.op(e))

    def solve(self, b, x0=None):
        return fgmres(self.levels[0].op, b, lambda v: self.cycle(0, v),
                      restart=self.p.outer_restart, tol=self.p.outer_tol,
                      maxiter=self.p.outer_maxiter, x0=x0, verify=True)

    def solve_even_odd(self, b):
        """Even-odd (red-black) preconditioned outer solve (Sec. 4 lists red-black
        preconditioning among the missing features).  With sites even / odd by the
        parity of x + y + z + t, D = [[C_ee, H_eo], [H_oe, C_oo]]:
          b^_o = b_o - H_oe C_ee^-1 b_e,
          FGMRES on S = C_oo - H_oe C_ee^-1 H_eo, right-preconditioned by the odd-odd
          block of the MG cycle (S^-1 is the odd-odd block of D^-1), stopping when
          ||b^_o - S x_o|| <= outer_tol ||b|| (equal to the full residual),
          x_e = C_ee^-1 (b_e - H_eo x_o).
        Odd-site vectors are kept as full fields that vanish on even sites."""
        D = self.levels[0].op
        ev = (parity(self.levels[0].dims) == 0)[..., None]
        od = ~ev
        b_hat = np.where(od, b - D(np.where(ev, self_solve(D, b), 0)), 0)

        def schur(v):
            Dv = D(v)
            return np.where(od, Dv - D(np.where(ev, self_solve(D, np.where(ev, Dv, 0)), 0)), 0)

        tol = self.p.outer_tol * norm(b) / norm(b_hat)
        x_o, info = fgmres(schur, b_hat, lambda v: np.where(od, self.cycle(0, v), 0),
                           restart=self.p.outer_restart, tol=tol, maxiter=self.p.outer_maxiter, verify=True)
        x_e = np.where(ev, self_solve(D, b - D(x_o)), 0)
        return x_e + x_o, info
