"""Schwarz alternating procedure (SAP) smoother (oracle; test infrastructure).

Sec. 4 (outlook) names SAP as the smoother commonly used on all multigrid levels and
gives no details of it.  Reading used here (multiplicative Schwarz over two colours of
blocks):

  * the blocks are the level's aggregates (the blocks of the next coarsening), coloured
    by the parity of the block's coordinates on the coarse lattice;
  * D_B is D with every hop that leaves its block removed (Dirichlet boundaries), i.e.
    the self term plus the hops between sites of the same block;
  * from x = 0, one SAP cycle is, for colour c = 0 then 1:
        r = b - D x restricted to the blocks of colour c,
        e = MR_k(D_B; r) with every block's own step length
            alpha_B = <p, r>_B / <p, p>_B   (sums over the block, p = D_B r),
        x += e;
  * the smoother S(D; b) is x after `cycles` SAP cycles.
Both the fine operator (WilsonClover) and a coarse operator (CoarseOperator) provide
the self / hop pieces this needs.

Even-odd (red-black) preconditioning of the block solves (Sec. 4 lists red-black
preconditioning among the missing features; the comparison code runs with it).  Reading
used here: sites are even or odd by the parity of x + y + z + t; the hops inside a block
connect opposite parities, so with D_B = [[C_ee, H_eo], [H_oe, C_oo]] (C the site-diagonal
self term, H the block-interior hops) the block system D_B e = r is solved as
  r^_o = r_o - H_oe C_ee^-1 r_e,
  e_o  = MR_k(S; r^_o) on the Schur complement S = C_oo - H_oe C_ee^-1 H_eo, one step
         length per block (sums over the block's odd sites),
  e_e  = C_ee^-1 (r_e - H_eo e_o).
With exact inner solves this is D_B^-1 r; with k MR steps it is a different (and better
conditioned) block smoother than MR_k on D_B.
"""
import numpy as np

from .lattice import face_mask, to_blocks


def block_interior(op, dims, block, f):
    """D_B f for all blocks at once (hops that leave a block dropped)."""
    out = op.apply_self(f)
    for mu in range(4):
        for sign in (+1, -1):
            leave = face_mask(dims, block, mu, sign)[..., None]
            out = out + np.where(leave, 0, op.apply_hop(mu, sign, f))
    return out


def colour(dims, block):
    """Colour (0 or 1) of the block of every site, shape (T, Z, Y, X)."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.indices((Lt, Lz, Ly, Lx))
    return (x // block[0] + y // block[1] + z // block[2] + t // block[3]) % 2


def block_sum(f, block):
    """Sum of f over each block's sites and components -> (Tc, Zc, Yc, Xc)."""
    return to_blocks(f, block).sum(axis=tuple(range(4, 4 + 4 + f.ndim - 4)))


def expand(a, block):
    """Per-block values (Tc, Zc, Yc, Xc) -> per-site (T, Z, Y, X, 1)."""
    bx, by, bz, bt = block
    e = np.repeat(np.repeat(np.repeat(np.repeat(a, bt, axis=0), bz, axis=1), by, axis=2), bx, axis=3)
    return e[..., None]


def _block_mr(apply, block, r, steps):
    """MR_k(A; r) from a zero guess for a block-diagonal A (apply), every block with its
    own step length alpha_B = <p, r>_B / <p, p>_B (0 if <p, p>_B = 0)."""
    e = np.zeros_like(r)
    for _ in range(steps):
        p = apply(r)
        pr = block_sum(np.conj(p) * r, block)
        pp = block_sum(np.abs(p) ** 2, block).real
        alpha = np.where(pp != 0.0, pr / np.where(pp != 0.0, pp, 1.0), 0.0)
        a = expand(alpha, block)
        e = e + a * r
        r = r - a * p
    return e


def block_mr(op, dims, block, r, steps):
    """MR_k(D_B; r) from a zero guess, every block with its own step length."""
    return _block_mr(lambda f: block_interior(op, dims, block, f), block, r, steps)


def parity(dims):
    """Site parity (x + y + z + t) % 2, shape (T, Z, Y, X)."""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.indices((Lt, Lz, Ly, Lx))
    return (x + y + z + t) % 2


def block_hops(op, dims, block, f):
    """H_B f: the hops of D between sites of the same block (no self term)."""
    out = np.zeros_like(f)
    for mu in range(4):
        for sign in (+1, -1):
            leave = face_mask(dims, block, mu, sign)[..., None]
            out = out + np.where(leave, 0, op.apply_hop(mu, sign, f))
    return out


def self_solve(op, f):
    """C(x)^-1 f(x) at every site: numpy's dense solver on each site's self block."""
    S = op.C if hasattr(op, "C") else op.A[0]
    return np.linalg.solve(S, f[..., None])[..., 0]


def block_mr_eo(op, dims, block, r, steps):
    """Even-odd preconditioned block solve: MR_k on each block's Schur complement on
    its odd sites, then the even sites by back substitution."""
    ev = (parity(dims) == 0)[..., None]
    od = ~ev
    hop = lambda f: block_hops(op, dims, block, f)
    r_hat = np.where(od, r - hop(np.where(ev, self_solve(op, r), 0)), 0)

    def schur(v):
        w = np.where(ev, self_solve(op, hop(v)), 0)
        return np.where(od, op.apply_self(v) - hop(w), 0)

    e_o = _block_mr(schur, block, r_hat, steps)
    e_e = np.where(ev, self_solve(op, r - hop(e_o)), 0)
    return e_e + e_o


def sap(op, dims, block, b, steps, cycles, eo=False):
    """The SAP smoother from a zero initial guess (eo: even-odd preconditioned block
    solves)."""
    col = colour(dims, block)[..., None]
    solve = block_mr_eo if eo else block_mr
    x = np.zeros_like(b)
    for _ in range(cycles):
        for c in (0, 1):
            r = np.where(col == c, b - op(x), 0)
            x = x + solve(op, dims, block, r, steps)
    return x
