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


def block_mr(op, dims, block, r, steps):
    """MR_k(D_B; r) from a zero guess, every block with its own step length."""
    e = np.zeros_like(r)
    for _ in range(steps):
        p = block_interior(op, dims, block, r)
        pr = block_sum(np.conj(p) * r, block)
        pp = block_sum(np.abs(p) ** 2, block).real
        alpha = np.where(pp != 0.0, pr / np.where(pp != 0.0, pp, 1.0), 0.0)
        a = expand(alpha, block)
        e = e + a * r
        r = r - a * p
    return e


def sap(op, dims, block, b, steps, cycles):
    """The SAP smoother from a zero initial guess."""
    col = colour(dims, block)[..., None]
    x = np.zeros_like(b)
    for _ in range(cycles):
        for c in (0, 1):
            r = np.where(col == c, b - op(x), 0)
            x = x + block_mr(op, dims, block, r, steps)
    return x
