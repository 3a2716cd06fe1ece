"""Coarse-grid operator D_c = P^dag D P as a nine-point stencil
(oracle; test infrastructure).

Sec. 2.1: CoarsenedMatrix creates the coarse Dslash (CoarsenOperator) and applies
it through Mdiag (the site-diagonal block) and Mdir (the hop in one direction);
the coarse matrix can itself be coarsened again using only these two, which gives
any number of levels.  Sec. 4: Grid's CoarsenOperator uses 9 stencil points.

Block order d = 0 self, d = 1 + 2 mu the +mu hop, d = 2 + 2 mu the -mu hop:
    y(x_c) = A_0(x_c) phi(x_c) + sum_mu [A_{+mu}(x_c) phi(x_c + mu) + A_{-mu}(x_c) phi(x_c - mu)].

Galerkin construction (reading): A_{+mu}(x_c)[a][b] collects every term of D from
a fine site x of aggregate x_c whose +mu neighbour lies in the next aggregate
(the +mu face of x_c), between column a of P at x and column b of P at x + mu;
likewise A_{-mu} for the -mu face.  The site term and all hops inside one
aggregate go to A_0.  Where the coarse extent is 2, x_c + mu = x_c - mu and the two
blocks stay separate (keyed by the face crossed); their sum is the dense entry.
"""
import numpy as np

from .lattice import face_mask, shift


def block_index(mu: int, sign: int) -> int:
    return 1 + 2 * mu + (0 if sign > 0 else 1)


class CoarseOperator:
    """Nine-block coarse operator; A has shape (9, Tc, Zc, Yc, Xc, nb, nb)."""

    def __init__(self, A: np.ndarray, dims):
        self.A = A
        self.dims = tuple(dims)
        self.ncomp = A.shape[-1]

    def apply_self(self, phi):
        """Mdiag: y(x) = A_0(x) phi(x)."""
        return np.einsum("...ab,...b->...a", self.A[0], phi)

    def apply_hop(self, mu: int, sign: int, phi):
        """Mdir: y(x) = A_{+-mu}(x) phi(x +- mu)."""
        return np.einsum("...ab,...b->...a", self.A[block_index(mu, sign)], shift(phi, mu, sign))

    def apply(self, phi):
        out = self.apply_self(phi)
        for mu in range(4):
            for sign in (+1, -1):
                out = out + self.apply_hop(mu, sign, phi)
        return out

    __call__ = apply


def coarsen(op, agg) -> CoarseOperator:
    """CoarsenOperator: the nine blocks of P^dag D P, column by column of P."""
    nb = agg.nbasis
    A = np.zeros((9,) + agg.cdims[::-1] + (nb, nb), dtype=np.complex128)
    faces = {(mu, s): face_mask(agg.fine_dims, agg.block, mu, s)[..., None]
             for mu in range(4) for s in (+1, -1)}
    for b in range(nb):
        Vb = agg.column_field(b)
        A[0][..., :, b] += agg.restrict(op.apply_self(Vb))
        for mu in range(4):
            for sign in (+1, -1):
                W = op.apply_hop(mu, sign, Vb)
                f = faces[(mu, sign)]
                A[block_index(mu, sign)][..., :, b] += agg.restrict(np.where(f, W, 0))
                A[0][..., :, b] += agg.restrict(np.where(f, 0, W))
    return CoarseOperator(A, agg.cdims)
