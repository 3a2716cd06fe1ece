"""Wilson-clover Dirac operator D (oracle; test infrastructure).

The paper runs multigrid directly on the Wilson-clover matrix D (Sec. 2.1) and
uses its gamma5-hermiticity (Sec. 2.2); it does not write D down.  Reading used
here (standard Sheikholeslami-Wohlert form, no kappa normalisation, periodic in
all four directions):

  D psi(x) = C(x) psi(x)
             - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                          + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]

  C(x) = (4 + m0) 1 + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} Fhat_{mu nu}(x)
       = (4 + m0) 1 + (c_sw/2) sum_{mu<nu} sigma_{mu nu} (x) (i Fhat_{mu nu}(x))

  Fhat_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag) / 8, Q_{mu nu}(x) = sum of the four
  plaquette leaves around x in the (mu, nu) plane, all with the same orientation,
  no trace subtraction.

The operator is stored as a nine-point stencil: D = S + sum_{mu, +-} H_{+-mu},
where S(x) = C(x) and H_{+mu} (H_{-mu}) is the term that reads psi(x + mu)
(psi(x - mu)).  The Galerkin coarsening (coarse.py) uses exactly this split.
"""
import numpy as np

from .gamma import GAMMA, sigma
from .lattice import shift, to_grid

I4 = np.eye(4, dtype=np.complex128)


def _mm(a, b):
    return np.einsum("...ij,...jk->...ik", a, b)


def _dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def plaquette_leaves(U: np.ndarray, mu: int, nu: int):
    """The four leaves of the clover at x in the (mu, nu) plane, each a closed
    path starting and ending at x with the orientation mu -> nu."""
    Um, Un = U[mu], U[nu]
    s = shift
    l1 = _mm(_mm(Um, s(Un, mu, +1)), _mm(_dag(s(Um, nu, +1)), _dag(Un)))
    Um_m = s(Um, mu, -1)
    l2 = _mm(_mm(Un, _dag(s(Um_m, nu, +1))), _mm(_dag(s(Un, mu, -1)), Um_m))
    Umn = s(Um_m, nu, -1)
    l3 = _mm(_mm(_dag(Um_m), _dag(s(s(Un, mu, -1), nu, -1))), _mm(Umn, s(Un, nu, -1)))
    Un_n = s(Un, nu, -1)
    l4 = _mm(_mm(_dag(Un_n), s(Um, nu, -1)), _mm(s(Un_n, mu, +1), _dag(Um)))
    return l1, l2, l3, l4


def field_strength(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Fhat_{mu nu}(x) = (Q - Q^dag)/8 (anti-Hermitian 3x3 per site)."""
    Q = sum(plaquette_leaves(U, mu, nu))
    return (Q - _dag(Q)) / 8.0


def clover_term(U: np.ndarray, m0: float, csw: float) -> np.ndarray:
    """C(x) as a 12x12 matrix per site (index 3*spin + colour), shape (T,Z,Y,X,12,12)."""
    site_shape = U.shape[1:5]
    C = np.zeros(site_shape + (12, 12), dtype=np.complex128)
    C[...] = (4.0 + m0) * np.eye(12)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            iF = 1j * field_strength(U, mu, nu)
            sg = sigma(mu, nu)
            C += (csw / 2.0) * np.einsum("st,...ab->...satb", sg, iF).reshape(site_shape + (12, 12))
    return C


class WilsonClover:
    """D on a periodic lattice; fields are (T, Z, Y, X, 12) complex128."""

    ncomp = 12

    def __init__(self, U_ext: np.ndarray, dims, m0: float, csw: float, clover=None):
        self.dims = tuple(dims)
        self.m0, self.csw = float(m0), float(csw)
        self.U = np.stack([to_grid(U_ext[mu], dims) for mu in range(4)])  # (4,T,Z,Y,X,3,3)
        self.C = clover_term(self.U, m0, csw) if clover is None else clover

    # ----- nine-point stencil pieces -----
    def apply_self(self, psi):
        return np.einsum("...ab,...b->...a", self.C, psi)

    def apply_hop(self, mu: int, sign: int, psi):
        sh = psi.shape
        p = shift(psi, mu, sign).reshape(sh[:4] + (4, 3))
        if sign > 0:
            t = np.einsum("...ab,...sb->...sa", self.U[mu], p)
            proj = I4 - GAMMA[mu]
        else:
            Ub = shift(self.U[mu], mu, -1)
            t = np.einsum("...ba,...sb->...sa", np.conj(Ub), p)
            proj = I4 + GAMMA[mu]
        return (-0.5 * np.einsum("st,...tb->...sb", proj, t)).reshape(sh)

    def apply(self, psi):
        out = self.apply_self(psi)
        for mu in range(4):
            for sign in (+1, -1):
                out = out + self.apply_hop(mu, sign, psi)
        return out

    __call__ = apply
