"""Euclidean gamma matrices in the chiral basis (oracle; test infrastructure).

The paper relies on gamma5-hermiticity (Sec. 2.2) and on the chiral projections
(1 +- gamma5)/2 of the prolongator (Sec. 2.2) but does not print a basis.  Reading
used here (Hermitian, chiral):
    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = x, y, z)
    gamma_t = [[0, 1], [1, 0]]
    gamma5  = gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1)
so spins 0,1 carry chirality + and spins 2,3 chirality -.
"""
import numpy as np

PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def gammas() -> np.ndarray:
    """gamma_mu for mu = 0..3 (x, y, z, t), shape (4, 4, 4)."""
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    z = np.zeros((2, 2))
    for k in range(3):
        g[k] = np.block([[z, -1j * PAULI[k]], [1j * PAULI[k], z]])
    g[3] = np.block([[z, np.eye(2)], [np.eye(2), z]])
    return g


GAMMA = gammas()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])
