"""Pins of the chiral gamma basis (Sec. 2.2 relies on gamma5 being diagonal)."""
import numpy as np

from oracle.gamma import GAMMA, GAMMA5, sigma


def test_clifford_algebra_exact():
    for mu in range(4):
        assert np.array_equal(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            anti = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.array_equal(anti, 2.0 * (mu == nu) * np.eye(4))


def test_gamma5_is_chiral_diagonal():
    assert np.array_equal(GAMMA5, np.diag([1, 1, -1, -1]).astype(complex))
    for mu in range(4):
        assert np.array_equal(GAMMA5 @ GAMMA[mu], -GAMMA[mu] @ GAMMA5)


def test_sigma_block_diagonal_in_chirality():
    for mu in range(4):
        for nu in range(4):
            s = sigma(mu, nu)
            assert np.allclose(s, s.conj().T)
            assert np.allclose(s[:2, 2:], 0) and np.allclose(s[2:, :2], 0)
    # sigma_xy = diag(-1, 1, -1, 1) in this basis (checked by hand from gamma_x gamma_y = i sigma_3 (+) i sigma_3)
    assert np.allclose(sigma(0, 1), np.diag([-1, 1, -1, 1]))
