"""Pins of block orthonormalisation, P and P^dag (Sec. 2.1 intergrid operators,
Sec. 2.2 chirality split, Sec. 3 block projection)."""
import itertools

import numpy as np

from oracle.aggregation import Aggregation
from oracle.gamma import GAMMA5
from oracle.lattice import to_grid
from paper_1904_08678_gb300 import inputs
from tests.helpers import rel, vdot

DIMS = (4, 2, 6, 4)
BLOCK = (2, 1, 3, 2)
NVEC = 5


def make_agg(dims=DIMS, block=BLOCK, nvec=NVEC, nc=12):
    V = int(np.prod(dims))
    vecs = [to_grid(v, dims) for v in inputs.complex_gaussian(21, 0, (nvec, V, nc))]
    return Aggregation(dims, block, vecs), vecs


def block_sites(dims, block, xc):
    """Fine (t, z, y, x) indices of aggregate xc = (xc, yc, zc, tc), by explicit loops."""
    out = []
    for dt, dz, dy, dx in itertools.product(range(block[3]), range(block[2]), range(block[1]), range(block[0])):
        out.append((xc[3] * block[3] + dt, xc[2] * block[2] + dz, xc[1] * block[1] + dy, xc[0] * block[0] + dx))
    return out


def test_qr_uniqueness_per_aggregate():
    """Q^dag M is upper triangular with a positive real diagonal and Q^dag Q = 1:
    this fixes Q uniquely for a full-rank panel M."""
    agg, raw = make_agg()
    cd = agg.cdims
    for xc in itertools.product(*[range(c) for c in cd]):
        sites = block_sites(DIMS, BLOCK, xc)
        for s in range(2):
            comps = range(6 * s, 6 * s + 6)
            M = np.array([[raw[i][st + (c,)] for i in range(NVEC)] for st in sites for c in comps])
            Q = np.array([[agg.v[i][st + (c,)] for i in range(NVEC)] for st in sites for c in comps])
            assert np.allclose(Q.conj().T @ Q, np.eye(NVEC), atol=1e-14)
            R = Q.conj().T @ M
            assert np.allclose(np.tril(R, -1), 0, atol=1e-13)
            d = np.diag(R)
            assert np.all(np.abs(d.imag) < 1e-13) and np.all(d.real > 0)
            assert np.allclose(Q @ R, M, atol=1e-13)


def test_restrict_brute_force():
    agg, _ = make_agg()
    V = int(np.prod(DIMS))
    psi = to_grid(inputs.complex_gaussian(22, 0, (V, 12)), DIMS)
    phi = agg.restrict(psi)
    for xc in itertools.product(*[range(c) for c in agg.cdims]):
        for s in range(2):
            for i in range(NVEC):
                acc = 0j
                for st in block_sites(DIMS, BLOCK, xc):
                    for c in range(6 * s, 6 * s + 6):
                        acc += np.conj(agg.v[i][st + (c,)]) * psi[st + (c,)]
                got = phi[xc[3], xc[2], xc[1], xc[0], s * NVEC + i]
                assert abs(got - acc) < 1e-13 * max(1, abs(acc))


def test_p_dag_p_identity_and_adjoint():
    agg, _ = make_agg()
    Vc = int(np.prod(agg.cdims))
    V = int(np.prod(DIMS))
    phi = to_grid(inputs.complex_gaussian(23, 0, (Vc, agg.nbasis)), agg.cdims)
    psi = to_grid(inputs.complex_gaussian(23, 1, (V, 12)), DIMS)
    assert rel(agg.restrict(agg.prolong(phi)), phi) < 1e-14
    lhs = vdot(agg.prolong(phi), psi)
    rhs = vdot(phi, agg.restrict(psi))
    assert abs(lhs - rhs) < 1e-13 * abs(rhs)


def test_gamma5_P_equals_P_sigma3():
    agg, _ = make_agg()
    Vc = int(np.prod(agg.cdims))
    phi = to_grid(inputs.complex_gaussian(24, 0, (Vc, agg.nbasis)), agg.cdims)
    sig3 = np.concatenate([np.ones(NVEC), -np.ones(NVEC)])
    g5 = np.kron(GAMMA5, np.eye(3))
    lhs = np.einsum("ab,...b->...a", g5, agg.prolong(phi))
    rhs = agg.prolong(phi * sig3)
    assert np.abs(lhs - rhs).max() < 1e-15


def test_coarse_level_chirality_is_component_halves():
    """On a coarse level (nc = 2*Nvec) the chirality split is first/second half."""
    dims, block = (4, 4, 2, 2), (2, 2, 1, 1)
    V = int(np.prod(dims))
    vecs = [to_grid(v, dims) for v in inputs.complex_gaussian(25, 0, (3, V, 8))]
    agg = Aggregation(dims, block, vecs)
    Vc = int(np.prod(agg.cdims))
    phi = to_grid(inputs.complex_gaussian(25, 1, (Vc, 6)), agg.cdims)
    up = agg.prolong(phi * np.array([1, 1, 1, 0, 0, 0]))
    assert np.abs(up[..., 4:]).max() == 0
    assert rel(agg.restrict(agg.prolong(phi)), phi) < 1e-14
