"""Pins of the oracle's Wilson-clover operator D (the fine operator of Sec. 2.1).

Each test checks D against something other than its own formula:
  * free-field plane waves against the closed-form momentum-space D(p);
  * gamma5-hermiticity (Sec. 2.2) for random SU(3) fields;
  * gauge covariance under a random SU(3) gauge transformation;
  * the clover term of abelian fields against closed forms built from link phases.
"""
import numpy as np
import pytest

from oracle.gamma import GAMMA, GAMMA5, sigma
from oracle.lattice import to_grid
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.helpers import rel, vdot

DIMS = (4, 6, 2, 8)  # anisotropic on purpose: a mixed-up axis fails


def coords(dims):
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.indices((Lt, Lz, Ly, Lx))
    return x, y, z, t


@pytest.mark.parametrize("m0", [-0.1, 0.37])
def test_free_field_plane_waves(m0):
    U = inputs.unit_gauge(DIMS)
    D = WilsonClover(U, DIMS, m0, csw=1.7)  # the clover vanishes at U = 1
    rng = np.random.default_rng(3)
    xs = coords(DIMS)
    for _ in range(6):
        n = [rng.integers(0, L) for L in DIMS]
        p = [2 * np.pi * n[mu] / DIMS[mu] for mu in range(4)]
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        phase = np.exp(1j * sum(p[mu] * xs[mu] for mu in range(4)))
        psi = (phase[..., None, None] * u).reshape(phase.shape + (12,))
        Dp = (m0 + sum(1 - np.cos(pm) for pm in p)) * np.eye(4) + 1j * sum(
            GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
        expect = (phase[..., None, None] * (Dp @ u)).reshape(psi.shape)
        assert rel(D(psi), expect) < 1e-14


def test_free_field_spectrum_small_lattice():
    dims = (2, 2, 2, 4)
    m0 = -0.3
    D = WilsonClover(inputs.unit_gauge(dims), dims, m0, csw=1.0)
    n = 12 * 32
    M = np.zeros((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex); e[j] = 1
        M[:, j] = D(to_grid(e.reshape(-1, 12), dims)).ravel()
    ev = np.sort_complex(np.round(np.linalg.eigvals(M), 10))
    expect = []
    for nt in range(4):
        for nz in range(2):
            for ny in range(2):
                for nx in range(2):
                    p = [2 * np.pi * nx / 2, 2 * np.pi * ny / 2, 2 * np.pi * nz / 2, 2 * np.pi * nt / 4]
                    re = m0 + sum(1 - np.cos(q) for q in p)
                    im = np.sqrt(sum(np.sin(q) ** 2 for q in p))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.sort_complex(np.round(np.array(expect), 10))
    assert np.allclose(ev, expect, atol=1e-9)


def test_gamma5_hermiticity():
    U = inputs.random_gauge(DIMS, 0.5, seed=11)
    D = WilsonClover(U, DIMS, -0.2, 1.3)
    V = int(np.prod(DIMS))
    phi = to_grid(inputs.complex_gaussian(5, 1, (V, 12)), DIMS)
    psi = to_grid(inputs.complex_gaussian(5, 2, (V, 12)), DIMS)
    g5 = np.kron(GAMMA5, np.eye(3))
    g5f = lambda f: np.einsum("ab,...b->...a", g5, f)
    lhs = vdot(phi, g5f(D(g5f(psi))))
    rhs = vdot(D(phi), psi)
    assert abs(lhs - rhs) / abs(rhs) < 1e-14
    # and D itself is not Hermitian (the hop is anti-Hermitian in part)
    assert abs(vdot(phi, D(psi)) - vdot(D(phi), psi)) / abs(rhs) > 1e-3


def test_gauge_covariance():
    U = inputs.random_gauge(DIMS, 0.4, seed=12)
    Om = inputs.random_gauge_transform(DIMS, seed=13)
    V = Om.shape[0]
    Omg = to_grid(Om, DIMS)
    Up = np.empty_like(U)
    for mu in range(4):
        Ug = to_grid(U[mu], DIMS)
        Om_fwd = np.roll(Omg, -1, axis=3 - mu)
        Up[mu] = (Omg @ Ug @ np.conj(np.swapaxes(Om_fwd, -1, -2))).reshape(V, 3, 3)
    D = WilsonClover(U, DIMS, 0.1, 1.1)
    Dp = WilsonClover(Up, DIMS, 0.1, 1.1)
    psi = to_grid(inputs.complex_gaussian(5, 3, (V, 12)), DIMS)
    rot = lambda f: np.einsum("...ab,...sb->...sa", Omg, f.reshape(f.shape[:4] + (4, 3))).reshape(f.shape)
    assert rel(Dp(rot(psi)), rot(D(psi))) < 1e-13


def _abelian_links(theta, charges=(1, 1, -2)):
    """U_mu(x) = diag(exp(i q_c theta_mu(x))) from angles theta[mu] of shape (T,Z,Y,X)."""
    q = np.array(charges, dtype=float)
    U = np.zeros((4,) + theta.shape[1:] + (3, 3), dtype=complex)
    for c in range(3):
        U[..., c, c] = np.exp(1j * q[c] * theta)
    return U.reshape(4, -1, 3, 3), q


@pytest.mark.parametrize("plane", [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
def test_uniform_abelian_flux_clover(plane):
    """Uniform flux phi through every (mu, nu) plaquette: C - (4 + m0) =
    -(c_sw/2) sin(q_c phi) sigma_{mu nu} (x) e_c e_c^dag, and zero in other planes."""
    dims = (4, 6, 4, 6)
    mu, nu = plane
    Lmu, Lnu = dims[mu], dims[nu]
    k = 1
    phi = 2 * np.pi * k / (Lmu * Lnu)
    x = coords(dims)
    theta = np.zeros((4,) + x[0].shape)
    theta[nu] = phi * x[mu]
    theta[mu] = np.where(x[mu] == Lmu - 1, -phi * Lmu * x[nu], 0.0)
    U, q = _abelian_links(theta)
    m0, csw = -0.3, 1.25
    D = WilsonClover(U, dims, m0, csw)
    C = D.C - (4 + m0) * np.eye(12)
    expect = np.zeros(12 * 12, dtype=complex).reshape(12, 12)
    for c in range(3):
        ec = np.zeros((3, 3)); ec[c, c] = 1
        expect += -(csw / 2) * np.sin(q[c] * phi) * np.kron(sigma(mu, nu), ec)
    assert np.abs(C - expect).max() < 1e-14


def test_random_abelian_clover_leaves():
    """For abelian links every leaf is exp(i q theta_P) of a plaquette touching x, so
    Fhat_{mu nu}(x) = (i/4) sum over the four plaquettes with a corner at x of sin(q theta_P)."""
    dims = (4, 4, 6, 4)
    rng = np.random.default_rng(8)
    theta = rng.uniform(-np.pi, np.pi, size=(4, dims[3], dims[2], dims[1], dims[0]))
    U, q = _abelian_links(theta)
    m0, csw = 0.2, 0.9
    D = WilsonClover(U, dims, m0, csw)
    sh = lambda f, m, s: np.roll(f, -s, axis=3 - m)
    expect = np.zeros(theta.shape[1:] + (12, 12), dtype=complex)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            tp = theta[mu] + sh(theta[nu], mu, 1) - sh(theta[mu], nu, 1) - theta[nu]  # plaquette at corner
            corners = [tp, sh(tp, mu, -1), sh(sh(tp, mu, -1), nu, -1), sh(tp, nu, -1)]
            for c in range(3):
                iF = 1j * (1j / 4) * sum(np.sin(q[c] * a) for a in corners)
                ec = np.zeros((3, 3)); ec[c, c] = 1
                expect += (csw / 2) * iF[..., None, None] * np.kron(sigma(mu, nu), ec)
    C = D.C - (4 + m0) * np.eye(12)
    assert np.abs(C - expect).max() < 1e-13
