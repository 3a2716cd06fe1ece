"""Pins of MR, GMRES and FGMRES (Sec. 2.1) against optimality conditions, the
minimal-residual property over explicit Krylov bases, and dense solves."""
import numpy as np

from oracle.lattice import to_grid
from oracle.solvers import fgmres, gmres, mr, norm
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.helpers import rel, vdot


def rand_matrix(n, seed, shift=4.0):
    rng = np.random.default_rng(seed)
    return shift * np.eye(n) + rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))


def test_mr_step_is_residual_minimiser():
    A = rand_matrix(2, 1, shift=1.0)
    Af = lambda v: A @ v
    b = np.array([0.3 + 1j, -2.0 + 0.5j])
    x = mr(Af, b, 1)
    r = b - A @ x
    assert abs(vdot(A @ b, r)) < 1e-14  # first-order optimality along A b
    rng = np.random.default_rng(2)
    alpha = (x / b)[0]
    for _ in range(50):
        d = 1e-3 * (rng.normal() + 1j * rng.normal())
        assert norm(b - (alpha + d) * (A @ b)) >= norm(r)


def test_mr_iterations_reduce_residual_monotonically():
    A = rand_matrix(20, 3)
    b = np.ones(20, dtype=complex)
    res = [norm(b - A @ mr(lambda v: A @ v, b, k)) for k in range(8)]
    assert all(res[k + 1] <= res[k] + 1e-15 for k in range(7))


def test_gmres_minimal_residual_over_krylov_space():
    n = 30
    A = rand_matrix(n, 4, shift=2.0)
    b = np.random.default_rng(5).normal(size=n) + 0j
    x, info = gmres(lambda v: A @ v, b, restart=12, tol=0.0, maxiter=12)
    K = np.stack([np.linalg.matrix_power(A, j) @ b for j in range(12)], axis=1)
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
    best = norm(b - A @ Q @ y)
    assert abs(norm(b - A @ x) - best) < 1e-10 * norm(b)
    assert abs(info.history[-1] * norm(b) - best) < 1e-10 * norm(b)


def test_gmres_matches_dense_solve_with_restarts():
    n = 40
    A = rand_matrix(n, 6, shift=20.0)
    b = np.random.default_rng(7).normal(size=n) + 1j
    x, info = gmres(lambda v: A @ v, b, restart=5, tol=1e-12, maxiter=500, verify=True)
    assert info.converged and info.restarts > 0
    assert rel(x, np.linalg.solve(A, b)) < 1e-10


def test_fgmres_exact_preconditioner_one_iteration():
    n = 25
    A = rand_matrix(n, 8)
    Ainv = np.linalg.inv(A)
    b = np.random.default_rng(9).normal(size=n) + 0j
    x, info = fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, restart=10, tol=1e-12)
    assert info.iterations == 1 and info.converged
    assert rel(x, np.linalg.solve(A, b)) < 1e-13


def test_fgmres_identity_preconditioner_equals_gmres():
    n = 30
    A = rand_matrix(n, 10, shift=3.0)
    b = np.random.default_rng(11).normal(size=n) + 0j
    x1, i1 = fgmres(lambda v: A @ v, b, lambda v: v, restart=8, tol=1e-11, maxiter=300)
    x2, i2 = gmres(lambda v: A @ v, b, restart=8, tol=1e-11, maxiter=300, verify=True)
    assert i1.iterations == i2.iterations
    assert rel(x1, x2) < 1e-12


def test_gmres_on_wilson_clover_matches_dense_solve():
    dims = (2, 2, 2, 4)
    U = inputs.random_gauge(dims, 0.3, 41)
    D = WilsonClover(U, dims, 0.2, 1.0)
    V = int(np.prod(dims))
    b = to_grid(inputs.source(dims, 0)[0].reshape(V, 12), dims)
    x, info = gmres(D, b, restart=20, tol=1e-12, maxiter=2000, verify=True)
    n = V * 12
    M = np.stack([D(to_grid(np.eye(n)[j].reshape(V, 12), dims)).ravel() for j in range(n)], axis=1)
    assert info.converged
    assert rel(x.ravel(), np.linalg.solve(M, b.ravel())) < 1e-10


def test_givens_rotation_complex_inputs():
    from oracle.solvers import givens
    rng = np.random.default_rng(12)
    for _ in range(20):
        a, b = rng.normal(size=2) + 1j * rng.normal(size=2)
        c, s, rho = givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        assert np.allclose(G @ G.conj().T, np.eye(2), atol=1e-15)
        out = G @ np.array([a, b])
        assert abs(out[1]) < 1e-15 and abs(out[0] - rho) < 1e-14
    c, s, rho = givens(0.0, 2.0 + 1j)
    assert abs((np.array([[c, s], [-np.conj(s), c]]) @ np.array([0, 2 + 1j]))[1]) < 1e-15
