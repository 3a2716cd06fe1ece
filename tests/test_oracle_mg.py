"""Pins of the multigrid cycle and solve (Sec. 2.1 recursive solver class,
FGMRES outer solver right-preconditioned by the MG cycle)."""
import numpy as np
import pytest

from oracle.lattice import to_grid
from oracle.mg import MGParams, Multigrid
from oracle.solvers import gmres
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.helpers import rel


def config1(eps=0.3, m0=-0.1):
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, eps, 1001)
    D = WilsonClover(U, dims, m0, 1.0)
    V = int(np.prod(dims))
    b = to_grid(inputs.source(dims, 0)[0].reshape(V, 12), dims)
    return dims, D, b


def test_block_1_nvec_6_is_exact_preconditioner():
    """Block 1^4 with Nvec = 6: P is unitary per site, D_c is unitarily similar to D,
    and with an exact coarse solve the cycle is D^-1: FGMRES needs one iteration."""
    dims, D, b = config1()
    V = int(np.prod(dims))
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 6, 0, 1001)]]
    p = MGParams(blocks=[(1, 1, 1, 1)], nvecs=[6], init_sweeps=1, coarse_restart=400,
                 coarse_tol=1e-13, coarse_maxiter=4000, outer_tol=1e-10)
    mg = Multigrid(D, p, iv)
    x, info = mg.solve(b)
    assert info.converged and info.iterations == 1


def test_config1_solve_matches_dense_solution():
    dims, D, b = config1()
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 8, 0, 1001)]]
    mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[8]), iv)
    x, info = mg.solve(b)
    assert info.converged and info.true_residual <= 1e-10
    x_ref, ir = gmres(D, b, restart=60, tol=1e-13, maxiter=5000, verify=True)
    assert ir.converged
    assert rel(x, x_ref) < 1e-8
    # the preconditioner helps: far fewer outer iterations than unpreconditioned GMRES(20)
    _, plain = gmres(D, b, restart=20, tol=1e-10, maxiter=5000, verify=True)
    assert info.iterations * 3 < plain.iterations


@pytest.mark.slow
def test_three_level_solve_converges():
    dims = (8, 8, 8, 8)
    U = inputs.random_gauge(dims, 0.3, 1003)
    D = WilsonClover(U, dims, -0.1, 1.0)
    V = int(np.prod(dims))
    b = to_grid(inputs.source(dims, 0)[0].reshape(V, 12), dims)
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 6, 0, 1003)],
          [to_grid(v, (4, 4, 4, 4)) for v in inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1003)]]
    p = MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvecs=[6, 4], refine_sweeps=1)
    mg = Multigrid(D, p, iv)
    x, info = mg.solve(b)
    assert info.converged and info.true_residual <= 1e-10
    assert rel(D(x), b) <= 1e-10


def test_refinement_reduces_iterations():
    """Sec. 2.1 / Table 2 trend: iterative-refinement sweeps improve the near-null space.

    The field strength and mass (eps 0.3, m0 -0.6) follow the gauge reading in which
    X = sum_a xi_a lambda_a has unit Gaussian coefficients in the Gell-Mann basis (no
    factor 1/2): with that normalisation the links are rougher, so m0 = -0.6 keeps D
    away from criticality on 4^4 while leaving the near-null space poor enough after
    one initial sweep that refinement has something to improve."""
    dims, D, b = config1(eps=0.3, m0=-0.6)
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 4, 0, 1001)]]
    its = []
    for nref in (0, 3):
        mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[4], init_sweeps=1, refine_sweeps=nref), iv)
        x, info = mg.solve(b)
        assert info.converged
        its.append(info.iterations)
    assert its[1] < its[0]


def test_gmres_smoother_never_leaves_a_larger_residual_than_mr():
    """MR(k) and GMRES(k) from a zero guess both stay in the Krylov space K_k(D, r);
    GMRES(k) minimises ||r - D x|| over all of it, so its smoothed residual is never
    larger than MR's (and differs from it: a dropped term in either shows here)."""
    dims, D, b = config1()
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 8, 0, 1001)]]
    for k in (1, 2, 4, 6):
        res = {}
        for sm in ("mr", "gmres"):
            mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[8], smoother_steps=k, smoother=sm), iv,
                           build=False)
            x = mg.smooth(0, b)
            res[sm] = np.linalg.norm((b - D(x)).ravel())
        assert res["gmres"] <= res["mr"] * (1 + 1e-12)
        if k == 1:
            assert abs(res["gmres"] - res["mr"]) <= 1e-12 * res["mr"]  # one step: the same minimiser
        else:
            assert res["gmres"] < res["mr"] * (1 - 1e-6)


def test_gmres_smoother_solve_converges_to_the_dense_solution():
    dims, D, b = config1()
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 8, 0, 1001)]]
    mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[8], smoother="gmres"), iv)
    x, info = mg.solve(b)
    assert info.converged and info.true_residual <= 1e-10
    x_ref, _ = gmres(D, b, restart=60, tol=1e-13, maxiter=5000, verify=True)
    assert rel(x, x_ref) < 1e-8


def three_level_parts(kcycle, steps=5, tol=0.1):
    dims = (8, 8, 8, 8)
    U = inputs.random_gauge(dims, 0.3, 1003)
    D = WilsonClover(U, dims, -0.1, 1.0)
    iv0 = [to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 6, 0, 1003)]
    iv1 = [to_grid(v, (4, 4, 4, 4)) for v in inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1003)]
    p = MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvecs=[6, 4], kcycle=kcycle, kcycle_steps=steps, kcycle_tol=tol)
    return dims, D, iv0, iv1, Multigrid(D, p, [iv0, iv1])


@pytest.mark.slow
def test_kcycle_with_exact_inner_solve_is_the_two_level_cycle_with_exact_coarse_solve():
    """With its FGMRES run to 1e-13 the K-cycle's intermediate solve is D_1^-1, so the
    three-level K-cycle equals the two-level cycle (same P_0) whose coarse GMRES is
    exact; the V-cycle (one cycle of level 1) does not."""
    dims, D, iv0, iv1, mgk = three_level_parts(True, steps=120, tol=1e-13)
    mg2 = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[6], coarse_restart=120, coarse_tol=1e-13,
                                coarse_maxiter=3000), [iv0])
    _, _, _, _, mgv = three_level_parts(False)
    V = int(np.prod(dims))
    r = to_grid(inputs.complex_gaussian(31, 0, (1, V, 12))[0], dims)
    ek, e2, ev = mgk.cycle(0, r), mg2.cycle(0, r), mgv.cycle(0, r)
    assert rel(ek, e2) < 1e-9
    assert rel(ev, e2) > 1e4 * max(rel(ek, e2), 1e-16)  # one V-cycle is far from the exact coarse solve


@pytest.mark.slow
def test_kcycle_solve_needs_no_more_iterations_than_the_vcycle():
    dims, D, iv0, iv1, mgk = three_level_parts(True)
    _, _, _, _, mgv = three_level_parts(False)
    V = int(np.prod(dims))
    b = to_grid(inputs.source(dims, 0)[0].reshape(V, 12), dims)
    xk, ik = mgk.solve(b)
    xv, iv = mgv.solve(b)
    assert ik.converged and iv.converged and ik.true_residual <= 1e-10
    assert ik.iterations <= iv.iterations
    assert rel(xk, xv) < 1e-8


# ---- the setup as inverse iteration (special cases with an exact smoother / cycle) ----
# On the free field (U = 1) of a lattice with extent 2 in every direction the momenta are
# p_mu in {0, pi}, so sin p_mu = 0 and the free Wilson operator is diagonal in momentum
# space with the real eigenvalue lambda(p) = 4 + m0 - sum_mu cos p_mu = m0 + 2 n_pi
# (n_pi: the number of components equal to pi), times the 12 x 12 identity.
FREE = (2, 2, 2, 2)


def free_operator(m0):
    V = int(np.prod(FREE))
    U = np.zeros((4, V, 3, 3), dtype=complex)
    U[:, :] = np.eye(3)
    return WilsonClover(U, FREE, m0, 1.0)


def free_inverse_power(v, m0, s):
    """D^-s v from the spectrum above (FFT over the four axes of the (T, Z, Y, X, 12) grid)."""
    F = np.fft.fftn(v, axes=(0, 1, 2, 3))
    p = [2 * np.pi * np.fft.fftfreq(n) for n in v.shape[:4]]
    pt, pz, py, px = np.meshgrid(*p, indexing="ij")
    lam = 4 + m0 - (np.cos(pt) + np.cos(pz) + np.cos(py) + np.cos(px))
    return np.fft.ifftn(F / lam[..., None] ** s, axes=(0, 1, 2, 3))


def free_vectors(n, seed):
    return [to_grid(v, FREE) for v in inputs.setup_vectors(FREE, 12, n, 0, seed)]


def test_free_spectrum_helper_inverts_the_operator():
    D, v = free_operator(-0.1), free_vectors(1, 1301)[0]
    assert rel(D(free_inverse_power(v, -0.1, 1)), v) < 1e-13


def test_initial_setup_is_normalised_inverse_iteration_with_an_exact_smoother():
    """GMRES with 5 steps solves the free operator exactly (5 distinct eigenvalues), so s
    initial sweeps give D^-s v0 / ||D^-s v0|| for every random vector v0."""
    m0 = -0.1
    D, iv = free_operator(m0), free_vectors(6, 1302)
    for s in (1, 3):
        mg = Multigrid(D, MGParams(blocks=[(1, 1, 1, 1)], nvecs=[6], smoother="gmres", smoother_steps=5,
                                   init_sweeps=s, refine_sweeps=0), [iv])
        for v0, v in zip(iv, mg.levels[0].vecs):
            want = free_inverse_power(v0, m0, s)
            assert rel(v, want / np.linalg.norm(want)) < 1e-12


def test_refinement_is_normalised_inverse_iteration_with_an_exact_cycle():
    """One-site aggregates with Nvec 6 make P unitary, so with a coarse solve to 1e-14 the
    cycle is D^-1 (the smoother then sees a zero residual): s refinement sweeps turn the
    vectors of the initial setup v into D^-s v / ||D^-s v||."""
    m0 = -0.1
    D, iv = free_operator(m0), free_vectors(6, 1303)
    kw = dict(blocks=[(1, 1, 1, 1)], nvecs=[6], init_sweeps=2, coarse_tol=1e-14, coarse_maxiter=200)
    v_init = Multigrid(D, MGParams(refine_sweeps=0, **kw), [iv]).levels[0].vecs
    v_ref = Multigrid(D, MGParams(refine_sweeps=2, **kw), [iv]).levels[0].vecs
    for v0, v in zip(v_init, v_ref):
        want = free_inverse_power(v0, m0, 2)
        assert rel(v, want / np.linalg.norm(want)) < 1e-10


def test_setup_sweeps_lower_the_rayleigh_quotient():
    """The MR(4) setup sweeps on a random gauge field drive every vector towards the low
    modes: ||D v|| / ||v|| falls with every sweep."""
    dims, D, _ = config1()
    iv = [to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 4, 0, 1304)]
    quotients = []
    for s in (0, 1, 2, 3):
        mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[4], init_sweeps=s, refine_sweeps=0), [iv])
        quotients.append([np.linalg.norm(D(v)) / np.linalg.norm(v) for v in mg.levels[0].vecs])
    q = np.array(quotients)
    assert np.all(q[1:] < q[:-1])


def test_even_odd_outer_solve_reaches_the_dense_solution():
    """The Schur-complement outer solve: its solution satisfies the full system to the
    outer tolerance and equals the dense solution; the odd-odd block of the cycle
    preconditions S about as well as the cycle preconditions D (within 2 iterations)."""
    dims, D, b = config1()
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 8, 0, 1001)]]
    mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[8]), iv)
    x, info = mg.solve_even_odd(b)
    assert info.converged
    assert np.linalg.norm(b - D(x)) <= 1.01e-10 * np.linalg.norm(b)
    x_ref, _ = gmres(D, b, restart=60, tol=1e-13, maxiter=5000, verify=True)
    assert rel(x, x_ref) < 1e-8
    _, plain = mg.solve(b)
    assert abs(info.iterations - plain.iterations) <= 2


def test_even_odd_coarsest_level_solve_reaches_the_dense_solution():
    """MG with the coarsest GMRES on the odd-site Schur complement (coarse_eo) preconditions
    FGMRES to the dense solution, in no more outer iterations than the plain coarsest
    solve (the Schur system is better conditioned, so its 0.05 GMRES is not worse)."""
    dims, D, b = config1()
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 8, 0, 1001)]]
    its = {}
    x_ref, _ = gmres(D, b, restart=60, tol=1e-13, maxiter=5000, verify=True)
    for eo in (False, True):
        mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[8], coarse_eo=eo), iv)
        x, info = mg.solve(b)
        assert info.converged and info.true_residual <= 1e-10
        its[eo] = info.iterations
        assert rel(x, x_ref) < 1e-8
    assert its[True] <= its[False] + 1


def test_setup_steps_are_invariant_under_positive_scaling():
    """The set-up normalises each vector after every sweep (inverse iteration), but every
    step that follows it is invariant under a positive scale c of a vector: the smoother
    (MR, and GMRES with a fixed number of steps) and the MG cycle, whose coarsest GMRES stops
    at a tolerance relative to its right-hand side, map c v to c times the result, and the
    block orthonormalisation (positive-diagonal QR per aggregate) of positively scaled
    columns is unchanged.  So an implementation may skip the normalisation: P and D_c stay
    the same up to rounding.  The scale factors span several decades."""
    from oracle.aggregation import block_orthonormalise
    from oracle.solvers import mr
    dims, D, b = config1()
    iv = [[to_grid(v, dims) for v in inputs.setup_vectors(dims, 12, 8, 0, 1001)]]
    for smoother in ("mr", "gmres"):
        mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[8], smoother=smoother), iv)
        for c in (1e-3, 7.3, 4.1e4):
            assert rel(mg.smooth(0, c * b), c * mg.smooth(0, b)) < 1e-13
            assert rel(mg.cycle(0, c * b), c * mg.cycle(0, b)) < 1e-12
    vecs = mg.levels[0].vecs
    scales = [10.0 ** (k - 3) * (1.0 + 0.1 * k) for k in range(len(vecs))]
    q1 = block_orthonormalise(vecs, (2, 2, 2, 2))
    q2 = block_orthonormalise([s * v for s, v in zip(scales, vecs)], (2, 2, 2, 2))
    assert rel(q2, q1) < 1e-13
    assert rel(mr(D, 3.0 * b, 4), 3.0 * mr(D, b, 4)) < 1e-14
