"""Pins of the SAP smoother (oracle/sap.py): special cases that reduce to independent
computations, and the minimal-residual property of every block's step."""
import numpy as np

from oracle.coarse import CoarseOperator
from oracle.lattice import from_blocks, to_blocks, to_grid
from oracle.mg import MGParams, Multigrid
from oracle.sap import block_interior, block_mr, block_mr_eo, block_sum, colour, parity, sap
from oracle.solvers import gmres, mr
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.helpers import rel

DIMS = (4, 4, 4, 8)


def wilson(eps=0.3, m0=-0.1, seed=1101):
    U = inputs.random_gauge(DIMS, eps, seed)
    return WilsonClover(U, DIMS, m0, 1.0)


def field(seed):
    V = int(np.prod(DIMS))
    return to_grid(inputs.complex_gaussian(seed, 0, (1, V, 12))[0], DIMS)


def test_site_blocks_are_red_black_clover_solves():
    """Blocks of one site: D_B = C(x), MR converges to C(x)^-1 r, and one SAP cycle is
    the even-site then odd-site exact local solve (computed here with numpy's solver).
    40 MR steps reach rounding level; far more would drive the per-site residuals into
    underflow, where the step ratio is no longer meaningful."""
    D, b = wilson(), field(1102)
    got = sap(D, DIMS, (1, 1, 1, 1), b, steps=40, cycles=1)
    par = colour(DIMS, (1, 1, 1, 1))
    x = np.zeros_like(b)
    for c in (0, 1):
        r = b - D(x)
        e = np.linalg.solve(D.C, r[..., None])[..., 0]
        x = x + np.where((par == c)[..., None], e, 0)
    assert rel(got, x) < 1e-12


def test_one_block_is_mr_on_the_dirichlet_operator():
    """A single block covering the lattice: SAP(1 cycle) = MR_k on D with the periodic
    wrap-around hops removed (its step lengths are the global ones)."""
    D, b = wilson(), field(1103)
    blk = DIMS
    got = sap(D, DIMS, blk, b, steps=5, cycles=1)
    want = mr(lambda f: block_interior(D, DIMS, blk, f), b, 5)
    assert rel(got, want) < 1e-13


def test_every_block_step_minimises_its_block_residual():
    D, b = wilson(), field(1104)
    blk = (2, 2, 2, 2)
    r = b.copy()
    e = block_mr(D, DIMS, blk, r, 1)
    p = block_interior(D, DIMS, blk, r)
    r1 = r - block_interior(D, DIMS, blk, e)
    base = block_sum(np.abs(r1) ** 2, blk).real
    for da in (1e-3, -1e-3, 1e-3j):
        # perturbing every block's step by da raises every block's residual
        r2 = r1 - da * p
        assert np.all(block_sum(np.abs(r2) ** 2, blk).real >= base)


def test_more_sap_cycles_reduce_the_residual():
    D, b = wilson(), field(1105)
    res = []
    for cyc in (1, 2, 4):
        x = sap(D, DIMS, (2, 2, 2, 2), b, steps=4, cycles=cyc)
        res.append(np.linalg.norm(b - D(x)) / np.linalg.norm(b))
    assert res[0] > res[1] > res[2]


def test_sap_on_a_coarse_operator_matches_the_blockwise_definition():
    """The same smoother on a coarse nine-block operator: the block-interior operator
    equals the dense operator with its inter-block entries removed."""
    rng = np.random.default_rng(5)
    cd, nb = (4, 4, 4, 4), 4
    A = rng.normal(size=(9,) + cd[::-1] + (nb, nb)) + 1j * rng.normal(size=(9,) + cd[::-1] + (nb, nb))
    A[0] += 8 * np.eye(nb)
    op = CoarseOperator(A, cd)
    f = rng.normal(size=cd[::-1] + (nb,)) + 1j * rng.normal(size=cd[::-1] + (nb,))
    blk = (2, 2, 2, 2)
    got = block_interior(op, cd, blk, f)
    # dense reference: apply the full operator to f restricted to each block, keep that block
    want = np.zeros_like(f)
    T, Z, Y, X = cd[::-1]
    for tb in range(0, T, 2):
        for zb in range(0, Z, 2):
            for yb in range(0, Y, 2):
                for xb in range(0, X, 2):
                    m = np.zeros(cd[::-1], dtype=bool)
                    m[tb:tb + 2, zb:zb + 2, yb:yb + 2, xb:xb + 2] = True
                    y = op(np.where(m[..., None], f, 0))
                    want[m] = y[m]
    assert rel(got, want) < 1e-13


def test_sap_preconditioned_solve_converges_to_the_dense_solution():
    D = wilson()
    V = int(np.prod(DIMS))
    b = to_grid(inputs.source(DIMS, 0)[0].reshape(V, 12), DIMS)
    iv = [[to_grid(v, DIMS) for v in inputs.setup_vectors(DIMS, 12, 8, 0, 1101)]]
    mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[8], smoother="sap"), iv)
    x, info = mg.solve(b)
    assert info.converged and info.true_residual <= 1e-10
    x_ref, _ = gmres(D, b, restart=60, tol=1e-13, maxiter=5000, verify=True)
    assert rel(x, x_ref) < 1e-8


def block_matrices(op, dims, block, nc):
    """Dense D_B of every block, (nblocks, bvol*nc, bvol*nc) in (local site, component)
    order: one stencil application per (local site, component) with that unit vector
    set in every block at once (blocks do not couple under D_B)."""
    bx, by, bz, bt = block
    bvol = bx * by * bz * bt
    T, Z, Y, X = dims[::-1]
    nbk = (T // bt) * (Z // bz) * (Y // by) * (X // bx)
    M = np.zeros((nbk, bvol * nc, bvol * nc), dtype=complex)
    for j in range(bvol):
        lx, ly, lz, lt = j % bx, (j // bx) % by, (j // (bx * by)) % bz, j // (bx * by * bz)
        for c in range(nc):
            f = np.zeros((T, Z, Y, X, nc), dtype=complex)
            f[lt::bt, lz::bz, ly::by, lx::bx, c] = 1.0
            y = to_blocks(block_interior(op, dims, block, f), block)  # (Tc, Zc, Yc, Xc, bt, bz, by, bx, nc)
            M[:, :, j * nc + c] = y.reshape(nbk, bvol * nc)
    return M


def exact_block_solve(op, dims, block, r, nc):
    M = block_matrices(op, dims, block, nc)
    rb = to_blocks(r, block)
    e = np.linalg.solve(M, rb.reshape(M.shape[0], -1)[..., None])[..., 0]
    return from_blocks(e.reshape(rb.shape))


def test_block_matrices_reproduce_the_block_interior_operator():
    D, f = wilson(), field(1106)
    blk = (2, 2, 2, 2)
    M = block_matrices(D, DIMS, blk, 12)
    fb = to_blocks(f, blk)
    y = (M @ fb.reshape(M.shape[0], -1)[..., None])[..., 0]
    assert rel(from_blocks(y.reshape(fb.shape)), block_interior(D, DIMS, blk, f)) < 1e-14


def test_even_odd_block_solve_converges_to_the_exact_block_solve():
    """The Schur-complement block solve, run to convergence, is D_B^-1 r block by block
    (dense solves of the assembled D_B); so is plain block MR."""
    D, r = wilson(), field(1107)
    blk = (2, 2, 2, 2)
    want = exact_block_solve(D, DIMS, blk, r, 12)
    assert rel(block_mr_eo(D, DIMS, blk, r, 60), want) < 1e-11
    assert rel(block_mr(D, DIMS, blk, r, 120), want) < 1e-11


def test_even_odd_block_solve_is_exact_on_even_sites_of_site_blocks():
    """Single-site blocks have no interior hops: the even sites get C^-1 r exactly, the
    odd sites MR on C, which converges to C^-1 r."""
    D, r = wilson(), field(1108)
    site = (1, 1, 1, 1)
    exact = np.linalg.solve(D.C, r[..., None])[..., 0]
    ev = (parity(DIMS) == 0)[..., None]
    e1 = block_mr_eo(D, DIMS, site, r, 1)
    assert rel(np.where(ev, e1, 0), np.where(ev, exact, 0)) < 1e-14
    assert rel(block_mr_eo(D, DIMS, site, r, 40), exact) < 1e-12


def test_even_odd_sap_step_beats_plain_block_mr_at_equal_steps():
    """With the same number of MR steps the Schur-complement block solve leaves a smaller
    block residual than MR on D_B (the point of the preconditioning) for these fields."""
    D, r = wilson(), field(1109)
    blk = (2, 2, 2, 2)
    for k in (1, 2, 4):
        res_eo = np.linalg.norm(r - block_interior(D, DIMS, blk, block_mr_eo(D, DIMS, blk, r, k)))
        res_pl = np.linalg.norm(r - block_interior(D, DIMS, blk, block_mr(D, DIMS, blk, r, k)))
        assert res_eo < res_pl, k


def test_even_odd_sap_preconditioned_solve_converges_to_the_dense_solution():
    D = wilson()
    V = int(np.prod(DIMS))
    b = to_grid(inputs.source(DIMS, 0)[0].reshape(V, 12), DIMS)
    iv = [[to_grid(v, DIMS) for v in inputs.setup_vectors(DIMS, 12, 8, 0, 1101)]]
    mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2)], nvecs=[8], smoother="sap", sap_eo=True), iv)
    x, info = mg.solve(b)
    assert info.converged and info.true_residual <= 1e-10
    x_ref, _ = gmres(D, b, restart=60, tol=1e-13, maxiter=5000, verify=True)
    assert rel(x, x_ref) < 1e-8
