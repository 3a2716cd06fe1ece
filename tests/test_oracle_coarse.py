"""Pins of the Galerkin coarse operator (Sec. 2.1 CoarsenOperator / Mdiag / Mdir;
Sec. 2.2 sigma3-hermiticity; Sec. 4: 9 stencil points).

The nine-block operator is compared with P^dag D P assembled by brute force from
dense matrices: D column by column (D is pinned in test_oracle_wilson.py) and P
column by column through prolongation (pinned in test_oracle_aggregation.py)."""
import numpy as np
import pytest

from oracle.aggregation import Aggregation
from oracle.coarse import coarsen, block_index
from oracle.lattice import to_grid
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.helpers import rel


def dense(op, dims, nc):
    V = int(np.prod(dims))
    n = V * nc
    M = np.zeros((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex); e[j] = 1
        M[:, j] = op(to_grid(e.reshape(V, nc), dims)).ravel()
    return M


def dense_P(agg):
    Vc = int(np.prod(agg.cdims))
    n = Vc * agg.nbasis
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex); e[j] = 1
        cols.append(agg.prolong(to_grid(e.reshape(Vc, agg.nbasis), agg.cdims)).ravel())
    return np.array(cols).T


def setup_two_level(dims, block, nvec, seed=31, eps=0.4):
    U = inputs.random_gauge(dims, eps, seed)
    D = WilsonClover(U, dims, -0.15, 1.0)
    V = int(np.prod(dims))
    vecs = [to_grid(v, dims) for v in inputs.complex_gaussian(seed, 1, (nvec, V, 12))]
    agg = Aggregation(dims, block, vecs)
    return U, D, agg, vecs


@pytest.mark.parametrize("dims,block", [((4, 4, 2, 4), (2, 2, 1, 2)), ((2, 4, 4, 6), (1, 2, 2, 2))])
def test_galerkin_identity(dims, block):
    U, D, agg, _ = setup_two_level(dims, block, nvec=3)
    Dc = coarsen(D, agg)
    P = dense_P(agg)
    ref = P.conj().T @ dense(D, dims, 12) @ P
    got = dense(Dc, agg.cdims, agg.nbasis)
    assert rel(got, ref) < 1e-13


def test_galerkin_identity_second_level():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, D, agg, _ = setup_two_level(dims, block, nvec=2)
    Dc = coarsen(D, agg)
    Vc = int(np.prod(agg.cdims))
    w = [to_grid(v, agg.cdims) for v in inputs.complex_gaussian(32, 2, (2, Vc, agg.nbasis))]
    agg2 = Aggregation(agg.cdims, (1, 2, 1, 1), w)
    Dc2 = coarsen(Dc, agg2)
    P2 = dense_P(agg2)
    ref = P2.conj().T @ dense(Dc, agg.cdims, agg.nbasis) @ P2
    assert rel(dense(Dc2, agg2.cdims, agg2.nbasis), ref) < 1e-13


def test_sigma3_hermiticity_blockwise():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, D, agg, _ = setup_two_level(dims, block, nvec=4)
    Dc = coarsen(D, agg)
    nv = agg.nvec
    s3 = np.diag(np.concatenate([np.ones(nv), -np.ones(nv)]))
    A = Dc.A
    dag = lambda a: np.conj(np.swapaxes(a, -1, -2))
    assert np.abs(s3 @ A[0] @ s3 - dag(A[0])).max() < 1e-14 * np.abs(A[0]).max()
    for mu in range(4):
        fwd = A[block_index(mu, +1)]
        bwd = A[block_index(mu, -1)]
        fwd_from_minus = np.roll(fwd, 1, axis=3 - mu)  # A_{+mu}(x_c - mu)
        assert np.abs(bwd - s3 @ dag(fwd_from_minus) @ s3).max() < 1e-14 * np.abs(fwd).max()


def test_coarse_operator_gauge_invariant():
    dims, block = (4, 4, 2, 4), (2, 2, 2, 2)
    U, D, agg, vecs = setup_two_level(dims, block, nvec=3)
    Om = inputs.random_gauge_transform(dims, seed=33)
    Omg = to_grid(Om, dims)
    V = Om.shape[0]
    Up = np.empty_like(U)
    for mu in range(4):
        Ug = to_grid(U[mu], dims)
        Up[mu] = (Omg @ Ug @ np.conj(np.swapaxes(np.roll(Omg, -1, axis=3 - mu), -1, -2))).reshape(V, 3, 3)
    rot = lambda f: np.einsum("...ab,...sb->...sa", Omg, f.reshape(f.shape[:4] + (4, 3))).reshape(f.shape)
    Dp = WilsonClover(Up, dims, -0.15, 1.0)
    aggp = Aggregation(dims, block, [rot(v) for v in vecs])
    assert rel(coarsen(Dp, aggp).A, coarsen(D, agg).A) < 1e-13


def test_free_field_constant_vectors_translation_invariant():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    D = WilsonClover(inputs.unit_gauge(dims), dims, 0.1, 1.0)
    V = int(np.prod(dims))
    rng = np.random.default_rng(0)
    vecs = [np.broadcast_to(rng.normal(size=12) + 1j * rng.normal(size=12), (4, 4, 4, 4, 12)).copy() for _ in range(2)]
    Dc = coarsen(D, Aggregation(dims, block, vecs))
    A = Dc.A.reshape(9, -1, 4, 4)
    assert np.abs(A - A[:, :1]).max() < 1e-14


def test_block_storage_convention():
    """Storage index 1 + 2 mu multiplies phi(x_c + mu), 2 + 2 mu multiplies phi(x_c - mu):
    checked by applying D_c to a delta function and reading A by raw index."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, D, agg, _ = setup_two_level(dims, block, nvec=2)
    Dc = coarsen(D, agg)
    nb = agg.nbasis
    y = (1, 0, 1, 0)  # (t, z, y, x) of the delta
    for col in (0, nb - 1):
        phi = np.zeros(agg.cdims[::-1] + (nb,), dtype=complex)
        phi[y + (col,)] = 1.0
        out = Dc(phi)
        for mu in range(4):
            ax = 3 - mu
            minus = list(y); minus[ax] = (y[ax] - 1) % 2
            plus = list(y); plus[ax] = (y[ax] + 1) % 2
            # coarse extent 2: x_c = y - mu and y + mu coincide; the output there is A[1+2mu] + A[2+2mu]
            got = out[tuple(minus)]
            exp = Dc.A[1 + 2 * mu][tuple(minus)][:, col] + Dc.A[2 + 2 * mu][tuple(plus)][:, col]
            assert np.abs(got - exp).max() < 1e-13
    # on a coarse extent 4 direction the two are distinguishable
    dims2, block2 = (8, 4, 4, 4), (2, 2, 2, 2)
    U2, D2, agg2, _ = setup_two_level(dims2, block2, nvec=2)
    Dc2 = coarsen(D2, agg2)
    phi = np.zeros(agg2.cdims[::-1] + (agg2.nbasis,), dtype=complex)
    phi[0, 0, 0, 2, 1] = 1.0
    out = Dc2(phi)
    assert np.abs(out[0, 0, 0, 1] - Dc2.A[1][0, 0, 0, 1][:, 1]).max() < 1e-14   # x_c = 1 reads +x at 2
    assert np.abs(out[0, 0, 0, 3] - Dc2.A[2][0, 0, 0, 3][:, 1]).max() < 1e-14   # x_c = 3 reads -x at 2


def _coarse_system(dims=(4, 4, 4, 8), block=(2, 2, 2, 2), nvec=3):
    U, D, agg, _ = setup_two_level(dims, block, nvec=nvec)
    Dc = coarsen(D, agg)
    Vc = int(np.prod(agg.cdims))
    b = to_grid(inputs.complex_gaussian(33, 0, (Vc, agg.nbasis)), agg.cdims)
    return Dc, agg, b


def test_even_odd_coarsest_solve_is_the_dense_solution():
    """Sec. 4 red-black preconditioning on the coarsest level: run to convergence, the
    Schur-complement solve (b^_o, GMRES on S, back substitution on the even sites) is the
    solution of the dense coarse system.  A flipped sign in b^_o, a dropped A_oe A_ee^-1 A_eo
    term in S or a dropped A_eo x_o in the back substitution each miss it by O(1)."""
    from oracle.mg import coarse_eo_solve
    Dc, agg, b = _coarse_system()
    M = dense(Dc, agg.cdims, agg.nbasis)
    want = np.linalg.solve(M, b.ravel()).reshape(b.shape)
    got = coarse_eo_solve(Dc, agg.cdims, b, restart=80, tol=1e-14, maxiter=2000)
    assert rel(got, want) < 1e-10


def test_even_odd_schur_complement_matches_the_dense_one():
    """The odd-site Schur complement of the nine-block operator equals
    D_oo - D_oe D_ee^-1 D_eo of the dense coarse matrix split by site parity."""
    from oracle.mg import coarse_eo_solve  # noqa: F401  (the reading under test)
    from oracle.sap import parity, self_solve
    Dc, agg, b = _coarse_system()
    cd, nb = agg.cdims, agg.nbasis
    M = dense(Dc, cd, nb)
    par = np.repeat(parity(cd).reshape(-1), nb)  # parity of every dense index
    e, o = np.where(par == 0)[0], np.where(par == 1)[0]
    S = M[np.ix_(o, o)] - M[np.ix_(o, e)] @ np.linalg.solve(M[np.ix_(e, e)], M[np.ix_(e, o)])
    ev = (parity(cd) == 0)[..., None]
    v = np.where(ev, 0, b)
    Dv = Dc(v)
    Sv = np.where(ev, 0, Dv - Dc(np.where(ev, self_solve(Dc, np.where(ev, Dv, 0)), 0)))
    assert rel(Sv.ravel()[o], S @ v.ravel()[o]) < 1e-12
    assert np.abs(Sv.ravel()[e]).max() == 0.0


def test_even_odd_coarsest_solve_needs_even_extents():
    from oracle.mg import coarse_eo_solve
    Dc, agg, b = _coarse_system(dims=(4, 4, 4, 6), block=(2, 2, 2, 2))  # coarse t extent 3
    with pytest.raises(ValueError):
        coarse_eo_solve(Dc, agg.cdims, b, restart=10, tol=1e-6, maxiter=10)
