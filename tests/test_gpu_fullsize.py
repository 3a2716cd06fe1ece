"""Parity at the benchmark's full size: 16^3x32, eps 0.25, m0 -0.2, csw 1, blocks 4^4
(coarse 4^3x8), Nvec 24 (nbasis 48), 3 + 2 setup sweeps, FP32 inner levels, solve as a
CUDA graph with autotuned coarse launch shapes -- the configuration bench.py times.

The oracle checks what it can afford at this size: whole stencil and coarse-operator
applications, the solve's true residual with the oracle's own D, and sampled
aggregates for the orthonormalisation, the transfers and the Galerkin blocks (each
sample recomputed from the library's near-null vectors and the oracle's D)."""
import numpy as np
import pytest

from oracle.coarse import CoarseOperator, block_index
from oracle.lattice import coarse_dims, face_mask, from_grid, to_grid
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, host, rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DIMS, BLOCK, NVEC = (16, 16, 16, 32), (4, 4, 4, 4), 24
V = int(np.prod(DIMS))
CD = coarse_dims(DIMS, BLOCK)
VC, NB = int(np.prod(CD)), 2 * NVEC


@pytest.fixture(scope="module")
def full(lib):
    p = lib.default_params(dims=DIMS, blocks=[BLOCK], nvec=[NVEC], m0=-0.2, csw=1.0, inner_prec=lib.F32,
                           setup_init_sweeps=3, setup_refine_sweeps=2, max_rhs=24, use_graphs=1, autotune=1)
    ctx = lib.Context(p)
    U = inputs.random_gauge(DIMS, 0.25, 1002)
    ctx.set_gauge(dev(U))
    ctx.setup(dev(inputs.setup_vectors(DIMS, 12, NVEC, 0, 1002)))
    D = WilsonClover(U, DIMS, -0.2, 1.0)
    P = dev(np.zeros((NVEC, V, 12), dtype=complex))
    ctx.get_nullvecs(0, P)
    vecs = host(P)
    A = dev(np.zeros((9, VC, NB, NB), dtype=complex))
    ctx.get_coarse_links(1, A)
    yield dict(ctx=ctx, D=D, vecs=vecs, A=host(A))
    ctx.close()


@pytest.mark.parametrize("prec,tol,nrhs", [(0, 1e-12, 1), (1, 1e-5, 1), (1, 1e-5, 24)])
def test_fullsize_dslash_matches_oracle(lib, full, prec, tol, nrhs):
    psi = inputs.complex_gaussian(61, nrhs, (nrhs, V, 12))
    out = dev(np.zeros_like(psi))
    full["ctx"].apply_D(dev(psi), out, nrhs=nrhs, prec=prec)
    got = host(out)
    check = range(nrhs) if nrhs < 4 else (0, 7, 16, nrhs - 1)  # the 24-rhs launch: sampled rhs
    for r in check:
        f = to_grid(psi[r].reshape(V, 12), DIMS)
        assert rel(got[r].reshape(V, 12), from_grid(full["D"](f))) < tol, r


def block_of(x_c):
    """Fine lexicographic site indices of aggregate x_c = (xc, yc, zc, tc)."""
    xs = [np.arange(BLOCK[k]) + x_c[k] * BLOCK[k] for k in range(4)]
    t, z, y, x = np.meshgrid(xs[3], xs[2], xs[1], xs[0], indexing="ij")
    return (x + DIMS[0] * (y + DIMS[1] * (z + DIMS[2] * t))).ravel()


# 16 sampled aggregates: the corners of the coarse lattice (their hops wrap around the
# periodic boundary in every direction) and seeded interior ones
SAMPLES = [(0, 0, 0, 0), (3, 3, 3, 7), (3, 0, 0, 0), (0, 3, 0, 7), (0, 0, 3, 0), (3, 3, 0, 7), (3, 1, 2, 7),
           (1, 3, 0, 4)] + [tuple(int(v) for v in x) for x in
                            np.random.default_rng(65).integers(0, [4, 4, 4, 8], size=(8, 4))]


def test_fullsize_nullvecs_are_block_orthonormal(full):
    v = full["vecs"]
    for x_c in SAMPLES:
        sites = block_of(x_c)
        for s in range(2):
            M = v[:, sites, 6 * s:6 * s + 6].reshape(NVEC, -1)
            G = M.conj() @ M.T
            assert np.abs(G - np.eye(NVEC)).max() < 1e-12


def test_fullsize_transfers_match_oracle_on_sampled_aggregates(lib, full):
    ctx, v = full["ctx"], full["vecs"]
    f = inputs.complex_gaussian(62, 0, (1, V, 12))
    phi = inputs.complex_gaussian(63, 0, (1, VC, NB))
    for prec, tol in ((0, 1e-12), (1, 1e-5)):
        rc = dev(np.zeros((1, VC, NB), dtype=complex))
        ctx.restrict(0, dev(f), rc, prec=prec)
        pf = dev(np.zeros_like(f))
        ctx.prolong(0, dev(phi), pf, prec=prec)
        rc, pf = host(rc)[0], host(pf)[0]
        for x_c in SAMPLES:
            sites = block_of(x_c)
            lex = x_c[0] + CD[0] * (x_c[1] + CD[1] * (x_c[2] + CD[2] * x_c[3]))
            want = np.concatenate([np.einsum("isc,sc->i", v[:, sites, 6 * s:6 * s + 6].conj(),
                                             f[0][sites, 6 * s:6 * s + 6]) for s in range(2)])
            assert rel(rc[lex], want) < tol
            pw = np.zeros((len(sites), 12), dtype=complex)
            for s in range(2):
                pw[:, 6 * s:6 * s + 6] = np.einsum("isc,i->sc", v[:, sites, 6 * s:6 * s + 6],
                                                   phi[0][lex, s * NVEC:(s + 1) * NVEC])
            assert rel(pf[sites], pw) < tol


def test_fullsize_galerkin_blocks_match_oracle_on_samples(full):
    """A_d(x_c)[:, b] = sum over B(x_c) of <Pi_s v_i, (face-masked D-piece of column b)>,
    recomputed with the oracle's D from the library's near-null vectors, for all nine
    blocks d and all 48 columns b of 16 sampled aggregates (FP32 coarsening: 1e-5,
    element-wise per block)."""
    D, v, A = full["D"], full["vecs"], full["A"]
    faces = {(mu, sign): from_grid(face_mask(DIMS, BLOCK, mu, sign)[..., None].astype(float))[:, 0] > 0
             for mu in range(4) for sign in (+1, -1)}
    sites = [block_of(x_c) for x_c in SAMPLES]
    lexs = [x_c[0] + CD[0] * (x_c[1] + CD[1] * (x_c[2] + CD[2] * x_c[3])) for x_c in SAMPLES]
    want = np.zeros((9, len(SAMPLES), NB, NB), dtype=complex)   # [d][sample][row][column]
    for b in range(NB):
        s_b, i_b = divmod(b, NVEC)
        col = np.zeros((V, 12), dtype=complex)
        col[:, 6 * s_b:6 * s_b + 6] = v[i_b][:, 6 * s_b:6 * s_b + 6]
        Vb = to_grid(col, DIMS)
        pieces = {0: from_grid(D.apply_self(Vb))}
        for mu in range(4):
            for sign in (+1, -1):
                W = from_grid(D.apply_hop(mu, sign, Vb))
                f = faces[(mu, sign)]
                pieces[block_index(mu, sign)] = np.where(f[:, None], W, 0)
                pieces[0] = pieces[0] + np.where(f[:, None], 0, W)
        for k, st in enumerate(sites):
            for d, fld in pieces.items():
                want[d, k, :, b] = np.concatenate([np.einsum("isc,sc->i", v[:, st, 6 * s:6 * s + 6].conj(),
                                                             fld[st, 6 * s:6 * s + 6]) for s in range(2)])
    for k, lex in enumerate(lexs):
        for d in range(9):
            assert rel(A[d, lex], want[d, k]) < 1e-5, (SAMPLES[k], d)


def test_fullsize_coarse_apply_matches_oracle(lib, full):
    A = full["A"]
    op = CoarseOperator(np.stack([to_grid(A[d], CD) for d in range(9)]), CD)
    phi = inputs.complex_gaussian(64, 0, (1, VC, NB))
    out = dev(np.zeros_like(phi))
    full["ctx"].apply_coarse(1, dev(phi), out, nrhs=1, prec=lib.F32)
    assert rel(host(out)[0], from_grid(op(to_grid(phi[0], CD)))) < 1e-5


def test_fullsize_solve_true_residual_by_oracle(lib, full):
    """Three solves (host-driven, capture, replay); the oracle's D recomputes the true
    residual of the returned x."""
    ctx, D = full["ctx"], full["D"]
    b = inputs.source(DIMS, 0)
    for _ in range(3):
        x = dev(np.zeros_like(b))
        st = ctx.solve(dev(b), x)
    assert st.graph == 1 and st.converged
    r = b[0].reshape(V, 12) - from_grid(D(to_grid(host(x)[0].reshape(V, 12), DIMS)))
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1e-10
    assert st.outer_iterations <= 40
