"""GPU parity of the operators through the C-ABI against the FP64 oracle.

Tolerances: 1e-12 relative for FP64 kernels, 1e-5 relative for FP32 kernels
(both stated by the task's acceptance bar); BF16/FP16 coarse links are
error-stated against FP64 (unit roundoff 2^-8 / 2^-11 of the link entries).
Lattices are chosen to span several CTAs with a ragged last tile and
anisotropic extents/blocks so that a mixed-up axis fails."""
import numpy as np
import pytest

from oracle.aggregation import Aggregation, block_orthonormalise
from oracle.coarse import CoarseOperator, coarsen
from oracle.lattice import coarse_dims, to_grid
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, ext, fields, host, rel, rel_norm

pytestmark = pytest.mark.gpu

CASES = [  # dims, block, nvec
    ((4, 4, 4, 4), (2, 2, 2, 2), 8),
    ((6, 4, 8, 10), (3, 2, 4, 5), 5),   # V = 1920: 15 CTAs of 128, odd nvec, anisotropic blocks
    ((8, 8, 8, 8), (4, 4, 2, 2), 4),
]


def make(lib, dims, block, nvec, prec=None, link_prec=None, max_rhs=4, nlev=2, blocks=None, **kw):
    p = lib.default_params(dims=dims, blocks=blocks or [block], nvec=[nvec] * 3, m0=-0.17, csw=1.13,
                           max_rhs=max_rhs, n_levels=nlev, **kw)
    if prec is not None:
        p.inner_prec = prec
    if link_prec is not None:
        p.coarse_link_prec = link_prec
    return lib.Context(p)


@pytest.mark.parametrize("dims,block,nvec", CASES)
def test_clover_matches_oracle(lib, dims, block, nvec):
    U = inputs.random_gauge(dims, 0.35, 2001)
    ctx = make(lib, dims, block, nvec)
    ctx.set_gauge(dev(U))
    V = int(np.prod(dims))
    C = dev(np.zeros((V, 12, 12), dtype=complex))
    ctx.get_clover(C)
    D = WilsonClover(U, dims, -0.17, 1.13)
    assert rel(host(C), D.C.reshape(V, 12, 12)) < 1e-13


@pytest.mark.parametrize("dims,block,nvec", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_dslash_matches_oracle(lib, dims, block, nvec, prec, tol):
    U = inputs.random_gauge(dims, 0.35, 2002)
    ctx = make(lib, dims, block, nvec)
    ctx.set_gauge(dev(U))
    V = int(np.prod(dims))
    D = WilsonClover(U, dims, -0.17, 1.13)
    # 1 rhs, an even count and an odd count (FP32 runs two rhs per thread: a short last pair)
    for nrhs in (1, 2, 3):
        psi = inputs.complex_gaussian(7, nrhs, (nrhs, V, 4, 3))
        out = dev(np.zeros_like(psi))
        ctx.apply_D(dev(psi), out, nrhs=nrhs, prec=prec)
        ref = np.stack([D(f).reshape(V, 4, 3) for f in fields(psi, dims, 12)])
        got = host(out)
        for r in range(nrhs):
            assert rel(got[r], ref[r]) < tol, (nrhs, r)


def test_dslash_host_buffers_match_device_buffers(lib):
    dims, block, nvec = CASES[1]
    U = inputs.random_gauge(dims, 0.35, 2003)
    ctx = make(lib, dims, block, nvec)
    ctx.set_gauge(U)  # host pointer path
    V = int(np.prod(dims))
    psi = inputs.complex_gaussian(7, 2, (1, V, 4, 3))
    out_h = np.zeros_like(psi)
    ctx.apply_D(psi, out_h)
    out_d = dev(np.zeros_like(psi))
    ctx.apply_D(dev(psi), out_d)
    assert np.array_equal(out_h, host(out_d))


@pytest.mark.parametrize("ortho_df", [0, 1], ids=["fp64", "double_float"])
@pytest.mark.parametrize("dims,block,nvec", CASES + [((8, 8, 8, 8), (4, 4, 4, 4), 24), ((8, 8, 8, 8), (4, 4, 4, 4), 7)])
def test_block_orthonormalisation_matches_oracle(lib, dims, block, nvec, ortho_df):
    """The three lattices of CASES, and the workloads' 4^4 aggregates (panels of 1536 rows:
    the double-float kernel takes its columns in pairs there; 7 columns leave the last one
    alone)."""
    V = int(np.prod(dims))
    raw = inputs.complex_gaussian(11, 3, (nvec, V, 12))
    ctx = make(lib, dims, block, nvec, ortho_df=ortho_df)
    ctx.set_nullvecs(0, dev(raw))
    got = dev(np.zeros_like(raw))
    ctx.get_nullvecs(0, got)
    ref = block_orthonormalise(fields(raw, dims, 12), block)
    assert rel(host(got), ref.reshape(nvec, V, 12)) < 1e-12


@pytest.mark.parametrize("dims,block,nvec", [CASES[0], CASES[1], ((8, 8, 8, 8), (4, 4, 4, 4), 24)],
                         ids=["one_column", "pairs_small", "pairs_4x4x4x4"])
def test_fp32_setup_orthonormalises_fp32_vectors_in_double_float(lib, dims, block, nvec):
    """FP32 inner levels with the double-float orthonormalisation: the setup's kernel reads
    the FP32 near-null vectors and writes P in FP64 and its FP32 copy in one pass.  With no
    setup sweeps the vectors are the given ones rounded to FP32, so P must be the oracle's
    block orthonormalisation of those rounded vectors to 1e-12, and the FP32 restriction,
    which reads the FP32 copy of P, the oracle's restriction to FP32 accuracy."""
    V = int(np.prod(dims))
    cd = coarse_dims(dims, block)
    Vc = int(np.prod(cd))
    iv = inputs.complex_gaussian(13, 3, (nvec, V, 12))
    iv32 = iv.astype(np.complex64).astype(np.complex128)
    ctx = make(lib, dims, block, nvec, prec=lib.F32, ortho_df=1, setup_init_sweeps=0, setup_refine_sweeps=0)
    ctx.set_gauge(dev(inputs.random_gauge(dims, 0.35, 2005)))
    ctx.setup(dev(iv))
    got = dev(np.zeros_like(iv))
    ctx.get_nullvecs(0, got)
    ref = block_orthonormalise(fields(iv32, dims, 12), block)
    assert rel(host(got), ref.reshape(nvec, V, 12)) < 1e-12
    agg = Aggregation(dims, block, fields(iv32, dims, 12))
    psi = inputs.complex_gaussian(13, 4, (3, V, 12))
    out = dev(np.zeros((3, Vc, 2 * nvec), dtype=complex))
    ctx.restrict(0, dev(psi), out, nrhs=3, prec=lib.F32)
    o = host(out)
    for r, f in enumerate(fields(psi, dims, 12)):
        assert rel(o[r], agg.restrict(f).reshape(Vc, -1)) < 1e-5


@pytest.mark.parametrize("dims,block,nvec", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_restrict_prolong_match_oracle(lib, dims, block, nvec, prec, tol):
    V = int(np.prod(dims))
    cd = coarse_dims(dims, block)
    Vc = int(np.prod(cd))
    raw = inputs.complex_gaussian(12, 3, (nvec, V, 12))
    ctx = make(lib, dims, block, nvec)
    ctx.set_nullvecs(0, dev(raw))
    agg = Aggregation(dims, block, fields(raw, dims, 12))
    nrhs = 4 if prec == 1 else 2
    psi = inputs.complex_gaussian(12, 4, (nrhs, V, 12))
    out = dev(np.zeros((nrhs, Vc, 2 * nvec), dtype=complex))
    ctx.restrict(0, dev(psi), out, nrhs=nrhs, prec=prec)
    got = host(out)
    for r, f in enumerate(fields(psi, dims, 12)):
        assert rel(got[r], agg.restrict(f).reshape(Vc, -1)) < tol
    phi = inputs.complex_gaussian(12, 5, (nrhs, Vc, 2 * nvec))
    outf = dev(np.zeros((nrhs, V, 12), dtype=complex))
    ctx.prolong(0, dev(phi), outf, nrhs=nrhs, prec=prec)
    gotf = host(outf)
    for r, f in enumerate(fields(phi, cd, 2 * nvec)):
        assert rel(gotf[r], agg.prolong(f).reshape(V, 12)) < tol


def random_links(seed, Vc, nb):
    A = inputs.complex_gaussian(seed, 9, (9, Vc, nb, nb))
    A[0] += 6.0 * np.eye(nb)
    return A


@pytest.mark.parametrize("dims,block,nvec", CASES)
@pytest.mark.parametrize("prec,lp,tol", [(0, 0, 1e-12), (1, 1, 1e-5), (1, 2, 5e-3), (1, 3, 1e-3)])
def test_coarse_apply_matches_oracle(lib, dims, block, nvec, prec, lp, tol):
    cd = coarse_dims(dims, block)
    Vc = int(np.prod(cd))
    nb = 2 * nvec
    A = random_links(13, Vc, nb)
    ctx = make(lib, dims, block, nvec, prec=prec, link_prec=lp if lp else None)
    ctx.set_coarse_links(1, dev(A))
    op = CoarseOperator(np.stack([to_grid(A[d], cd) for d in range(9)]), cd)
    for nrhs in (1, 4):
        phi = inputs.complex_gaussian(14, nrhs, (nrhs, Vc, nb))
        out = dev(np.zeros_like(phi))
        ctx.apply_coarse(1, dev(phi), out, nrhs=nrhs, prec=prec)
        got = host(out)
        for r, f in enumerate(fields(phi, cd, nb)):
            assert rel(got[r], op(f).reshape(Vc, nb)) < tol
    # links round trip
    back = dev(np.zeros_like(A))
    ctx.get_coarse_links(1, back)
    assert rel(host(back), A) < (1e-15 if prec == 0 else tol)


@pytest.mark.parametrize("dims,block,nvec", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_coarsen_matches_oracle(lib, dims, block, nvec, prec, tol):
    U = inputs.random_gauge(dims, 0.35, 2004)
    V = int(np.prod(dims))
    cd = coarse_dims(dims, block)
    raw = inputs.complex_gaussian(15, 3, (nvec, V, 12))
    ctx = make(lib, dims, block, nvec, prec=prec)
    ctx.set_gauge(dev(U))
    ctx.set_nullvecs(0, dev(raw))
    ctx.coarsen(0)
    nb = 2 * nvec
    A = dev(np.zeros((9, int(np.prod(cd)), nb, nb), dtype=complex))
    ctx.get_coarse_links(1, A)
    D = WilsonClover(U, dims, -0.17, 1.13)
    ref = coarsen(D, Aggregation(dims, block, fields(raw, dims, 12))).A.reshape(9, -1, nb, nb)
    assert rel(host(A), ref) < tol


def test_coarsen_second_level_matches_oracle(lib):
    dims, b0, b1, nv = (8, 8, 4, 8), (2, 2, 2, 2), (2, 2, 1, 2), (4, 3)
    U = inputs.random_gauge(dims, 0.35, 2005)
    V = int(np.prod(dims))
    cd1 = coarse_dims(dims, b0)
    cd2 = coarse_dims(cd1, b1)
    V1 = int(np.prod(cd1))
    p = lib.default_params(dims=dims, blocks=[b0, b1], nvec=list(nv), n_levels=3, m0=-0.17, csw=1.13, max_rhs=4)
    ctx = lib.Context(p)
    ctx.set_gauge(dev(U))
    raw0 = inputs.complex_gaussian(16, 3, (nv[0], V, 12))
    raw1 = inputs.complex_gaussian(16, 4, (nv[1], V1, 2 * nv[0]))
    ctx.set_nullvecs(0, dev(raw0))
    ctx.coarsen(0)
    ctx.set_nullvecs(1, dev(raw1))
    ctx.coarsen(1)
    nb2 = 2 * nv[1]
    A2 = dev(np.zeros((9, int(np.prod(cd2)), nb2, nb2), dtype=complex))
    ctx.get_coarse_links(2, A2)
    D = WilsonClover(U, dims, -0.17, 1.13)
    D1 = coarsen(D, Aggregation(dims, b0, fields(raw0, dims, 12)))
    D2 = coarsen(D1, Aggregation(cd1, b1, fields(raw1, cd1, 2 * nv[0])))
    assert rel(host(A2), D2.A.reshape(9, -1, nb2, nb2)) < 1e-12


def test_tensor_core_coarse_apply_exact_on_bf16_representable_data(lib):
    """Multi-rhs coarse apply on tcgen05 (BF16 operands, FP32 accumulation): with
    small-integer links and vectors every product and partial sum is exact, so the
    result must equal the FP64 oracle exactly."""
    dims, block, nvec = (8, 8, 8, 8), (2, 2, 2, 2), 24
    cd = coarse_dims(dims, block)
    Vc, nb = int(np.prod(cd)), 2 * nvec
    rng = np.random.default_rng(71)
    A = (rng.integers(-3, 4, size=(9, Vc, nb, nb)) + 1j * rng.integers(-3, 4, size=(9, Vc, nb, nb))).astype(complex)
    p = lib.default_params(dims=dims, blocks=[block], nvec=[nvec], max_rhs=70, inner_prec=lib.F32,
                           coarse_link_prec=lib.BF16)
    ctx = lib.Context(p)
    ctx.set_coarse_links(1, dev(A))
    op = CoarseOperator(np.stack([to_grid(A[d], cd) for d in range(9)]), cd)
    for nrhs in (8, 16, 37, 70):
        phi = (rng.integers(-2, 3, size=(nrhs, Vc, nb)) + 1j * rng.integers(-2, 3, size=(nrhs, Vc, nb))).astype(complex)
        out = dev(np.zeros_like(phi))
        ctx.apply_coarse(1, dev(phi), out, nrhs=nrhs, prec=lib.F32)
        got = host(out)
        for r, f in enumerate(fields(phi, cd, nb)):
            assert np.array_equal(got[r], op(f).reshape(Vc, nb)), (nrhs, r)


@pytest.mark.parametrize("nvec", [8, 24, 32])
def test_tensor_core_coarse_apply_matches_oracle(lib, nvec):
    """Random data: BF16 rounding of links and vectors (unit roundoff 2^-8 each) bounds the
    error.  Rounding errors of random sign make it about 2^-8 / sqrt(3) per operand,
    ~2e-3 of the result's 2-norm (bar 5e-3).  Element-wise, relative to the largest entry of
    each output field, the worst of 4096 x 16 entries is ~6e-3 at nbasis 16 (bar 1.2e-2)."""
    dims, block = (8, 8, 8, 8), (2, 2, 2, 2)
    cd = coarse_dims(dims, block)
    Vc, nb = int(np.prod(cd)), 2 * nvec
    A = random_links(72, Vc, nb)
    p = lib.default_params(dims=dims, blocks=[block], nvec=[nvec], max_rhs=20, inner_prec=lib.F32,
                           coarse_link_prec=lib.BF16)
    ctx = lib.Context(p)
    ctx.set_coarse_links(1, dev(A))
    op = CoarseOperator(np.stack([to_grid(A[d], cd) for d in range(9)]), cd)
    phi = inputs.complex_gaussian(73, 0, (20, Vc, nb))
    out = dev(np.zeros_like(phi))
    ctx.apply_coarse(1, dev(phi), out, nrhs=20, prec=lib.F32)
    got = host(out)
    for r, f in enumerate(fields(phi, cd, nb)):
        want = op(f).reshape(Vc, nb)
        assert rel_norm(got[r], want) < 5e-3 and rel(got[r], want) < 1.2e-2


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
@pytest.mark.parametrize("nrhs", [16, 40])
def test_restrict_many_rhs_matches_oracle(lib, prec, tol, nrhs):
    """Register-blocked GEMM path of the restriction (>= 16 rhs: setup batches, coarsening)."""
    dims, block, nvec = (8, 4, 4, 8), (4, 2, 2, 4), 12
    V = int(np.prod(dims))
    cd = coarse_dims(dims, block)
    Vc = int(np.prod(cd))
    raw = inputs.complex_gaussian(81, 3, (nvec, V, 12))
    ctx = make(lib, dims, block, nvec, max_rhs=nrhs)
    ctx.set_nullvecs(0, dev(raw))
    agg = Aggregation(dims, block, fields(raw, dims, 12))
    psi = inputs.complex_gaussian(82, 4, (nrhs, V, 12))
    out = dev(np.zeros((nrhs, Vc, 2 * nvec), dtype=complex))
    ctx.restrict(0, dev(psi), out, nrhs=nrhs, prec=prec)
    got = host(out)
    for r, f in enumerate(fields(psi, dims, 12)):
        assert rel(got[r], agg.restrict(f).reshape(Vc, -1)) < tol


@pytest.mark.parametrize("ortho_df", [0, 1], ids=["fp64", "double_float"])
@pytest.mark.parametrize("dims,block,nvec", [((8, 8, 4, 4), (4, 4, 2, 2), 16), ((8, 8, 8, 8), (4, 4, 4, 4), 16)],
                         ids=["agg64", "agg256"])
def test_block_orthonormalisation_ill_conditioned_panels(lib, ortho_df, dims, block, nvec):
    """Nearly parallel near-null candidates (condition number ~1e3 per aggregate) make
    the second Gram-Schmidt pass necessary; Q must stay orthonormal and equal to the
    positive-diagonal QR factor within the conditioning (FP64 and double-float; on 4^4
    aggregates the double-float kernel's paired columns take their second passes too)."""
    V = int(np.prod(dims))
    base = inputs.complex_gaussian(91, 0, (1, V, 12))
    raw = base + 1e-3 * inputs.complex_gaussian(91, 1, (nvec, V, 12))
    ctx = make(lib, dims, block, nvec, ortho_df=ortho_df)
    ctx.set_nullvecs(0, dev(raw))
    got = dev(np.zeros_like(raw))
    ctx.get_nullvecs(0, got)
    ref = block_orthonormalise(fields(raw, dims, 12), block)
    assert rel(host(got), ref.reshape(nvec, V, 12)) < 1e-9
    agg_g = Aggregation(dims, block, fields(host(got), dims, 12), orthonormalise=False)
    cd = coarse_dims(dims, block)
    phi = to_grid(inputs.complex_gaussian(92, 0, (int(np.prod(cd)), 2 * nvec)), cd)
    assert rel(agg_g.restrict(agg_g.prolong(phi)), phi) < 1e-13  # P^dag P = 1
