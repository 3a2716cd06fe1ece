"""The five-block coarse apply (params.coarse_sigma3, launch kind 5) against the FP64
oracle.

The hop blocks of a Galerkin operator D_c = P^dag D P obey
A_{-mu}(x) = sigma3 A_{+mu}(x - mu)^dag sigma3 (gamma5-hermiticity of D with
gamma5 P = P sigma3, Sec. 2.2; pinned block by block on the oracle in
tests/test_oracle_coarse.py), so the kernel that reads only A_0 and the four
forward blocks (Sec. 4: five stencil points) must reproduce the oracle's nine-point
apply.  Tolerances as for the nine-block kernels: 1e-12 (FP64), 1e-5 (FP32), and the
BF16 / FP16 link bars of test_gpu_operators.py.  The lattices include a coarse
extent of 2, where the +mu and -mu neighbours of a site coincide and only the
face-keyed split tells the two hops apart."""
import numpy as np
import pytest

from oracle.aggregation import Aggregation
from oracle.coarse import coarsen
from oracle.lattice import coarse_dims
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, fields, host, rel

pytestmark = pytest.mark.gpu

CASES = [  # dims, block, nvec
    ((4, 4, 4, 4), (2, 2, 2, 2), 8),
    ((6, 4, 8, 10), (3, 2, 4, 5), 5),    # coarse 2^4: +mu and -mu neighbours coincide
    ((8, 8, 8, 8), (2, 2, 2, 2), 24),    # nbasis 48: the headline's level-1 block size
]


def galerkin_ctx(lib, dims, block, nvec, prec, link_prec=None, seed=2101):
    p = lib.default_params(dims=dims, blocks=[block], nvec=[nvec] * 3, m0=-0.17, csw=1.13, max_rhs=4, n_levels=2,
                           coarse_sigma3=1)
    p.inner_prec = prec
    if link_prec is not None:
        p.coarse_link_prec = link_prec
    ctx = lib.Context(p)
    U = inputs.random_gauge(dims, 0.35, seed)
    V = int(np.prod(dims))
    raw = inputs.complex_gaussian(seed, 3, (nvec, V, 12))
    ctx.set_gauge(dev(U))
    ctx.set_nullvecs(0, dev(raw))
    ctx.coarsen(0)
    op = coarsen(WilsonClover(U, dims, -0.17, 1.13), Aggregation(dims, block, fields(raw, dims, 12)))
    return ctx, op


def apply_kind5(lib, ctx, dims, block, nvec, prec, op, seed, **tile):
    cd = coarse_dims(dims, block)
    Vc, nb = int(np.prod(cd)), 2 * nvec
    pr = lib.F64 if prec == lib.F64 else lib.F32
    ctx.set_coarse_tile(1, 1, pr, kind=5, **tile)
    assert ctx.get_coarse_tile(1, 1, pr)["kind"] == 5
    phi = inputs.complex_gaussian(seed, 1, (1, Vc, nb))
    out = dev(np.zeros_like(phi))
    ctx.apply_coarse(1, dev(phi), out, nrhs=1, prec=pr)
    ref = op(fields(phi, cd, nb)[0]).reshape(Vc, nb)
    return rel(host(out)[0], ref)


@pytest.mark.parametrize("dims,block,nvec", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_five_block_apply_matches_oracle(lib, dims, block, nvec, prec, tol):
    ctx, op = galerkin_ctx(lib, dims, block, nvec, prec)
    assert apply_kind5(lib, ctx, dims, block, nvec, prec, op, 2102, threads=256, parts=1, stages=1) < tol


@pytest.mark.parametrize("threads,stages", [(512, 2), (256, 1), (128, 2), (64, 1)])
def test_five_block_launch_shapes(lib, threads, stages):
    """Two rows in flight per warp, and from 42 down to 2 row groups sharing the backward
    blocks (64 threads: 2 groups of 24 FP32 chunks per 48-entry row)."""
    dims, block, nvec = (8, 8, 8, 8), (2, 2, 2, 2), 24
    ctx, op = galerkin_ctx(lib, dims, block, nvec, 1, seed=2103)
    assert apply_kind5(lib, ctx, dims, block, nvec, 1, op, 2104, threads=threads, parts=1, stages=stages) < 1e-5


@pytest.mark.parametrize("lp,tol", [(2, 5e-3), (3, 1e-3)], ids=["bf16", "fp16"])
@pytest.mark.parametrize("dims,block,nvec", [((8, 8, 8, 8), (2, 2, 2, 2), 24), ((6, 4, 8, 10), (3, 2, 4, 5), 5)],
                         ids=["nbasis48", "nbasis10"])
def test_five_block_low_precision_links(lib, lp, tol, dims, block, nvec):
    """BF16 / FP16 link storage: the five-block copy is taken from the rounded nine-block
    links, so the error is that of the rounding (unit roundoff 2^-8 / 2^-11 of the
    entries) against the FP64 oracle.  nbasis 10 is not a whole number of 16-byte link
    chunks, so the backward blocks are read column by column there."""
    ctx, op = galerkin_ctx(lib, dims, block, nvec, 1, link_prec=lp, seed=2105)
    assert apply_kind5(lib, ctx, dims, block, nvec, 1, op, 2106, threads=256, parts=1, stages=2) < tol


def test_five_block_needs_a_galerkin_operator(lib):
    """Links given by the caller carry no symmetry: kind 5 is refused for them."""
    dims, block, nvec = (4, 4, 4, 4), (2, 2, 2, 2), 4
    ctx, _ = galerkin_ctx(lib, dims, block, nvec, 1)
    cd = coarse_dims(dims, block)
    Vc, nb = int(np.prod(cd)), 2 * nvec
    A = inputs.complex_gaussian(2107, 9, (9, Vc, nb, nb))
    with pytest.raises(lib.WcmgError):  # one CTA per site only
        ctx.set_coarse_tile(1, 1, lib.F32, kind=5, threads=256, parts=2, stages=1)
    ctx.set_coarse_links(1, dev(A))
    with pytest.raises(lib.WcmgError):
        ctx.set_coarse_tile(1, 1, lib.F32, kind=5, threads=256, parts=1, stages=1)
    # without params.coarse_sigma3 there is no five-block copy either
    p = lib.default_params(dims=dims, blocks=[block], nvec=[nvec] * 3, m0=-0.17, csw=1.13, max_rhs=4, n_levels=2)
    c2 = lib.Context(p)
    c2.set_gauge(dev(inputs.random_gauge(dims, 0.35, 2108)))
    c2.set_nullvecs(0, dev(inputs.complex_gaussian(2108, 3, (nvec, int(np.prod(dims)), 12))))
    c2.coarsen(0)
    with pytest.raises(lib.WcmgError):
        c2.set_coarse_tile(1, 1, lib.F32, kind=5, threads=256, parts=1, stages=1)


def test_solve_with_five_block_coarse_applies(lib):
    """A two-level FP32-inner solve whose one-rhs coarse applies all use kind 5 reaches
    the 1e-10 true residual (checked with the oracle's D) in the iterations of the
    nine-block solve, give or take one."""
    dims, block, nvec = (8, 8, 8, 8), (4, 4, 4, 4), 8
    V = int(np.prod(dims))
    U = inputs.random_gauge(dims, 0.3, 2109)
    b = inputs.source(dims, 5, nrhs=1)
    its = {}
    for s3 in (0, 1):
        p = lib.default_params(dims=dims, blocks=[block], nvec=[nvec], m0=-0.1, csw=1.0, max_rhs=1, n_levels=2,
                               coarse_sigma3=s3, autotune=0)
        p.inner_prec = lib.F32
        ctx = lib.Context(p)
        ctx.set_gauge(dev(U))
        ctx.setup_seeded(2109)
        if s3:
            ctx.set_coarse_tile(1, 1, lib.F32, kind=5, threads=256, parts=1, stages=1)
        x = dev(np.zeros_like(b))
        st = ctx.solve(dev(b), x)
        D = WilsonClover(U, dims, -0.1, 1.0)
        xg = fields(host(x), dims, 12)[0]
        r = np.linalg.norm((fields(b, dims, 12)[0] - D(xg)).ravel()) / np.linalg.norm(b.ravel())
        assert r < 1e-10
        its[s3] = st.outer_iterations
    assert abs(its[1] - its[0]) <= 1
