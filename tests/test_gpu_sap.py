"""GPU parity of the SAP smoother (Sec. 4; oracle/sap.py): two colour passes over the
level's aggregates, block-local MR on D_B with one step length per block.  The smoother
alone on the fine and on a coarse level, and inside the setup, the cycle, the solve and
a graph replay, against the FP64 oracle."""
import numpy as np
import pytest

from oracle.coarse import CoarseOperator
from oracle.lattice import coarse_dims, to_grid
from oracle.mg import MGParams, Multigrid
from oracle.sap import sap
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, fields, host, rel

pytestmark = pytest.mark.gpu


def fine_ctx(lib, dims, block, nvec, prec=0, seed=1201, **kw):
    p = lib.default_params(dims=dims, blocks=[block], nvec=[nvec], m0=-0.1, csw=1.0, inner_prec=prec,
                           smoother=lib.SMOOTHER_SAP, **kw)
    ctx = lib.Context(p)
    U = inputs.random_gauge(dims, 0.3, seed)
    ctx.set_gauge(dev(U))
    return ctx, WilsonClover(U, dims, -0.1, 1.0)


# (dims, block, steps, cycles): the (6,4,4,4) lattice has an odd number of aggregates
# along x, so two neighbouring aggregates across the boundary share a colour; aggregates
# of up to 256 sites take the fused one-CTA-per-block pass (4^4; a ragged 24-thread
# warp for 2x2x2x3), larger ones (4x4x4x5 = 320 sites) the per-step kernels
CASES = [((4, 4, 4, 8), (2, 2, 2, 2), 4, 1), ((4, 4, 4, 8), (2, 2, 2, 4), 3, 2), ((6, 4, 4, 4), (2, 2, 2, 2), 2, 3),
         ((4, 4, 4, 4), (1, 1, 1, 1), 5, 1), ((4, 4, 4, 4), (4, 4, 4, 4), 4, 1), ((8, 8, 8, 8), (4, 4, 4, 4), 4, 1),
         ((4, 4, 4, 6), (2, 2, 2, 3), 3, 1), ((8, 4, 4, 10), (4, 4, 4, 5), 3, 1), ((4, 4, 4, 5), (4, 4, 4, 5), 2, 1)]


@pytest.mark.parametrize("dims,block,steps,cycles", CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)], ids=["f64", "f32"])
def test_fine_sap_matches_oracle(lib, dims, block, steps, cycles, prec, tol):
    nrhs = 2
    ctx, D = fine_ctx(lib, dims, block, 4, prec, sap_cycles=cycles, max_rhs=nrhs)
    V = int(np.prod(dims))
    b = inputs.complex_gaussian(1202, 0, (nrhs, V, 12))
    x = dev(np.zeros_like(b))
    ctx.krylov(0, 2, dev(b), x, nrhs=nrhs, steps_or_restart=steps)
    got = host(x)
    for r, f in enumerate(fields(b, dims, 12)):
        assert rel(got[r], sap(D, dims, block, f, steps, cycles).reshape(V, 12)) < tol, r


def three_level(lib, **kw):
    dims, b0, b1 = (8, 8, 8, 8), (2, 2, 2, 2), (2, 2, 2, 2)
    p = lib.default_params(dims=dims, blocks=[b0, b1], nvec=[6, 4], n_levels=3, m0=-0.1, csw=1.0,
                           smoother=lib.SMOOTHER_SAP, **kw)
    ctx = lib.Context(p)
    U = inputs.random_gauge(dims, 0.3, 1203)
    ctx.set_gauge(dev(U))
    iv0 = inputs.setup_vectors(dims, 12, 6, 0, 1203)
    iv1 = inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1203)
    ctx.setup(dev(np.concatenate([iv0.ravel(), iv1.ravel()])))
    return ctx, WilsonClover(U, dims, -0.1, 1.0), [fields(iv0, dims, 12), fields(iv1, (4, 4, 4, 4), 12)]


def test_coarse_level_sap_matches_oracle(lib):
    """SAP on level 1 (coarse nine-block operator, nbasis 12) over its own aggregates,
    the oracle running on the library's FP64 coarse links."""
    ctx, _, _ = three_level(lib, max_rhs=2)
    cd, nb = (4, 4, 4, 4), 12
    Vc = int(np.prod(cd))
    A = dev(np.zeros((9, Vc, nb, nb), dtype=complex))
    ctx.get_coarse_links(1, A)
    A = host(A)
    op = CoarseOperator(np.stack([to_grid(A[d], cd) for d in range(9)]), cd)
    b = inputs.complex_gaussian(1204, 0, (2, Vc, nb))
    x = dev(np.zeros_like(b))
    ctx.krylov(1, 2, dev(b), x, nrhs=2, steps_or_restart=4)
    got = host(x)
    for r in range(2):
        want = sap(op, cd, (2, 2, 2, 2), to_grid(b[r], cd), 4, 1)
        assert rel(got[r], want.reshape(Vc, nb)) < 1e-12, r


def test_sap_setup_cycle_and_solve_match_oracle(lib):
    """SAP as the smoother of the setup sweeps (initial and refinement), the cycle and
    the solve, all levels, against the oracle's multigrid with the same smoother."""
    dims, block, nvec = (4, 4, 4, 8), (2, 2, 2, 2), 8
    ctx, D = fine_ctx(lib, dims, block, nvec, 0, setup_refine_sweeps=1, sap_cycles=1)
    iv = inputs.setup_vectors(dims, 12, nvec, 0, 1201)
    ctx.setup(dev(iv))
    mg = Multigrid(D, MGParams(blocks=[block], nvecs=[nvec], smoother="sap", refine_sweeps=1),
                   [fields(iv, dims, 12)])
    V = int(np.prod(dims))
    P = dev(np.zeros((nvec, V, 12), dtype=complex))
    ctx.get_nullvecs(0, P)
    assert rel(host(P), mg.levels[0].agg.v.reshape(nvec, V, 12)) < 1e-9
    r = inputs.complex_gaussian(1205, 0, (1, V, 12))
    e = dev(np.zeros_like(r))
    ctx.mg_cycle(dev(r), e)
    assert rel(host(e)[0], mg.cycle(0, fields(r, dims, 12)[0]).reshape(V, 12)) < 1e-9
    b = inputs.source(dims, 0)
    x = dev(np.zeros_like(b))
    st = ctx.solve(dev(b), x)
    xo, info = mg.solve(fields(b, dims, 12)[0])
    assert st.converged and st.true_residual <= 1e-10
    assert rel(host(x)[0].reshape(V, 12), xo.reshape(V, 12)) < 1e-8
    assert abs(st.outer_iterations - info.iterations) <= 1


@pytest.mark.parametrize("kcycle", [0, 1], ids=["vcycle", "kcycle"])
def test_three_level_sap_cycle_matches_oracle(lib, kcycle):
    ctx, D, iv = three_level(lib, kcycle=kcycle)
    mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvecs=[6, 4], smoother="sap",
                               kcycle=bool(kcycle)), iv)
    V = 4096
    r = inputs.complex_gaussian(1206, 0, (1, V, 12))
    e = dev(np.zeros_like(r))
    ctx.mg_cycle(dev(r), e)
    assert rel(host(e)[0], mg.cycle(0, fields(r, (8, 8, 8, 8), 12)[0]).reshape(V, 12)) < 1e-9


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32_inner"])
def test_sap_graph_replay_matches_host_driven(lib, prec):
    dims, block = (8, 8, 8, 8), (2, 2, 2, 2)
    ref, _ = fine_ctx(lib, dims, block, 6, prec, seed=1207)
    ctx, _ = fine_ctx(lib, dims, block, 6, prec, seed=1207, use_graphs=1)
    iv = dev(inputs.setup_vectors(dims, 12, 6, 0, 1207))
    ref.setup(iv)
    ctx.setup(iv)
    b = inputs.source(dims, 0)
    xe = dev(np.zeros_like(b))
    se = ref.solve(dev(b), xe)
    assert se.graph == 0 and se.converged
    for call in range(3):
        x = dev(np.zeros_like(b))
        st = ctx.solve(dev(b), x)
        assert st.graph == (1 if call else 0) and st.converged and st.true_residual <= 1e-10
        assert st.outer_iterations == se.outer_iterations and st.coarse_iterations == se.coarse_iterations
        assert rel(host(x), host(xe)) < 1e-13


def test_sap_on_coarsest_level_is_rejected(lib):
    ctx, _ = fine_ctx(lib, (4, 4, 4, 4), (2, 2, 2, 2), 4)
    ctx.setup(dev(inputs.setup_vectors((4, 4, 4, 4), 12, 4, 0, 1201)))
    b = dev(np.zeros((1, 16, 8), dtype=complex))
    with pytest.raises(lib.WcmgError) as e:
        ctx.krylov(1, 2, b, dev(np.zeros((1, 16, 8), dtype=complex)), nrhs=1, steps_or_restart=2)
    assert e.value.code == lib.ERR_ARG


def test_clover_inverse_matches_dense_inverse(lib):
    dims = (4, 4, 4, 8)
    ctx, D = fine_ctx(lib, dims, (2, 2, 2, 2), 4, sap_eo=1)
    V = int(np.prod(dims))
    Ci = dev(np.zeros((V, 12, 12), dtype=complex))
    ctx.get_clover_inverse(Ci)
    want = np.linalg.inv(D.C).reshape(V, 12, 12)
    assert rel(host(Ci), want) < 1e-13


# even-odd block solves: x extents even; 2x2x2x3 aggregates have first sites of both
# parities, 2x1x1x1 ones a single even-odd pair (ragged warps)
EO_CASES = [((4, 4, 4, 8), (2, 2, 2, 2), 4, 1), ((4, 4, 4, 8), (2, 2, 2, 4), 3, 2), ((6, 4, 4, 4), (2, 2, 2, 2), 2, 3),
            ((8, 8, 8, 8), (4, 4, 4, 4), 4, 1), ((4, 4, 4, 4), (4, 4, 4, 4), 3, 1), ((4, 4, 4, 6), (2, 2, 2, 3), 3, 1),
            ((4, 2, 2, 4), (2, 1, 1, 1), 2, 2)]


@pytest.mark.parametrize("dims,block,steps,cycles", EO_CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)], ids=["f64", "f32"])
def test_fine_sap_even_odd_matches_oracle(lib, dims, block, steps, cycles, prec, tol):
    nrhs = 2
    ctx, D = fine_ctx(lib, dims, block, 2, prec, sap_cycles=cycles, sap_eo=1, max_rhs=nrhs)
    V = int(np.prod(dims))
    b = inputs.complex_gaussian(1208, 0, (nrhs, V, 12))
    x = dev(np.zeros_like(b))
    ctx.krylov(0, 2, dev(b), x, nrhs=nrhs, steps_or_restart=steps)
    got = host(x)
    for r, f in enumerate(fields(b, dims, 12)):
        assert rel(got[r], sap(D, dims, block, f, steps, cycles, eo=True).reshape(V, 12)) < tol, r


def test_sap_even_odd_setup_cycle_and_solve_match_oracle(lib):
    dims, block, nvec = (4, 4, 4, 8), (2, 2, 2, 2), 8
    ctx, D = fine_ctx(lib, dims, block, nvec, 0, setup_refine_sweeps=1, sap_eo=1)
    iv = inputs.setup_vectors(dims, 12, nvec, 0, 1201)
    ctx.setup(dev(iv))
    mg = Multigrid(D, MGParams(blocks=[block], nvecs=[nvec], smoother="sap", sap_eo=True, refine_sweeps=1),
                   [fields(iv, dims, 12)])
    V = int(np.prod(dims))
    P = dev(np.zeros((nvec, V, 12), dtype=complex))
    ctx.get_nullvecs(0, P)
    assert rel(host(P), mg.levels[0].agg.v.reshape(nvec, V, 12)) < 1e-9
    r = inputs.complex_gaussian(1209, 0, (1, V, 12))
    e = dev(np.zeros_like(r))
    ctx.mg_cycle(dev(r), e)
    assert rel(host(e)[0], mg.cycle(0, fields(r, dims, 12)[0]).reshape(V, 12)) < 1e-9
    b = inputs.source(dims, 0)
    x = dev(np.zeros_like(b))
    st = ctx.solve(dev(b), x)
    xo, info = mg.solve(fields(b, dims, 12)[0])
    assert st.converged and st.true_residual <= 1e-10
    assert rel(host(x)[0].reshape(V, 12), xo.reshape(V, 12)) < 1e-8
    assert abs(st.outer_iterations - info.iterations) <= 1


def test_sap_even_odd_graph_replay_matches_host_driven(lib):
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    ref, _ = fine_ctx(lib, dims, block, 6, 1, seed=1210, sap_eo=1)
    ctx, _ = fine_ctx(lib, dims, block, 6, 1, seed=1210, sap_eo=1, use_graphs=1)
    iv = dev(inputs.setup_vectors(dims, 12, 6, 0, 1210))
    ref.setup(iv)
    ctx.setup(iv)
    b = inputs.source(dims, 0)
    xe = dev(np.zeros_like(b))
    se = ref.solve(dev(b), xe)
    assert se.graph == 0 and se.converged
    for call in range(3):
        x = dev(np.zeros_like(b))
        st = ctx.solve(dev(b), x)
        assert st.graph == (1 if call else 0) and st.converged and st.true_residual <= 1e-10
        assert st.outer_iterations == se.outer_iterations and st.coarse_iterations == se.coarse_iterations
        assert rel(host(x), host(xe)) < 1e-13


def test_clover_inverse_needs_sap_eo(lib):
    ctx, _ = fine_ctx(lib, (4, 4, 4, 4), (2, 2, 2, 2), 4)
    with pytest.raises(lib.WcmgError) as e:
        ctx.get_clover_inverse(dev(np.zeros((256, 12, 12), dtype=complex)))
    assert e.value.code == lib.ERR_STATE
