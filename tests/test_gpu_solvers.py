"""GPU parity of MR, GMRES, the MG cycle, the setup and the FGMRES solve
against the FP64 oracle (Sec. 2.1)."""
import numpy as np
import pytest

from oracle.aggregation import Aggregation
from oracle.coarse import coarsen
from oracle.lattice import coarse_dims, to_grid
from oracle.mg import MGParams, Multigrid
from oracle.solvers import gmres, mr
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, fields, host, rel, rel_norm, residual

pytestmark = pytest.mark.gpu

DIMS, BLOCK, NVEC = (4, 4, 4, 4), (2, 2, 2, 2), 8


def config1_ctx(lib, prec=0, **kw):
    p = lib.default_params(dims=DIMS, blocks=[BLOCK], nvec=[NVEC], m0=-0.1, csw=1.0, inner_prec=prec, **kw)
    ctx = lib.Context(p)
    U = inputs.random_gauge(DIMS, 0.3, 1001)
    ctx.set_gauge(dev(U))
    return ctx, WilsonClover(U, DIMS, -0.1, 1.0)


@pytest.mark.parametrize("steps", [1, 2, 4, 7])
def test_mr_matches_oracle(lib, steps):
    """One step (the iterate directly), two (no middle step), the configurations' four and
    seven, for three rhs at once."""
    ctx, D = config1_ctx(lib, max_rhs=3)
    V = 256
    b = inputs.complex_gaussian(21, 0, (3, V, 12))
    x = dev(np.zeros_like(b))
    ctx.krylov(0, 0, dev(b), x, nrhs=3, steps_or_restart=steps)
    got = host(x)
    for r, f in enumerate(fields(b, DIMS, 12)):
        assert rel(got[r], mr(D, f, steps).reshape(V, 12)) < 1e-12


@pytest.mark.parametrize("nrhs", [1, 3, 4])
def test_mr_fp32_fused_reductions_match_oracle(lib, nrhs):
    """FP32 MR: <p, r> and <p, p> come out of the Dslash epilogue (two rhs per thread)."""
    ctx, D = config1_ctx(lib, prec=1, max_rhs=4)
    V = 256
    b = inputs.complex_gaussian(25, nrhs, (nrhs, V, 12))
    x = dev(np.zeros_like(b))
    ctx.krylov(0, 0, dev(b), x, nrhs=nrhs, steps_or_restart=4)
    got = host(x)
    for r, f in enumerate(fields(b, DIMS, 12)):
        assert rel(got[r], mr(D, f, 4).reshape(V, 12)) < 1e-5


def test_gmres_fixed_iterations_matches_oracle(lib):
    ctx, D = config1_ctx(lib, max_rhs=2)
    V = 256
    b = inputs.complex_gaussian(22, 0, (2, V, 12))
    x = dev(np.zeros_like(b))
    its = ctx.krylov(0, 1, dev(b), x, nrhs=2, steps_or_restart=10, tol=0.0, maxiter=25)
    assert its == 25
    got = host(x)
    for r, f in enumerate(fields(b, DIMS, 12)):
        ref, info = gmres(D, f, restart=10, tol=0.0, maxiter=25)
        assert info.iterations == 25
        assert rel(got[r], ref.reshape(V, 12)) < 1e-11


def test_gmres_tolerance_batched_rhs_freeze(lib):
    """rhs of different difficulty in one batch: each stops at its own iteration."""
    ctx, D = config1_ctx(lib, max_rhs=2)
    V = 256
    b = inputs.complex_gaussian(23, 0, (2, V, 12))
    b[1] *= 1e-3
    x = dev(np.zeros_like(b))
    ctx.krylov(0, 1, dev(b), x, nrhs=2, steps_or_restart=20, tol=1e-6, maxiter=500)
    got = host(x)
    for r, f in enumerate(fields(b, DIMS, 12)):
        ref, info = gmres(D, f, restart=20, tol=1e-6, maxiter=500)
        assert rel(got[r], ref.reshape(V, 12)) < 1e-9


def oracle_mg(D, iv, **kw):
    return Multigrid(D, MGParams(blocks=[BLOCK], nvecs=[NVEC], **kw), [fields(iv, DIMS, 12)])


@pytest.mark.parametrize("ortho_df", [0, 1], ids=["fp64_ortho", "double_float_ortho"])
def test_setup_and_cycle_match_oracle(lib, ortho_df):
    ctx, D = config1_ctx(lib, ortho_df=ortho_df)
    iv = inputs.setup_vectors(DIMS, 12, NVEC, 0, 1001)
    ctx.setup(dev(iv))
    mg = oracle_mg(D, iv)
    V = 256
    P = dev(np.zeros((NVEC, V, 12), dtype=complex))
    ctx.get_nullvecs(0, P)
    assert rel(host(P), mg.levels[0].agg.v.reshape(NVEC, V, 12)) < 1e-10
    cd = coarse_dims(DIMS, BLOCK)
    A = dev(np.zeros((9, 16, 16, 16), dtype=complex))
    ctx.get_coarse_links(1, A)
    assert rel(host(A), mg.levels[1].op.A.reshape(9, 16, 16, 16)) < 1e-10
    r = inputs.complex_gaussian(24, 0, (1, V, 12))
    e = dev(np.zeros_like(r))
    ctx.mg_cycle(dev(r), e)
    ref = mg.cycle(0, fields(r, DIMS, 12)[0])
    assert rel(host(e)[0], ref.reshape(V, 12)) < 1e-9


@pytest.mark.parametrize("ortho_df", [0, 1], ids=["fp64_ortho", "double_float_ortho"])
def test_setup_with_refinement_matches_oracle(lib, ortho_df):
    ctx, D = config1_ctx(lib, setup_refine_sweeps=2, ortho_df=ortho_df)
    iv = inputs.setup_vectors(DIMS, 12, NVEC, 0, 1001)
    ctx.setup(dev(iv))
    mg = oracle_mg(D, iv, refine_sweeps=2)
    A = dev(np.zeros((9, 16, 16, 16), dtype=complex))
    ctx.get_coarse_links(1, A)
    assert rel(host(A), mg.levels[1].op.A.reshape(9, 16, 16, 16)) < 1e-8


def test_solve_matches_oracle_fp64(lib):
    ctx, D = config1_ctx(lib)
    iv = inputs.setup_vectors(DIMS, 12, NVEC, 0, 1001)
    ctx.setup(dev(iv))
    b = inputs.source(DIMS, 0)
    x = dev(np.zeros_like(b))
    st = ctx.solve(dev(b), x)
    assert st.converged and st.true_residual <= 1e-10
    mg = oracle_mg(D, iv)
    xo, info = mg.solve(fields(b, DIMS, 12)[0])
    assert rel(host(x)[0].reshape(256, 12), xo.reshape(256, 12)) < 1e-8
    assert abs(st.outer_iterations - info.iterations) <= 1


def test_solve_mixed_precision_reaches_1e10(lib):
    ctx, D = config1_ctx(lib, prec=1)
    iv = inputs.setup_vectors(DIMS, 12, NVEC, 0, 1001)
    ctx.setup(dev(iv))
    b = inputs.source(DIMS, 0)
    x = dev(np.zeros_like(b))
    st = ctx.solve(dev(b), x)
    assert st.converged and st.true_residual <= 1e-10
    xr = host(x)[0].reshape(256, 12)
    assert residual(D(to_grid(xr, DIMS)).reshape(256, 12), b[0].reshape(256, 12)) <= 1e-10


def test_three_level_solve(lib):
    dims = (8, 8, 8, 8)
    p = lib.default_params(dims=dims, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[6, 4], n_levels=3, m0=-0.1,
                           csw=1.0, setup_refine_sweeps=1)
    ctx = lib.Context(p)
    U = inputs.random_gauge(dims, 0.3, 1003)
    ctx.set_gauge(dev(U))
    V = 4096
    iv = np.concatenate([inputs.setup_vectors(dims, 12, 6, 0, 1003).ravel(),
                         inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1003).ravel()])
    ctx.setup(dev(iv))
    b = inputs.source(dims, 0)
    x = dev(np.zeros_like(b))
    st = ctx.solve(dev(b), x)
    assert st.converged and st.true_residual <= 1e-10
    D = WilsonClover(U, dims, -0.1, 1.0)
    iv0 = inputs.setup_vectors(dims, 12, 6, 0, 1003)
    iv1 = inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1003)
    mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvecs=[6, 4], refine_sweeps=1),
                   [fields(iv0, dims, 12), fields(iv1, (4, 4, 4, 4), 12)])
    xo, info = mg.solve(fields(b, dims, 12)[0])
    assert rel(host(x)[0].reshape(V, 12), xo.reshape(V, 12)) < 1e-8
    assert abs(st.outer_iterations - info.iterations) <= 1


def test_checkpoint_round_trip_bitwise(lib, tmp_path):
    ctx, D = config1_ctx(lib)
    iv = inputs.setup_vectors(DIMS, 12, NVEC, 0, 1001)
    ctx.setup(dev(iv))
    b = inputs.source(DIMS, 0)
    x1 = dev(np.zeros_like(b))
    ctx.solve(dev(b), x1)
    path = str(tmp_path / "setup.bin")
    ctx.save_setup(path)
    ctx2, _ = config1_ctx(lib)
    ctx2.load_setup(path)
    x2 = dev(np.zeros_like(b))
    ctx2.solve(dev(b), x2)
    assert np.array_equal(host(x1), host(x2))


def test_solve_before_setup_is_state_error(lib):
    ctx, D = config1_ctx(lib)
    b = inputs.source(DIMS, 0)
    with pytest.raises(lib.WcmgError) as e:
        ctx.solve(dev(b), dev(np.zeros_like(b)))
    assert e.value.code == lib.ERR_STATE


def test_not_converged_reported(lib):
    ctx, D = config1_ctx(lib, outer_maxiter=2)
    iv = inputs.setup_vectors(DIMS, 12, NVEC, 0, 1001)
    ctx.setup(dev(iv))
    b = inputs.source(DIMS, 0)
    st = ctx.solve(dev(b), dev(np.zeros_like(b)), allow_not_converged=True)
    assert not st.converged and st.outer_iterations == 2


def test_gmres_smoother_setup_cycle_and_solve_match_oracle(lib):
    """GMRES(4) as the smoother (zero guess, no restart) in the setup sweeps and the cycle."""
    ctx, D = config1_ctx(lib, smoother=lib.SMOOTHER_GMRES, setup_refine_sweeps=1)
    iv = inputs.setup_vectors(DIMS, 12, NVEC, 0, 1001)
    ctx.setup(dev(iv))
    mg = oracle_mg(D, iv, smoother="gmres", refine_sweeps=1)
    V = 256
    P = dev(np.zeros((NVEC, V, 12), dtype=complex))
    ctx.get_nullvecs(0, P)
    assert rel(host(P), mg.levels[0].agg.v.reshape(NVEC, V, 12)) < 1e-9
    r = inputs.complex_gaussian(26, 0, (1, V, 12))
    e = dev(np.zeros_like(r))
    ctx.mg_cycle(dev(r), e)
    assert rel(host(e)[0], mg.cycle(0, fields(r, DIMS, 12)[0]).reshape(V, 12)) < 1e-9
    b = inputs.source(DIMS, 0)
    x = dev(np.zeros_like(b))
    st = ctx.solve(dev(b), x)
    xo, info = mg.solve(fields(b, DIMS, 12)[0])
    assert st.converged and st.true_residual <= 1e-10
    assert rel(host(x)[0].reshape(V, 12), xo.reshape(V, 12)) < 1e-8
    assert abs(st.outer_iterations - info.iterations) <= 1


@pytest.mark.parametrize("kcycle", [0, 1], ids=["vcycle", "kcycle"])
def test_three_level_cycles_match_oracle(lib, kcycle):
    """Three levels with the V-cycle (one cycle of level 1 as its coarse solve) and the
    K-cycle (FGMRES(5) to 0.1 around the level-1 cycle): cycle output and solve vs the oracle."""
    dims, b0, b1 = (8, 8, 8, 8), (2, 2, 2, 2), (2, 2, 2, 2)
    p = lib.default_params(dims=dims, blocks=[b0, b1], nvec=[6, 4], n_levels=3, m0=-0.1, csw=1.0, kcycle=kcycle)
    ctx = lib.Context(p)
    U = inputs.random_gauge(dims, 0.3, 1003)
    ctx.set_gauge(dev(U))
    iv0 = inputs.setup_vectors(dims, 12, 6, 0, 1003)
    iv1 = inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1003)
    ctx.setup(dev(np.concatenate([iv0.ravel(), iv1.ravel()])))
    D = WilsonClover(U, dims, -0.1, 1.0)
    mg = Multigrid(D, MGParams(blocks=[b0, b1], nvecs=[6, 4], kcycle=bool(kcycle)),
                   [fields(iv0, dims, 12), fields(iv1, (4, 4, 4, 4), 12)])
    V = 4096
    r = inputs.complex_gaussian(32, 0, (1, V, 12))
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


def test_seeded_setup_draws_the_fields_of_the_input_generator(lib):
    """wcmg_setup_seeded generates the random vectors on the device with the counter-based
    generator of the test inputs (exact uniforms, FP32 Box-Muller transform): with no
    smoothing sweeps P is the block-orthonormalised random vectors, equal to those of the
    host-generated (FP64-transformed) fields to FP32 rounding, on both levels; with setup
    sweeps they still agree to that order.  Compared in the 2-norm: element-wise, FP32
    evaluation of log(1 - u) for tiny u leaves samples of small radius an absolute error of
    ~1e-5, up to 4e-5 of the largest entry."""
    dims = (8, 8, 8, 8)
    kw = dict(dims=dims, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[6, 4], n_levels=3, m0=-0.1, csw=1.0)
    U = inputs.random_gauge(dims, 0.3, 1401)
    iv = np.concatenate([inputs.setup_vectors(dims, 12, 6, 0, 1401).ravel(),
                         inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1401).ravel()])
    for sweeps, tol in ((0, 1e-6), (3, 1e-5)):
        P = []
        for seeded in (False, True):
            ctx = lib.Context(lib.default_params(setup_init_sweeps=sweeps, setup_refine_sweeps=min(sweeps, 1), **kw))
            ctx.set_gauge(dev(U))
            if seeded:
                ctx.setup_seeded(1401)
            else:
                ctx.setup(dev(iv))
            P0 = dev(np.zeros((6, 4096, 12), dtype=complex))
            P1 = dev(np.zeros((4, 256, 12), dtype=complex))
            ctx.get_nullvecs(0, P0)
            ctx.get_nullvecs(1, P1)
            P.append((host(P0), host(P1)))
        assert rel_norm(P[1][0], P[0][0]) < tol and rel_norm(P[1][1], P[0][1]) < tol


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32_inner"])
def test_even_odd_coarsest_solve_matches_oracle(lib, prec):
    """coarse_eo: the coarsest GMRES runs on the odd-site Schur complement (Sec. 4
    red-black preconditioning).  The MG cycle equals the oracle's cycle with the same
    even-odd coarsest solve; the solve reaches the oracle's solution."""
    ctx, D = config1_ctx(lib, prec=prec, coarse_eo=1)
    iv = inputs.setup_vectors(DIMS, 12, NVEC, 0, 1001)
    ctx.setup(dev(iv))
    mg = oracle_mg(D, iv, coarse_eo=True)
    V = 256
    r = inputs.complex_gaussian(27, 0, (1, V, 12))
    e = dev(np.zeros_like(r))
    ctx.mg_cycle(dev(r), e)
    ref = mg.cycle(0, fields(r, DIMS, 12)[0]).reshape(V, 12)
    assert rel(host(e)[0], ref) < (1e-9 if prec == 0 else 1e-4)
    b = inputs.source(DIMS, 0)
    x = dev(np.zeros_like(b))
    st = ctx.solve(dev(b), x)
    assert st.converged and st.true_residual <= 1e-10
    xo, info = mg.solve(fields(b, DIMS, 12)[0])
    assert rel(host(x)[0].reshape(V, 12), xo.reshape(V, 12)) < 1e-8
    if prec == 0:
        assert abs(st.outer_iterations - info.iterations) <= 1


def test_even_odd_coarsest_solve_three_levels_and_graph_replay(lib):
    """Three levels (8^4 -> 4^4 -> 2^4) with the even-odd coarsest solve: the cycle equals
    the oracle's; FP32 inner levels under CUDA-graph replay reproduce the host-driven
    solve."""
    dims = (8, 8, 8, 8)
    kw = dict(dims=dims, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[6, 4], n_levels=3, m0=-0.1, csw=1.0, coarse_eo=1)
    U = inputs.random_gauge(dims, 0.3, 1061)
    iv0 = inputs.setup_vectors(dims, 12, 6, 0, 1061)
    iv1 = inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1061)
    ctx = lib.Context(lib.default_params(**kw))
    ctx.set_gauge(dev(U))
    ctx.setup(dev(np.concatenate([iv0.ravel(), iv1.ravel()])))
    D = WilsonClover(U, dims, -0.1, 1.0)
    mg = Multigrid(D, MGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvecs=[6, 4], coarse_eo=True),
                   [fields(iv0, dims, 12), fields(iv1, (4, 4, 4, 4), 12)])
    V = 4096
    r = inputs.complex_gaussian(28, 0, (1, V, 12))
    e = dev(np.zeros_like(r))
    ctx.mg_cycle(dev(r), e)
    assert rel(host(e)[0], mg.cycle(0, fields(r, dims, 12)[0]).reshape(V, 12)) < 1e-9
    g = lib.Context(lib.default_params(inner_prec=lib.F32, use_graphs=1, **kw))
    g.set_gauge(dev(U))
    g.setup(dev(np.concatenate([iv0.ravel(), iv1.ravel()])))
    b = inputs.source(dims, 0)
    runs = []
    for _ in range(3):
        x = dev(np.zeros_like(b))
        runs.append((g.solve(dev(b), x), host(x)))
    assert [st.graph for st, _ in runs] == [0, 1, 1]
    for st, x in runs:
        assert st.converged and st.true_residual <= 1e-10
        assert st.outer_iterations == runs[0][0].outer_iterations
        assert rel(x, runs[0][1]) < 1e-13
