"""The solve as one CUDA graph (device-side stopping tests, Sec. 2.1 FGMRES /
GMRES) and the batched solve of lattices of uneven sizes in one graph launch.

A replay runs the same kernels with the same arguments in the same order as
the host-driven solve, so its iterates, iteration counts and solution agree
with the host-driven ones (up to the last bits); the solution also matches the
FP64 oracle's multigrid solve."""
import numpy as np
import pytest

from oracle.mg import MGParams, Multigrid
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, fields, host, rel

pytestmark = pytest.mark.gpu


def make_ctx(lib, dims, block, nvec, prec, seed, eps=0.3, m0=-0.1, setup=True, **kw):
    p = lib.default_params(dims=dims, blocks=[block], nvec=[nvec], m0=m0, csw=1.0, inner_prec=prec, **kw)
    ctx = lib.Context(p)
    U = inputs.random_gauge(dims, eps, seed)
    ctx.set_gauge(dev(U))
    iv = inputs.setup_vectors(dims, 12, nvec, 0, seed)
    if setup:
        ctx.setup(dev(iv))
    return ctx, U, iv


@pytest.mark.parametrize("prec,smoother", [(0, 0), (1, 0), (1, 1)], ids=["f64", "f32_inner", "f32_gmres_smoother"])
def test_graph_replay_matches_host_driven(lib, prec, smoother):
    dims, block = (8, 8, 8, 8), (2, 2, 2, 2)
    ref, U, iv = make_ctx(lib, dims, block, 6, prec, 1021, smoother=smoother)
    ctx, _, _ = make_ctx(lib, dims, block, 6, prec, 1021, use_graphs=1, smoother=smoother)
    b = inputs.source(dims, 0)
    xe = dev(np.zeros_like(b))
    se = ref.solve(dev(b), xe)
    assert se.graph == 0 and se.converged
    runs = []
    for _ in range(3):
        x = dev(np.zeros_like(b))
        runs.append((ctx.solve(dev(b), x), host(x)))
    assert [st.graph for st, _ in runs] == [0, 1, 1]
    for st, x in runs:
        assert st.converged and st.true_residual <= 1e-10
        assert st.outer_iterations == se.outer_iterations
        assert st.coarse_iterations == se.coarse_iterations
        assert rel(x, host(xe)) < 1e-13
    # a replay launches every kernel of the host-driven solve plus its control kernels
    assert runs[2][0].kernel_launches >= se.kernel_launches
    if prec == 0:
        D = WilsonClover(U, dims, -0.1, 1.0)
        mg = Multigrid(D, MGParams(blocks=[block], nvecs=[6]), [fields(iv, dims, 12)])
        xo, info = mg.solve(fields(b, dims, 12)[0])
        assert rel(runs[2][1][0].reshape(-1, 12), xo.reshape(-1, 12)) < 1e-8
        assert abs(runs[2][0].outer_iterations - info.iterations) <= 1


@pytest.mark.parametrize("kcycle", [0, 1], ids=["vcycle", "kcycle"])
def test_graph_replay_three_levels(lib, kcycle):
    dims = (8, 8, 8, 8)
    kw = dict(dims=dims, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[6, 4], n_levels=3, m0=-0.1, csw=1.0,
              inner_prec=1, setup_refine_sweeps=1, kcycle=kcycle)
    U = inputs.random_gauge(dims, 0.3, 1003)
    iv = np.concatenate([inputs.setup_vectors(dims, 12, 6, 0, 1003).ravel(),
                         inputs.setup_vectors((4, 4, 4, 4), 12, 4, 1, 1003).ravel()])
    out = []
    for g in (0, 1):
        ctx = lib.Context(lib.default_params(use_graphs=g, **kw))
        ctx.set_gauge(dev(U))
        ctx.setup(dev(iv))
        b = inputs.source(dims, 0)
        for _ in range(3 if g else 1):
            x = dev(np.zeros_like(b))
            st = ctx.solve(dev(b), x)
        out.append((st, host(x)))
    (se, xe), (sg, xg) = out
    assert sg.graph == 1 and sg.converged and sg.true_residual <= 1e-10
    assert sg.outer_iterations == se.outer_iterations and sg.coarse_iterations == se.coarse_iterations
    assert rel(xg, xe) < 1e-13


def test_graph_not_converged_stops_at_maxiter(lib):
    ctx, _, _ = make_ctx(lib, (4, 4, 4, 4), (2, 2, 2, 2), 8, 1, 1001, outer_maxiter=3, use_graphs=1)
    b = inputs.source((4, 4, 4, 4), 0)
    sts = [ctx.solve(dev(b), dev(np.zeros_like(b)), allow_not_converged=True) for _ in range(2)]
    assert sts[1].graph == 1
    for st in sts:
        assert not st.converged and st.outer_iterations == 3


def test_graph_non_finite_source_is_nan_error(lib):
    ctx, _, _ = make_ctx(lib, (4, 4, 4, 4), (2, 2, 2, 2), 8, 1, 1001, use_graphs=1)
    b = inputs.source((4, 4, 4, 4), 0)
    ctx.solve(dev(b), dev(np.zeros_like(b)))  # host-driven (first solve)
    bad = b.copy()
    bad[0, 3, 2] = np.nan
    with pytest.raises(lib.WcmgError) as e:
        ctx.solve(dev(bad), dev(np.zeros_like(b)))
    assert e.value.code == lib.ERR_NAN
    st = ctx.solve(dev(b), dev(np.zeros_like(b)))  # the context stays usable
    assert st.graph == 1 and st.converged


UNEVEN = [((4, 4, 4, 4), (2, 2, 2, 2), 1031), ((8, 8, 8, 8), (4, 4, 4, 4), 1032),
          ((12, 12, 12, 8), (4, 4, 4, 4), 1033)]


def test_batch_of_uneven_lattices_matches_single_solves(lib):
    """The batch equals the single solves of the same contexts (same kernels, so to the
    last bits) and the oracle: each member's solution has a true residual <= 1e-10
    under the oracle's own D, and on the two smaller lattices it equals the solution of
    the oracle's FP64 multigrid solve (both solved to 1e-10; D is well conditioned at
    these parameters, so the two agree to 1e-8)."""
    nrhs = 2
    refs, ctxs, bs, gauges, ivs = [], [], [], [], []
    for dims, block, seed in UNEVEN:
        r, U, iv = make_ctx(lib, dims, block, 6, 1, seed, max_rhs=nrhs)
        c, _, _ = make_ctx(lib, dims, block, 6, 1, seed, max_rhs=nrhs)
        V = int(np.prod(dims))
        b = inputs.complex_gaussian(seed, 0, (nrhs, V, 12))
        refs.append(r)
        ctxs.append(c)
        bs.append(b)
        gauges.append(U)
        ivs.append(iv)
    want = []
    for r, b in zip(refs, bs):
        x = dev(np.zeros_like(b))
        want.append((r.solve(dev(b), x, nrhs=nrhs), host(x)))
    for call in range(3):
        xs = [dev(np.zeros_like(b)) for b in bs]
        sts = lib.Context.solve_batch(ctxs, [dev(b) for b in bs], xs, nrhs=[nrhs] * len(bs))
        for (sw, xw), st, x in zip(want, sts, xs):
            assert st.graph == (1 if call else 0)
            assert st.converged and st.true_residual <= 1e-10
            assert st.outer_iterations == sw.outer_iterations
            assert st.coarse_iterations == sw.coarse_iterations
            assert rel(host(x), xw) < 1e-13
    for k, ((dims, block, _), U, iv, b, x) in enumerate(zip(UNEVEN, gauges, ivs, bs, xs)):
        V = int(np.prod(dims))
        D = WilsonClover(U, dims, -0.1, 1.0)
        got = host(x)
        mg = Multigrid(D, MGParams(blocks=[block], nvecs=[6]), [fields(iv, dims, 12)]) if k < 2 else None
        for q, f in enumerate(fields(b, dims, 12)):
            xq = got[q].reshape(V, 12)
            r = f.reshape(V, 12) - D(fields(xq[None], dims, 12)[0]).reshape(V, 12)
            assert np.linalg.norm(r) / np.linalg.norm(f) <= 1e-10, (dims, q)
            if mg is not None:
                xo, info = mg.solve(f)
                assert info.converged
                assert rel(xq, xo.reshape(V, 12)) < 1e-8, (dims, q)


def test_batch_rejects_repeated_context(lib):
    ctx, _, _ = make_ctx(lib, (4, 4, 4, 4), (2, 2, 2, 2), 8, 1, 1001)
    b = inputs.source((4, 4, 4, 4), 0)
    with pytest.raises(lib.WcmgError) as e:
        lib.Context.solve_batch([ctx, ctx], [dev(b), dev(b)], [dev(np.zeros_like(b)), dev(np.zeros_like(b))])
    assert e.value.code == lib.ERR_ARG
