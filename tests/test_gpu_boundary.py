"""GPU tests of the boundary calls that set the clover term, solve from an initial
guess and checkpoint the learned network (Sec. 2.1 statement of the problem: set
the gauge field and clover term, solve D x = b), all through the C-ABI against the
FP64 oracle."""
import os
import tempfile

import numpy as np
import pytest

from oracle.lattice import to_grid
from oracle.mg import MGParams, Multigrid
from oracle.wilson import WilsonClover
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, fields, host, rel, residual

pytestmark = pytest.mark.gpu

DIMS, BLOCK, NVEC = (6, 4, 8, 10), (3, 2, 4, 5), 5   # V = 1920: ragged last CTA, anisotropic


def _ctx(lib, dims=DIMS, block=BLOCK, nvec=NVEC, **kw):
    p = lib.default_params(dims=dims, blocks=[block], nvec=[nvec], m0=-0.17, csw=1.13, max_rhs=3, **kw)
    return lib.Context(p)


def random_chiral_clover(V, seed, diag=4.0 - 0.17):
    """A clover term of no Sheikholeslami-Wohlert form: per site two random Hermitian
    6x6 blocks (chirality + on spins 0, 1; chirality - on spins 2, 3) plus (4 + m0)."""
    rng = np.random.default_rng(seed)
    C = np.zeros((V, 12, 12), dtype=complex)
    for h in range(2):
        X = rng.normal(size=(V, 6, 6)) + 1j * rng.normal(size=(V, 6, 6))
        C[:, 6 * h:6 * h + 6, 6 * h:6 * h + 6] = 0.3 * (X + np.conj(np.swapaxes(X, 1, 2)))
    C += diag * np.eye(12)
    return C


@pytest.mark.parametrize("csw", [0.0, 1.9])
def test_set_clover_rebuilds_with_a_new_csw(lib, csw):
    V = int(np.prod(DIMS))
    U = inputs.random_gauge(DIMS, 0.35, 5001)
    ctx = _ctx(lib)
    ctx.set_gauge(dev(U))
    ctx.set_clover(csw)
    C = dev(np.zeros((V, 12, 12), dtype=complex))
    ctx.get_clover(C)
    D = WilsonClover(U, DIMS, -0.17, csw)
    assert rel(host(C), D.C.reshape(V, 12, 12)) < 1e-13
    psi = inputs.complex_gaussian(5002, 0, (2, V, 4, 3))
    out = dev(np.zeros_like(psi))
    ctx.apply_D(dev(psi), out, nrhs=2, prec=lib.F64)
    for r, f in enumerate(fields(psi, DIMS, 12)):
        assert rel(host(out)[r].reshape(V, 12), D(f).reshape(V, 12)) < 1e-12


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_set_clover_raw_matches_oracle_with_a_non_sw_clover(lib, prec, tol):
    V = int(np.prod(DIMS))
    U = inputs.random_gauge(DIMS, 0.35, 5003)
    Craw = random_chiral_clover(V, 5004)
    ctx = _ctx(lib)
    ctx.set_gauge(dev(U))
    ctx.set_clover_raw(dev(Craw))
    back = dev(np.zeros_like(Craw))
    ctx.get_clover(back)
    assert rel(host(back), Craw) < 1e-15
    D = WilsonClover(U, DIMS, -0.17, 1.13, clover=to_grid(Craw, DIMS))
    psi = inputs.complex_gaussian(5005, 0, (3, V, 4, 3))
    out = dev(np.zeros_like(psi))
    ctx.apply_D(dev(psi), out, nrhs=3, prec=prec)
    for r, f in enumerate(fields(psi, DIMS, 12)):
        assert rel(host(out)[r].reshape(V, 12), D(f).reshape(V, 12)) < tol


def test_set_clover_raw_rejects_blocks_it_cannot_store(lib):
    """A block coupling the two chiralities, or a non-Hermitian block, is rejected and the
    context keeps its previous clover term."""
    V = int(np.prod(DIMS))
    U = inputs.random_gauge(DIMS, 0.35, 5006)
    ctx = _ctx(lib)
    ctx.set_gauge(dev(U))
    ref = dev(np.zeros((V, 12, 12), dtype=complex))
    ctx.get_clover(ref)
    good = random_chiral_clover(V, 5007)
    off = good.copy()
    off[V - 1, 1, 8] = off[V - 1, 8, 1] = 0.5          # chirality coupling at the last site
    nonherm = good.copy()
    nonherm[17, 3, 4] += 0.25j                          # C != C^dag at one site
    for bad in (off, nonherm):
        with pytest.raises(lib.WcmgError) as e:
            ctx.set_clover_raw(dev(bad))
        assert e.value.code == lib.ERR_ARG
    now = dev(np.zeros((V, 12, 12), dtype=complex))
    ctx.get_clover(now)
    assert np.array_equal(host(now), host(ref))


@pytest.mark.parametrize("prec,graphs", [(0, 0), (1, 0), (1, 1)])
def test_solve_from_an_initial_guess(lib, prec, graphs):
    """wcmg_solve_ex with zero_guess = 0 starts from the caller's x: a perturbed solution
    converges in fewer outer iterations than a cold start, still meets the true
    residual (recomputed with the oracle's D), and in FP64 follows the oracle's FGMRES
    started from the same guess."""
    dims, block, nvec = (4, 4, 4, 4), (2, 2, 2, 2), 8
    V = 256
    U = inputs.random_gauge(dims, 0.3, 1001)
    ctx = lib.Context(lib.default_params(dims=dims, blocks=[block], nvec=[nvec], m0=-0.1, csw=1.0,
                                         inner_prec=prec, use_graphs=graphs))
    ctx.set_gauge(dev(U))
    iv = inputs.setup_vectors(dims, 12, nvec, 0, 1001)
    ctx.setup(dev(iv))
    b = inputs.source(dims, 0)
    D = WilsonClover(U, dims, -0.1, 1.0)
    x = dev(np.zeros_like(b))
    cold = ctx.solve(dev(b), x)
    xs = host(x)
    x0 = xs + 1e-6 * inputs.complex_gaussian(5008, 0, xs.shape)
    for _ in range(3 if graphs else 1):     # graphs: host-driven, capture, replay
        xg = dev(x0)
        warm = ctx.solve_ex(dev(b), xg, zero_guess=0)
        assert warm.converged and warm.true_residual <= 1e-10
        assert warm.outer_iterations < cold.outer_iterations
        got = host(xg)[0].reshape(V, 12)
        assert residual(D(to_grid(got, dims)).reshape(V, 12), b[0].reshape(V, 12)) <= 1e-10
    if prec == 0:
        mg = Multigrid(D, MGParams(blocks=[block], nvecs=[nvec]), [[to_grid(v, dims) for v in iv]])
        xo, info = mg.solve(fields(b, dims, 12)[0], x0=to_grid(x0[0].reshape(V, 12), dims))
        assert abs(warm.outer_iterations - info.iterations) <= 1
        assert rel(got, xo.reshape(V, 12)) < 1e-8
    # a guess that already solves the system comes back unchanged, with no iteration
    xg = dev(host(xg))
    before = host(xg)
    st = ctx.solve_ex(dev(b), xg, zero_guess=0)
    assert st.outer_iterations == 0 and np.array_equal(host(xg), before)
    # zero_guess = 1 ignores x's contents: the cold solve again
    xg = dev(x0)
    st = ctx.solve_ex(dev(b), xg, zero_guess=1)
    assert st.outer_iterations == cold.outer_iterations


def test_solve_from_an_initial_guess_host_buffers(lib):
    dims, block, nvec = (4, 4, 4, 4), (2, 2, 2, 2), 8
    U = inputs.random_gauge(dims, 0.3, 1001)
    ctx = lib.Context(lib.default_params(dims=dims, blocks=[block], nvec=[nvec], m0=-0.1, csw=1.0))
    ctx.set_gauge(U)
    ctx.setup(inputs.setup_vectors(dims, 12, nvec, 0, 1001))
    b = inputs.source(dims, 0)
    x = np.zeros_like(b)
    cold = ctx.solve(b, x)
    x0 = x + 1e-7 * inputs.complex_gaussian(5009, 0, x.shape)
    warm = ctx.solve_ex(b, x0, zero_guess=0)
    assert warm.converged and warm.outer_iterations < cold.outer_iterations
    assert rel(x0, x) < 1e-8


def test_network_checkpoint_round_trip_is_bitwise(lib):
    V = int(np.prod(DIMS))
    U = inputs.random_gauge(DIMS, 0.3, 5010)
    a = _ctx(lib)
    a.set_gauge(dev(U))
    rng = np.random.default_rng(5011)
    W = 0.1 * (rng.normal(size=3456) + 1j * rng.normal(size=3456))
    a.ptc_set_weights(dev(W))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "net.bin")
        a.save_net(path)
        assert os.path.getsize(path) == 8 + 16 + 3456 * 8
        b = _ctx(lib)
        b.set_gauge(dev(U))
        with pytest.raises(lib.WcmgError):
            b.save_net(os.path.join(d, "none.bin"))          # no weights yet
        b.load_net(path)
        wa, wb = dev(np.zeros(3456, dtype=complex)), dev(np.zeros(3456, dtype=complex))
        a.ptc_get_weights(wa)
        b.ptc_get_weights(wb)
        assert np.array_equal(host(wa), host(wb))
        r = inputs.complex_gaussian(5012, 0, (1, V, 4, 3))
        oa, ob = dev(np.zeros_like(r)), dev(np.zeros_like(r))
        a.ptc_forward(dev(r), oa)
        b.ptc_forward(dev(r), ob)
        assert np.array_equal(host(oa), host(ob))
        with open(os.path.join(d, "bad.bin"), "wb") as f:
            f.write(b"WCMGNET1" + bytes(16))
        with pytest.raises(lib.WcmgError) as e:
            b.load_net(os.path.join(d, "bad.bin"))
        assert e.value.code == lib.ERR_ARG


@pytest.mark.parametrize("polls", [0, 1000])
def test_bounded_device_wait_gives_up_and_the_context_stays_usable(lib, polls):
    """Failure detection without a fault: a device-side mbarrier wait that nothing
    completes gives up after its poll limit, sets the context's device-wait word, and the
    call returns WCMG_ERR_TIMEOUT.  The word is cleared: a second self-test times out
    again, and the operators that follow still match the oracle."""
    from oracle.aggregation import Aggregation
    from oracle.coarse import coarsen
    from oracle.lattice import coarse_dims
    ctx = _ctx(lib)
    U = inputs.random_gauge(DIMS, 0.35, 2401)
    ctx.set_gauge(dev(U))
    assert ctx.check_bounded_wait(polls) == lib.ERR_TIMEOUT
    assert ctx.check_bounded_wait(polls) == lib.ERR_TIMEOUT
    with pytest.raises(lib.WcmgError) as e:
        ctx.check_bounded_wait(-1)
    assert e.value.code == lib.ERR_ARG
    V = int(np.prod(DIMS))
    D = WilsonClover(U, DIMS, -0.17, 1.13)
    psi = inputs.complex_gaussian(2402, 0, (1, V, 4, 3))
    out = dev(np.zeros_like(psi))
    ctx.apply_D(dev(psi), out)
    assert rel(host(out)[0], D(fields(psi, DIMS, 12)[0]).reshape(V, 4, 3)) < 1e-12
    raw = inputs.complex_gaussian(2403, 0, (NVEC, V, 12))
    ctx.set_nullvecs(0, dev(raw))
    ctx.coarsen(0)
    cd = coarse_dims(DIMS, BLOCK)
    Vc, nb = int(np.prod(cd)), 2 * NVEC
    op = coarsen(D, Aggregation(DIMS, BLOCK, fields(raw, DIMS, 12)))
    phi = inputs.complex_gaussian(2404, 0, (1, Vc, nb))
    y = dev(np.zeros_like(phi))
    ctx.apply_coarse(1, dev(phi), y, nrhs=1, prec=lib.F64)
    assert rel(host(y)[0], op(fields(phi, cd, nb)[0]).reshape(Vc, nb)) < 1e-12
