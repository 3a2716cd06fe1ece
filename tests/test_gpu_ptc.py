"""GPU parity of the learned coarse correction (parallel-transport convolution
network) against the FP64 oracle, its training, and its use inside the solve.
FP32 kernels: 1e-5 relative tolerance against the FP64 oracle."""
import numpy as np
import pytest

from oracle.lattice import to_grid
from oracle.ptc import NHOP, PTC
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, fields, host, rel

pytestmark = pytest.mark.gpu


def weights(seed):
    rng = np.random.default_rng(seed)
    W1 = (rng.normal(size=(12, 1, NHOP, 4, 4)) + 1j * rng.normal(size=(12, 1, NHOP, 4, 4))) * 0.2
    W2 = (rng.normal(size=(1, 12, NHOP, 4, 4)) + 1j * rng.normal(size=(1, 12, NHOP, 4, 4))) * 0.2
    return W1, W2


def packed(W1, W2):
    return np.ascontiguousarray(np.concatenate([W1.ravel(), W2.ravel()]))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 8, 10)])
def test_ptc_forward_and_backward_match_oracle(lib, dims):
    V = int(np.prod(dims))
    U = inputs.random_gauge(dims, 0.3, 3001)
    block = tuple(2 for _ in dims)
    ctx = lib.Context(lib.default_params(dims=dims, blocks=[block], nvec=[4], max_rhs=2))
    ctx.set_gauge(dev(U))
    W1, W2 = weights(3002)
    ctx.ptc_set_weights(dev(packed(W1, W2)))
    back = dev(np.zeros(3456, dtype=complex))
    ctx.ptc_get_weights(back)
    assert rel(host(back), packed(W1, W2)) < 1e-7
    net = PTC(U, dims)
    r = inputs.complex_gaussian(3003, 0, (2, V, 4, 3))
    out = dev(np.zeros_like(r))
    ctx.ptc_forward(dev(r), out, nrhs=2)
    fr = fields(r, dims, 12)
    caches = []
    for q in range(2):
        ref, cache = net.forward(W1, W2, fr[q])
        caches.append(cache)
        assert rel(host(out)[q].reshape(V, 12), ref.reshape(V, 12)) < 1e-5
    g = inputs.complex_gaussian(3004, 0, (2, V, 4, 3))
    gin = dev(np.zeros_like(g))
    gW = dev(np.zeros(3456, dtype=complex))
    ctx.ptc_backward(dev(r), dev(g), gin, gW, nrhs=2)
    gW1 = np.zeros_like(W1); gW2 = np.zeros_like(W2)
    fg = fields(g, dims, 12)
    for q in range(2):
        a1, a2, gr = net.backward(W1, W2, caches[q], fg[q])
        gW1 += a1; gW2 += a2
        assert rel(host(gin)[q].reshape(V, 12), gr.reshape(V, 12)) < 1e-5
    assert rel(host(gW), packed(gW1, gW2)) < 1e-5


DIMS_T = (8, 8, 8, 16)


def setup_small(lib, dims=DIMS_T):
    """Configuration-2 parameters (eps 0.25, m0 -0.2, blocks 4^4, Nvec 24) on 8^3 x 16."""
    p = lib.default_params(dims=dims, blocks=[(4, 4, 4, 4)], nvec=[24], m0=-0.2, csw=1.0, inner_prec=lib.F32,
                           setup_refine_sweeps=2, max_rhs=24)
    ctx = lib.Context(p)
    ctx.set_gauge(dev(inputs.random_gauge(dims, 0.25, 3010)))
    ctx.setup(dev(inputs.setup_vectors(dims, 12, 24, 0, 3010)))
    return ctx


def test_trained_network_gains_over_no_coarse_correction(lib):
    """The learned cycle replaces P D_c^-1 P^dag r by N(r).  With zero weights this is
    the smoother alone; the trained network must need fewer outer iterations, and as
    a warm start of the coarsest GMRES it must not cost coarse iterations."""
    b = inputs.source(DIMS_T, 0)
    ctx = setup_small(lib)
    plain = ctx.solve(dev(b), dev(np.zeros_like(b)))
    ctx.ptc_set_weights(dev(np.zeros(3456, dtype=complex)))
    ctx.set_coarse_mode(lib.COARSE_LEARNED, 0.0)
    zero = ctx.solve(dev(b), dev(np.zeros_like(b)))
    ctx.close()
    ctx = setup_small(lib)
    st = ctx.ptc_train(npairs=24, batch=4, steps=300, lr=1e-2, target_tol=1e-6, seed=5)
    assert st.loss_final < 0.95 * min(1.0, st.loss_initial)
    ctx.set_coarse_mode(lib.COARSE_LEARNED, 0.0)
    trained = ctx.solve(dev(b), dev(np.zeros_like(b)))
    assert zero.converged and trained.converged and trained.true_residual <= 1e-10
    assert trained.outer_iterations < zero.outer_iterations
    ctx.set_coarse_mode(lib.COARSE_WARMSTART)
    warm = ctx.solve(dev(b), dev(np.zeros_like(b)))
    assert warm.converged and warm.learned_cycles > 0
    assert warm.coarse_iterations <= plain.coarse_iterations
    ctx.set_coarse_mode(lib.COARSE_LEARNED, 0.9)
    fb = ctx.solve(dev(b), dev(np.zeros_like(b)))
    assert fb.converged and fb.true_residual <= 1e-10


def test_learned_mode_without_weights_is_state_error(lib):
    ctx = setup_small(lib)
    ctx.set_coarse_mode(lib.COARSE_LEARNED)
    b = inputs.source(DIMS_T, 0)
    with pytest.raises(lib.WcmgError) as e:
        ctx.solve(dev(b), dev(np.zeros_like(b)))
    assert e.value.code == lib.ERR_STATE


def test_training_on_fresh_pools_generalises_and_transfers_to_a_larger_lattice(lib):
    """Pools of pairs are regenerated during training; the held-out loss (a pool never
    trained on) stays below the zero network's 1.  The weights act per site and hop,
    so a network trained on 8^3 x 16 deploys unchanged on 8^3 x 32 (another gauge
    field): there it must still beat the cycle without coarse correction."""
    ctx = setup_small(lib)
    st = ctx.ptc_train(npairs=12, batch=4, steps=240, lr=1e-2, target_tol=1e-6, seed=7, refresh=30)
    assert st.pairs_total == 12 * 8
    assert st.loss_heldout < 0.97 and st.loss_final < 0.97
    W = dev(np.zeros(3456, dtype=complex))
    ctx.ptc_get_weights(W)
    ctx.close()
    big = (8, 8, 8, 32)
    p = lib.default_params(dims=big, blocks=[(4, 4, 4, 4)], nvec=[24], m0=-0.2, csw=1.0, inner_prec=lib.F32,
                           setup_refine_sweeps=2, max_rhs=24)
    out = {}
    for name, w in (("zero", dev(np.zeros(3456, dtype=complex))), ("trained", W)):
        c2 = lib.Context(p)
        c2.set_gauge(dev(inputs.random_gauge(big, 0.25, 3020)))
        c2.setup(dev(inputs.setup_vectors(big, 12, 24, 0, 3020)))
        c2.ptc_set_weights(w)
        c2.set_coarse_mode(lib.COARSE_LEARNED, 0.0)
        b = inputs.source(big, 0)
        out[name] = c2.solve(dev(b), dev(np.zeros_like(b)))
        c2.close()
    assert out["trained"].converged and out["trained"].true_residual <= 1e-10
    assert out["trained"].outer_iterations < out["zero"].outer_iterations
