"""Pins of the oracle's parallel-transport convolution network (learned coarse
correction): transport adjointness and covariance, gauge and translation
equivariance of the network, linearity, and Wirtinger gradients against central
finite differences in FP64."""
import numpy as np
import pytest

from oracle.lattice import to_grid
from oracle.ptc import NHOP, PTC, adam_step
from paper_1904_08678_gb300 import inputs
from tests.helpers import rel, vdot

DIMS = (4, 2, 4, 6)


def field(seed, dims=DIMS):
    V = int(np.prod(dims))
    return to_grid(inputs.complex_gaussian(seed, 3, (V, 12)), dims)


def weights(seed):
    rng = np.random.default_rng(seed)
    W1 = (rng.normal(size=(12, 1, NHOP, 4, 4)) + 1j * rng.normal(size=(12, 1, NHOP, 4, 4))) * 0.2
    W2 = (rng.normal(size=(1, 12, NHOP, 4, 4)) + 1j * rng.normal(size=(1, 12, NHOP, 4, 4))) * 0.2
    return W1, W2


def gauge_rotate(U, Om, dims):
    Omg = to_grid(Om, dims)
    V = Om.shape[0]
    Up = np.empty_like(U)
    for mu in range(4):
        Up[mu] = (Omg @ to_grid(U[mu], dims) @ np.conj(np.swapaxes(np.roll(Omg, -1, axis=3 - mu), -1, -2))).reshape(V, 3, 3)
    rot = lambda f: np.einsum("...ab,...sb->...sa", Omg, f.reshape(f.shape[:4] + (4, 3))).reshape(f.shape)
    return Up, rot


def test_transport_free_field_is_a_shift():
    net = PTC(inputs.unit_gauge(DIMS), DIMS)
    f = field(1)
    for mu in range(4):
        assert np.array_equal(net.transport(f, 1 + 2 * mu), np.roll(f, -1, axis=3 - mu))
        assert np.array_equal(net.transport(f, 2 + 2 * mu), np.roll(f, 1, axis=3 - mu))


def test_transport_adjoint_identity():
    net = PTC(inputs.random_gauge(DIMS, 0.4, 5), DIMS)
    f, g = field(2), field(3)
    for h in range(NHOP):
        lhs = vdot(g, net.transport(f, h))
        rhs = vdot(net.transport_adj(g, h), f)
        assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_network_gauge_equivariance():
    U = inputs.random_gauge(DIMS, 0.4, 6)
    Om = inputs.random_gauge_transform(DIMS, 7)
    Up, rot = gauge_rotate(U, Om, DIMS)
    W1, W2 = weights(8)
    r = field(4)
    n1, _ = PTC(U, DIMS).forward(W1, W2, r)
    n2, _ = PTC(Up, DIMS).forward(W1, W2, rot(r))
    assert rel(n2, rot(n1)) < 1e-13


def test_network_translation_equivariance():
    U = inputs.random_gauge(DIMS, 0.4, 9)
    W1, W2 = weights(10)
    r = field(5)
    net = PTC(U, DIMS)
    n, _ = net.forward(W1, W2, r)
    # shift the whole configuration by one site in y and two in t
    sh = lambda a, lead=0: np.roll(np.roll(a, 1, axis=lead + 2), 2, axis=lead + 0)
    Ug = np.stack([to_grid(U[mu], DIMS) for mu in range(4)])
    Us = np.stack([sh(Ug[mu]) for mu in range(4)]).reshape(4, -1, 3, 3)
    ns, _ = PTC(Us, DIMS).forward(W1, W2, sh(r))
    assert rel(ns, sh(n)) < 1e-14


def test_network_is_linear():
    net = PTC(inputs.random_gauge(DIMS, 0.4, 11), DIMS)
    W1, W2 = weights(12)
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    r1, r2 = field(6), field(7)
    lhs, _ = net.forward(W1, W2, a * r1 + b * r2)
    n1, _ = net.forward(W1, W2, r1)
    n2, _ = net.forward(W1, W2, r2)
    assert rel(lhs, a * n1 + b * n2) < 1e-13


@pytest.mark.parametrize("which", ["W1", "W2", "r"])
def test_gradients_match_central_finite_differences(which):
    dims = (2, 2, 2, 4)
    net = PTC(inputs.random_gauge(dims, 0.4, 13), dims)
    W1, W2 = weights(14)
    r, e = field(8, dims), field(9, dims)
    L, gW1, gW2, gr = net.loss_and_grad(W1, W2, r, e)
    rng = np.random.default_rng(15)
    h = 1e-6
    target = {"W1": W1, "W2": W2, "r": r}[which]
    grad = {"W1": gW1, "W2": gW2, "r": gr}[which]
    for _ in range(3):
        d = rng.normal(size=target.shape) + 1j * rng.normal(size=target.shape)

        def L_at(t):
            args = {"W1": W1, "W2": W2, "r": r}
            args[which] = t
            return net.loss_and_grad(args["W1"], args["W2"], args["r"], e)[0]

        fd = (L_at(target + h * d) - L_at(target - h * d)) / (2 * h)
        an = 2.0 * np.real(np.vdot(grad.ravel(), d.ravel()))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_adam_reduces_loss_on_a_fixed_pair():
    dims = (2, 2, 2, 4)
    net = PTC(inputs.random_gauge(dims, 0.3, 16), dims)
    W1, W2 = weights(17)
    r = field(10, dims)
    e = net.forward(*weights(18), r)[0]  # a target the network can represent
    m1 = np.zeros(2 * W1.size); v1 = np.zeros_like(m1)
    m2 = np.zeros(2 * W2.size); v2 = np.zeros_like(m2)
    L0 = net.loss_and_grad(W1, W2, r, e)[0]
    for t in range(1, 41):
        L, g1, g2, _ = net.loss_and_grad(W1, W2, r, e)
        W1 = adam_step(W1, g1, m1, v1, t, lr=1e-2)
        W2 = adam_step(W2, g2, m2, v2, t, lr=1e-2)
    assert net.loss_and_grad(W1, W2, r, e)[0] < 0.5 * L0
