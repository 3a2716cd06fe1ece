"""Gauge-equivariant parallel-transport convolution (PTC) network (oracle; test
infrastructure).

The paper has no learned component; this follows the learned coarse-correction
pattern of the benchmark configurations: a small linear network N that maps a
fine residual r to an approximation of the multigrid coarse-grid correction
e = P D_c^-1 P^dag r (Sec. 2.1 operators).  Readings:

  * hops h = 0 (identity), 1 + 2 mu (+mu), 2 + 2 mu (-mu), as for the coarse blocks;
    parallel transport  (T_{+mu} f)(x) = U_mu(x) f(x + mu),
                        (T_{-mu} f)(x) = U_mu(x - mu)^dag f(x - mu),
    so T_{+-mu}^dag = T_{-+mu} and T_0 = 1;
  * one layer: out_i(x) = sum_j sum_h W_{ijh} (T_h in_j)(x) with W_{ijh} a complex
    4x4 spin matrix (acting on spin, the transport acts on colour), no bias and no
    activation, so N stays a fixed linear map (a valid flexible preconditioner);
  * two layers, 1 -> 12 -> 1 spinor fields; weights W1 (12, 1, 9, 4, 4), W2 (1, 12, 9, 4, 4);
  * loss L = ||N(r) - e||^2 / ||e||^2; gradients are Wirtinger derivatives
    dL/d conj(.), for which dL = 2 Re sum conj(grad) * delta.
"""
import numpy as np

from .lattice import shift
from .lattice import to_grid

NHOP = 9


def _dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


class PTC:
    def __init__(self, U_ext, dims):
        self.dims = tuple(dims)
        self.U = np.stack([to_grid(U_ext[mu], dims) for mu in range(4)])  # (4,T,Z,Y,X,3,3)

    def transport(self, f, h):
        """(T_h f), f of shape (T,Z,Y,X,12)."""
        if h == 0:
            return f
        mu, back = (h - 1) // 2, (h - 1) % 2
        g = f.reshape(f.shape[:4] + (4, 3))
        if not back:
            t = np.einsum("...ab,...sb->...sa", self.U[mu], shift(g, mu, +1))
        else:
            t = np.einsum("...ba,...sb->...sa", np.conj(shift(self.U[mu], mu, -1)), shift(g, mu, -1))
        return t.reshape(f.shape)

    def transport_adj(self, g, h):
        """T_h^dag g."""
        if h == 0:
            return g
        mu, back = (h - 1) // 2, (h - 1) % 2
        return self.transport(g, 1 + 2 * mu + (0 if back else 1))

    @staticmethod
    def spin_mul(W, f):
        """(W f)[s, c] = sum_t W[s, t] f[t, c] for a 4x4 spin matrix W."""
        g = f.reshape(f.shape[:4] + (4, 3))
        return np.einsum("st,...tc->...sc", W, g).reshape(f.shape)

    def layer(self, W, inputs):
        nout, nin = W.shape[:2]
        Tin = [[self.transport(inputs[j], h) for h in range(NHOP)] for j in range(nin)]
        outs = []
        for i in range(nout):
            acc = np.zeros_like(inputs[0])
            for j in range(nin):
                for h in range(NHOP):
                    acc = acc + self.spin_mul(W[i, j, h], Tin[j][h])
            outs.append(acc)
        return outs, Tin

    def layer_backward(self, W, Tin, gouts):
        """Given dL/d conj(out_i): dL/d conj(W) and dL/d conj(in_j)."""
        nout, nin = W.shape[:2]
        gW = np.zeros_like(W)
        gin = []
        for j in range(nin):
            acc = np.zeros_like(gouts[0])
            for h in range(NHOP):
                th = Tin[j][h].reshape(Tin[j][h].shape[:4] + (4, 3))
                back = np.zeros_like(gouts[0])
                for i in range(nout):
                    gi = gouts[i].reshape(gouts[i].shape[:4] + (4, 3))
                    gW[i, j, h] = np.einsum("nac,nbc->ab", gi.reshape(-1, 4, 3), np.conj(th).reshape(-1, 4, 3))
                    back = back + self.spin_mul(_dag(W[i, j, h]), gouts[i])
                acc = acc + self.transport_adj(back, h)
            gin.append(acc)
        return gW, gin

    def forward(self, W1, W2, r):
        hidden, T1 = self.layer(W1, [r])
        out, T2 = self.layer(W2, hidden)
        return out[0], (hidden, T1, T2)

    def backward(self, W1, W2, cache, gout):
        hidden, T1, T2 = cache
        gW2, ghid = self.layer_backward(W2, T2, [gout])
        gW1, gin = self.layer_backward(W1, T1, ghid)
        return gW1, gW2, gin[0]

    def loss_and_grad(self, W1, W2, r, e):
        """L = ||N(r) - e||^2 / ||e||^2 and its Wirtinger gradients."""
        n, cache = self.forward(W1, W2, r)
        d = n - e
        ee = float(np.vdot(e.ravel(), e.ravel()).real)
        L = float(np.vdot(d.ravel(), d.ravel()).real) / ee
        gW1, gW2, gr = self.backward(W1, W2, cache, d / ee)
        return L, gW1, gW2, gr


def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam on the real and imaginary parts of complex weights; the real gradient of
    L with respect to (Re w, Im w) is 2 (Re g, Im g) for g = dL/d conj(w)."""
    gr = 2.0 * np.concatenate([g.real.ravel(), g.imag.ravel()])
    m[:] = b1 * m + (1 - b1) * gr
    v[:] = b2 * v + (1 - b2) * gr * gr
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    step = lr * mh / (np.sqrt(vh) + eps)
    n = w.size
    return w - (step[:n] + 1j * step[n:]).reshape(w.shape)
