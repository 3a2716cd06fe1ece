"""Aggregation: block orthonormalisation, prolongation P and restriction P^dag
(oracle; test infrastructure).

Sec. 2.1: the intergrid operators live in Grid's Aggregation class and are built
from near-null vectors found by the setup.  Sec. 2.2: chirality is preserved by
splitting each near-null vector psi_i into its two chiral halves,
    P = [ (1 + gamma5)/2 psi_i , (1 - gamma5)/2 psi_i ],
so the coarse space has nbasis = 2 * Nvec components per aggregate.  Sec. 3: the
restriction is a block inner product over the fine sites of each aggregate
(blockProject).

Readings:
  * Aggregates are hypercubic blocks of the fine lattice (block extents b_mu); the
    coarse lattice is periodic with extents L_mu / b_mu.
  * Column order on a coarse site: first the Nvec chirality-+ columns, then the
    Nvec chirality-- columns, so coarse gamma5 is sigma3 = diag(+1 x Nvec, -1 x Nvec).
  * The chirality of a component is "first half / second half" of the site
    components: spins 0,1 (chiral basis) on the fine level, coarse components
    [0, Nvec) / [Nvec, 2 Nvec) on coarser levels.
  * Block orthonormalisation: for each aggregate and chirality the panel
    [Pi_s psi_1 | ... | Pi_s psi_Nvec] restricted to the aggregate is replaced by
    the Q factor of its QR decomposition with positive real diag(R) (unique for a
    full-rank panel; equals Gram-Schmidt in the order i = 1..Nvec).
"""
import numpy as np

from .lattice import coarse_dims, from_blocks, to_blocks


def block_orthonormalise(vecs, block):
    """vecs: sequence of Nvec fields (T,Z,Y,X,nc).  Returns an array
    (Nvec, T,Z,Y,X,nc) whose chiral halves are orthonormal on every aggregate."""
    V = np.stack([np.asarray(v) for v in vecs])
    nvec, nc = V.shape[0], V.shape[-1]
    half = nc // 2
    Vb = np.stack([to_blocks(v, block) for v in V])  # (nvec, Tc,Zc,Yc,Xc, bt,bz,by,bx, nc)
    cshape = Vb.shape[1:5]
    nsite = int(np.prod(Vb.shape[5:9]))
    out = np.empty_like(Vb)
    for s in range(2):
        part = Vb[..., s * half:(s + 1) * half]
        # panel per coarse site: rows = (block site, component), columns = vector index
        M = part.reshape((nvec,) + cshape + (nsite * half,))
        M = np.moveaxis(M, 0, -1)  # (Tc,Zc,Yc,Xc, rows, nvec)
        Q, R = np.linalg.qr(M)
        d = np.diagonal(R, axis1=-2, axis2=-1)
        if np.any(np.abs(d) == 0):
            raise np.linalg.LinAlgError("rank-deficient aggregate panel")
        Q = Q * (d / np.abs(d))[..., None, :]
        Q = np.moveaxis(Q, -1, 0).reshape(part.shape)
        out[..., s * half:(s + 1) * half] = Q
    return np.stack([from_blocks(o) for o in out])


class Aggregation:
    """Prolongator built from block-orthonormalised near-null vectors."""

    def __init__(self, fine_dims, block, vecs, orthonormalise=True):
        self.fine_dims = tuple(fine_dims)
        self.block = tuple(block)
        self.cdims = coarse_dims(fine_dims, block)
        self.v = block_orthonormalise(vecs, block) if orthonormalise else np.stack(vecs)
        self.nvec = self.v.shape[0]
        self.nc = self.v.shape[-1]
        self.half = self.nc // 2
        self.nbasis = 2 * self.nvec

    def chiral_part(self, f, s):
        out = np.zeros_like(f)
        out[..., s * self.half:(s + 1) * self.half] = f[..., s * self.half:(s + 1) * self.half]
        return out

    def column_field(self, b):
        """Column b of P as a global fine field: Pi_s v_i with (s, i) = divmod(b, Nvec)."""
        s, i = divmod(b, self.nvec)
        return self.chiral_part(self.v[i], s)

    def restrict(self, psi):
        """phi(x_c)[s*Nvec + i] = sum_{x in B(x_c)} <Pi_s v_i(x), Pi_s psi(x)>."""
        pb = to_blocks(psi, self.block)
        out = np.zeros(pb.shape[:4] + (self.nbasis,), dtype=np.complex128)
        for s in range(2):
            sl = slice(s * self.half, (s + 1) * self.half)
            for i in range(self.nvec):
                vb = to_blocks(self.v[i], self.block)
                out[..., s * self.nvec + i] = np.sum(np.conj(vb[..., sl]) * pb[..., sl], axis=(4, 5, 6, 7, 8))
        return out

    def prolong(self, phi):
        """psi(x) = sum_{s,i} Pi_s v_i(x) phi(x_c(x))[s*Nvec + i]."""
        out = np.zeros(self.v.shape[1:], dtype=np.complex128)
        ob = to_blocks(out, self.block)
        for s in range(2):
            sl = slice(s * self.half, (s + 1) * self.half)
            for i in range(self.nvec):
                vb = to_blocks(self.v[i], self.block)
                coef = phi[..., s * self.nvec + i][:, :, :, :, None, None, None, None, None]
                ob[..., sl] += vb[..., sl] * coef
        return from_blocks(ob)
