"""Helpers of the GPU parity tests: build contexts, move arrays, call the oracle."""
import numpy as np

from oracle.lattice import to_grid


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    return t.cpu().numpy()


def rel_norm(a, b):
    """The 2-norm ratio ||a - b|| / ||b|| alone (for claims stated in that norm)."""
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def residual(Dx, b):
    """True relative residual ||b - D x|| / ||b|| (2-norm over the whole field): the
    stopping test of the solver, checked with the oracle's D."""
    Dx = np.asarray(Dx); b = np.asarray(b)
    return float(np.linalg.norm((b - Dx).ravel()) / np.linalg.norm(b.ravel()))


def rel(a, b):
    """Relative error of `a` against the reference `b`, the larger of two measures:
    the 2-norm ratio ||a - b|| / ||b|| over the whole array, and the element-wise
    ratio max|a - b| / max|b| taken separately for every index of the leading axis
    (every rhs, vector, direction or slice) and maximised over them.  The second
    fails a systematic error confined to a few sites, one face or one chirality,
    which a whole-field 2-norm can average away."""
    a = np.asarray(a); b = np.asarray(b)
    assert a.shape == b.shape, (a.shape, b.shape)
    d = np.abs(a - b)
    norm = float(np.linalg.norm(d.ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
    if b.ndim >= 2 and b.shape[0] > 1:
        dm = d.reshape(b.shape[0], -1).max(axis=1)
        bm = np.abs(b).reshape(b.shape[0], -1).max(axis=1)
        sup = float(np.max(dm / np.maximum(bm, 1e-300)))
    else:
        sup = float(d.max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0
    return max(norm, sup)


def fields(arr, dims, nc):
    V = int(np.prod(dims))
    return [to_grid(np.asarray(a).reshape(V, nc), dims) for a in arr]


def ext(fields_list):
    """list of (T,Z,Y,X,nc) -> external [n][V][nc]"""
    return np.ascontiguousarray(np.stack([f.reshape(-1, f.shape[-1]) for f in fields_list]))
