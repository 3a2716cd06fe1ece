"""Small helpers shared by the tests (no method arithmetic)."""
import numpy as np

from oracle.lattice import to_grid


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def grid_fields(arr, dims):
    """[n][V][...] external -> list of (T,Z,Y,X,ncomp) oracle fields."""
    return [to_grid(a.reshape(a.shape[0], -1), dims) for a in arr]


def vdot(a, b):
    return complex(np.vdot(np.ravel(a), np.ravel(b)))
