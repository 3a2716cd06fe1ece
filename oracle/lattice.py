"""Lattice geometry helpers (oracle; test infrastructure).

Directions mu = 0, 1, 2, 3 are x, y, z, t.  A field of shape (T, Z, Y, X, ...)
stores site (x, y, z, t) at index [t, z, y, x]; boundaries are periodic in all
four directions.
"""
import numpy as np


def axis(mu: int) -> int:
    return 3 - mu


def volume(dims) -> int:
    return int(np.prod(dims))


def to_grid(a: np.ndarray, dims) -> np.ndarray:
    """External [V, ...] (x fastest) -> (T, Z, Y, X, ...)."""
    Lx, Ly, Lz, Lt = dims
    return np.asarray(a).reshape((Lt, Lz, Ly, Lx) + a.shape[1:])


def from_grid(g: np.ndarray) -> np.ndarray:
    return g.reshape((-1,) + g.shape[4:])


def shift(f: np.ndarray, mu: int, sign: int) -> np.ndarray:
    """g(x) = f(x + sign * mu_hat) with periodic wrap."""
    return np.roll(f, -sign, axis=axis(mu))


def coarse_dims(dims, block):
    out = []
    for L, b in zip(dims, block):
        if b <= 0 or L % b:
            raise ValueError(f"extent {L} not divisible by block {b}")
        out.append(L // b)
    return tuple(out)


def to_blocks(f: np.ndarray, block) -> np.ndarray:
    """(T, Z, Y, X, *c) -> (Tc, Zc, Yc, Xc, bt, bz, by, bx, *c)."""
    T, Z, Y, X = f.shape[:4]
    bx, by, bz, bt = block
    rest = f.shape[4:]
    g = f.reshape((T // bt, bt, Z // bz, bz, Y // by, by, X // bx, bx) + rest)
    nr = len(rest)
    return g.transpose((0, 2, 4, 6, 1, 3, 5, 7) + tuple(8 + i for i in range(nr)))


def from_blocks(g: np.ndarray) -> np.ndarray:
    Tc, Zc, Yc, Xc, bt, bz, by, bx = g.shape[:8]
    rest = g.shape[8:]
    nr = len(rest)
    f = g.transpose((0, 4, 1, 5, 2, 6, 3, 7) + tuple(8 + i for i in range(nr)))
    return f.reshape((Tc * bt, Zc * bz, Yc * by, Xc * bx) + rest)


def face_mask(dims, block, mu: int, sign: int) -> np.ndarray:
    """True at fine sites x whose neighbour x + sign*mu_hat lies in another block."""
    Lx, Ly, Lz, Lt = dims
    coord = np.indices((Lt, Lz, Ly, Lx))[axis(mu)]
    b = block[mu]
    return (coord % b == b - 1) if sign > 0 else (coord % b == 0)
