"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the multigrid method's arithmetic: it only draws
numbers.  Both sides receive its output as plain arrays, so neither side needs a
random-number generator of its own and the two never disagree on inputs.

Generator (counter based, host only):
  * SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014) applied to the counter
        c = seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03 + index  (mod 2**64)
  * uniform double u = (out >> 11) * 2**-53 in [0, 1)
  * normals by Box-Muller from the pair (u[2k], u[2k+1]).

Gauge links: U = exp(i * eps * X) with X = sum_a xi_a lambda_a (Gell-Mann
lambda_a, xi_a ~ N(0,1) iid per link: a unit Gaussian in the Gell-Mann basis of
traceless Hermitian matrices, E tr X^2 = 16), exponentiated through the eigen-
decomposition of the Hermitian X and re-unitarised (Gram-Schmidt on rows 0-1,
row 2 = conj(row0 x row1)) so that U^dagger U = 1 and det U = 1 to rounding.
With this normalisation the bare masses of the benchmark configurations
(eps, m0) = (0.3, -0.1), (0.25, -0.2), (0.2, -0.25) all lie above the critical
mass (smallest Re(lambda) of D on 4^4: 0.62, 0.29, 0.058).

Layouts (external, lexicographic site index s = x + Lx*(y + Ly*(z + Lz*t))):
  gauge  : complex128 [4][V][3][3]   U_mu(x), the link x -> x + mu
  spinor : complex128 [V][4][3]      (spin-major, colour-minor)
  coarse : complex128 [V_c][ncomp]
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from counter (seed, stream, offset + i)."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64(seed % 2**64) * _GOLDEN + np.uint64(stream % 2**64) * _STREAM
        c = base + idx
    out = _splitmix64(c)
    return (out >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles (Box-Muller on consecutive uniform pairs)."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def complex_gaussian(seed: int, stream: int, shape) -> np.ndarray:
    """Complex array with independent N(0,1) real and imaginary parts."""
    n = int(np.prod(shape))
    z = normal(seed, stream, 2 * n)
    return (z[0::2] + 1j * z[1::2]).reshape(shape)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_a, shape (8, 3, 3)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j; l[1][1, 0] = 1j
    l[2][0, 0] = 1; l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j; l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j; l[6][2, 1] = 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return l


def _reunitarise(U: np.ndarray) -> np.ndarray:
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _links(eps: float, seed: int, start: int, count: int) -> np.ndarray:
    """Links start .. start + count - 1 (flat index mu * V + s) of random_gauge.

    Link n takes the normals 8n .. 8n + 7 of stream 0, which Box-Muller makes from
    the uniforms 8n .. 8n + 7 (four whole pairs), so any range of links comes out
    exactly as in one pass over all of them."""
    u = uniform(seed, 0, 8 * count, offset=8 * start)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    z = np.empty(8 * count)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    X = np.einsum("na,aij->nij", z.reshape(count, 8), gell_mann())
    w, Q = np.linalg.eigh(X)
    U = np.einsum("nij,nj,nkj->nik", Q, np.exp(1j * eps * w), np.conj(Q))
    return _reunitarise(U)


def _links_job(a):
    return _links(*a)


def random_gauge(dims, eps: float, seed: int, workers: int = 0) -> np.ndarray:
    """SU(3) links U_mu(x) = exp(i eps X), external layout [4][V][3][3].

    workers > 1: the links are computed in contiguous ranges by that many spawned
    processes (identical values: every link depends on its own counters only)."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    n = 4 * V
    if workers <= 1 or n < (1 << 20):
        return _links(eps, seed, 0, n).reshape(4, V, 3, 3)
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    chunk = -(-n // (4 * workers))
    jobs = [(eps, seed, s, min(chunk, n - s)) for s in range(0, n, chunk)]
    out = np.empty((n, 3, 3), dtype=np.complex128)
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for (_, _, s, c), part in zip(jobs, ex.map(_links_job, jobs)):
            out[s:s + c] = part
    return out.reshape(4, V, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3)).copy()


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix Omega(x) per site, shape [V][3][3]."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    xi = normal(seed, 7, V * 8).reshape(V, 8)
    X = np.einsum("na,aij->nij", xi, gell_mann() / 2.0)
    w, Q = np.linalg.eigh(X)
    U = np.einsum("nij,nj,nkj->nik", Q, np.exp(2j * w), np.conj(Q))
    return _reunitarise(U)


def source(dims, seed: int = 0, nrhs: int = 1, stream: int = 0) -> np.ndarray:
    """Gaussian fine source(s), [nrhs][V][4][3] complex128."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    return complex_gaussian(seed, stream, (nrhs, V, 4, 3))


def setup_vectors(dims, ncomp: int, nvec: int, level: int, seed: int) -> np.ndarray:
    """Initial near-null candidates of one level, [nvec][V_level][ncomp] complex128.

    Vector i of level l uses stream 1 + 1000*l + i."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    return np.stack([complex_gaussian(seed, 1 + 1000 * level + i, (V, ncomp)) for i in range(nvec)])
