"""The allocation-free block orthonormalisation entry point.

Some callers cannot allocate device memory: all of their device memory belongs to
another allocator (a host framework's caching pool, for example), and a call to
cudaMalloc / cudaFree would synchronise the whole device or fail once that pool
holds the memory.  wcmg_block_orthonormalise_noalloc serves them with a fixed
file-scope working array instead of allocations.

Its output must be the Q factor, with positive real diag(R), of every aggregate's
chirality panel: the same result as the oracle's block orthonormalisation and as
the library's own context path (wcmg_set_nullvecs then wcmg_get_nullvecs).  Two
calls in a row on different inputs check that the shared working array's leftover
contents never leak into a result.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle.aggregation import block_orthonormalise
from oracle.lattice import to_blocks
from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, ext, fields, host, rel

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 4), (2, 2, 2, 2), 8, 61), ((6, 4, 8, 10), (3, 2, 4, 5), 5, 62)]


def _noalloc(lib, vin, vout, dims, block, nvec):
    d = (ctypes.c_int * 4)(*dims)
    b = (ctypes.c_int * 4)(*block)
    return lib.wcmg_block_orthonormalise_noalloc(vin.data_ptr(), vout.data_ptr(), d, b, nvec, None)


def _context_path(lib, raw, dims, block, nvec):
    ctx = lib.Context(lib.default_params(dims=dims, blocks=[block], nvec=[nvec]))
    ctx.set_nullvecs(0, dev(raw))
    out = dev(np.zeros_like(raw))
    ctx.get_nullvecs(0, out)
    ctx.close()
    return host(out)


def _oracle(raw, dims, block):
    V = int(np.prod(dims))
    q = block_orthonormalise(fields(raw.reshape(raw.shape[0], V, 12), dims, 12), block)
    return ext(list(q)).reshape(raw.shape)


def _panels(vecs, dims, block):
    """(chirality, aggregate, rows, nvec) panels of fine fields given as [nvec][V][4][3]."""
    nvec = vecs.shape[0]
    V = int(np.prod(dims))
    vb = np.stack([to_blocks(f, block) for f in fields(vecs.reshape(nvec, V, 12), dims, 12)])
    vb = vb.reshape((nvec, -1, int(np.prod(block)), 12))  # (nvec, aggregate, block site, 12)
    out = []
    for s in range(2):
        part = vb[..., 6 * s:6 * s + 6].reshape(nvec, vb.shape[1], -1)
        out.append(np.moveaxis(part, 0, -1))  # (aggregate, rows, nvec)
    return out


def _check_q_factor(q, raw, dims, block):
    """Q^dag Q = 1 on every aggregate and chirality, and R = Q^dag A upper triangular
    with a positive real diagonal (the unique QR of a full-rank panel)."""
    for Qs, As in zip(_panels(q, dims, block), _panels(raw, dims, block)):
        nvec = Qs.shape[-1]
        G = np.einsum("arj,ark->ajk", np.conj(Qs), Qs)
        assert np.max(np.abs(G - np.eye(nvec))) < 1e-13
        R = np.einsum("arj,ark->ajk", np.conj(Qs), As)
        d = np.diagonal(R, axis1=1, axis2=2)
        scale = np.max(np.abs(R))
        assert np.all(d.real > 0) and np.max(np.abs(d.imag)) < 1e-12 * scale
        assert np.max(np.abs(np.tril(R, -1))) < 1e-12 * scale


def test_noalloc_matches_oracle_and_context_path_two_calls(lib):
    import torch
    raws = [inputs.complex_gaussian(seed, 7, (nvec, int(np.prod(dims)), 4, 3)) for dims, block, nvec, seed in CASES]
    for (dims, block, nvec, _), raw in zip(CASES, raws):   # two calls in a row, different inputs
        out = dev(np.zeros_like(raw))
        assert _noalloc(lib, dev(raw), out, dims, block, nvec) == lib.OK
        torch.cuda.synchronize()
        got = host(out)
        assert rel(got, _oracle(raw, dims, block)) < 1e-12
        assert rel(got, _context_path(lib, raw, dims, block, nvec)) < 1e-12
        _check_q_factor(got, raw, dims, block)
    dims, block, nvec, _ = CASES[0]                          # and the first input again, in place
    buf = dev(raws[0])
    assert _noalloc(lib, buf, buf, dims, block, nvec) == lib.OK
    assert rel(host(buf), _oracle(raws[0], dims, block)) < 1e-12


def test_noalloc_rejects_sizes_beyond_the_fixed_array(lib):
    dims, block, nvec = (8, 8, 8, 8), (2, 2, 2, 2), 8   # 8 * 4096 * 12 > WCMG_NOALLOC_MAX_ELEMS
    assert nvec * 4096 * 12 > lib.NOALLOC_MAX_ELEMS
    x = dev(np.zeros((1, 1), dtype=complex))
    assert _noalloc(lib, x, x, dims, block, nvec) == lib.ERR_ARG
    assert _noalloc(lib, x, x, (4, 4, 4, 6), (2, 2, 2, 4), 4) == lib.ERR_ARG   # 6 % 4 != 0
