"""The allocation-free block orthonormalisation entry point (for callers that
cannot allocate device memory because their device memory belongs to another
allocator) must return what the context-based path returns: wcmg_set_nullvecs
followed by wcmg_get_nullvecs.  Two calls in a row on different inputs check
that the shared working array's leftover contents do not leak into a result.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1904_08678_gb300 import inputs
from tests.gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 4), (2, 2, 2, 2), 8, 61), ((6, 4, 8, 10), (3, 2, 4, 5), 5, 62)]


def _noalloc(lib, vin, vout, dims, block, nvec):
    d = (ctypes.c_int * 4)(*dims)
    b = (ctypes.c_int * 4)(*block)
    return lib.wcmg_block_orthonormalise_noalloc(vin.data_ptr(), vout.data_ptr(), d, b, nvec, None)


def _reference(lib, raw, dims, block, nvec):
    ctx = lib.Context(lib.default_params(dims=dims, blocks=[block], nvec=[nvec]))
    ctx.set_nullvecs(0, dev(raw))
    out = dev(np.zeros_like(raw))
    ctx.get_nullvecs(0, out)
    ctx.close()
    return host(out)


def test_noalloc_matches_context_path_two_calls(lib):
    import torch
    raws = [inputs.complex_gaussian(seed, 7, (nvec, int(np.prod(dims)), 4, 3)) for dims, block, nvec, seed in CASES]
    refs = [_reference(lib, r, c[0], c[1], c[2]) for r, c in zip(raws, CASES)]
    for (dims, block, nvec, _), raw, ref in zip(CASES, raws, refs):   # two calls in a row, different inputs
        out = dev(np.zeros_like(raw))
        assert _noalloc(lib, dev(raw), out, dims, block, nvec) == lib.OK
        torch.cuda.synchronize()
        assert rel(host(out), ref) < 1e-12
    dims, block, nvec, _ = CASES[0]                                   # and the first input again, in place
    buf = dev(raws[0])
    assert _noalloc(lib, buf, buf, dims, block, nvec) == lib.OK
    assert rel(host(buf), refs[0]) < 1e-12


def test_noalloc_rejects_sizes_beyond_the_fixed_array(lib):
    dims, block, nvec = (8, 8, 8, 8), (2, 2, 2, 2), 8   # 8 * 4096 * 12 > WCMG_NOALLOC_MAX_ELEMS
    assert nvec * 4096 * 12 > lib.NOALLOC_MAX_ELEMS
    x = dev(np.zeros((1, 1), dtype=complex))
    assert _noalloc(lib, x, x, dims, block, nvec) == lib.ERR_ARG
    assert _noalloc(lib, x, x, (4, 4, 4, 6), (2, 2, 2, 4), 4) == lib.ERR_ARG   # 6 % 4 != 0
