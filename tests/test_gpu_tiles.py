"""Launch shapes of the nine-point coarse apply (Sec. 2.1 Mdiag + Mdir, K4/K4m)
and the autotuner that picks among them.

With small-integer links and vectors every product and partial sum is exact in
FP32 (and in BF16/FP16 storage), so EVERY launch shape must reproduce the FP64
oracle bit for bit: any indexing slip in any shape fails."""
import numpy as np
import pytest

from oracle.coarse import CoarseOperator
from oracle.lattice import coarse_dims, to_grid
from tests.gpu_util import dev, fields, host

pytestmark = pytest.mark.gpu

DIMS, BLOCK, NVEC = (8, 8, 8, 8), (2, 2, 2, 2), 24


def stream_fits(lk, nb, rows, stages):
    """Shared memory of the streaming one-rhs kernel (kind 3) within its 200 KiB limit."""
    ld = (9 * nb + 3) // 4 * 4
    lb, vb = {"f64": (16, 16), "f32": (8, 8), "bf16": (4, 8), "f16": (4, 8)}[lk]
    r128 = lambda x: (x + 127) // 128 * 128
    return 2 * r128(ld * vb) + stages * r128(rows * ld * lb) <= 200 * 1024


def mma4_fits(nb, ntile, mm, stages):
    """Shared memory of the bulk-copy tensor-core kernel (kind 4) within its 220 KiB limit."""
    r1k = lambda x: (x + 1023) // 1024 * 1024
    a = r1k(nb // 4 * nb * 16 + max(mm - nb, 0) * 16)
    b = r1k(nb // 4 * 2 * ntile * 16)
    return stages * (a + b) <= 220 * 1024


def candidate_tiles(nrhs, lk, nb):
    """Shapes the library's autotuner times, plus extreme valid ones."""
    t = []
    if nrhs == 1:
        t += [dict(kind=0, threads=th, parts=p) for th in (256, 512) for p in (1, 2, 4, 8)]
        t += [dict(kind=0, threads=64, parts=nb), dict(kind=0, threads=96, parts=3)]
        if lk != "f64":  # two link rows in flight per warp (rows of at most 8 chunks per lane)
            t += [dict(kind=0, threads=th, parts=p, stages=2) for th, p in ((256, 1), (512, 2), (96, 5), (64, nb))]
        t += [dict(kind=1, rhs_per_cta=1, parts=p) for p in (1, 2, 4, 8, 16, nb)]
        # streaming pipeline: the autotuner's shapes, a ragged last chunk (48 % 5, 48 % 7)
        # and the shallowest / deepest pipelines
        shapes = [(th, cr, st) for th in (256, 512) for cr in (8, 16) for st in (3, 4, 6)]
        shapes += [(128, 5, 2), (512, 3, 8), (256, 7, 5), (128, nb, 2)]
        ld = (9 * nb + 3) // 4 * 4
        t += [dict(kind=3, threads=th, parts=cr, stages=st) for th, cr, st in shapes
              if stream_fits(lk, nb, cr, st) and 4 * th >= ld]
    else:
        t += [dict(kind=1, rhs_per_cta=rr, parts=p) for rr in (1, 4, 8) if rr <= nrhs or rr == 4
              for p in (0, 1, 2, 4, 8, 16)]
        if lk == "bf16":
            t += [dict(kind=2, ntile=n) for n in (16, 32, 48, 64) if n <= (nrhs + 15) // 16 * 16]
            # bulk-copy tensor cores: both MMA heights, rhs tiles from 8 (many tiles, a
            # ragged last one) to 64, shallow and deep pipelines
            t += [dict(kind=4, threads=mm, ntile=n, stages=st) for mm in (64, 128) for n in (8, 16, 40, 64)
                  for st in (2, 4, 6) if n <= max(8, (nrhs + 7) // 8 * 8) and mma4_fits(nb, n, mm, st)]
            # one TMEM accumulator (the next item's MMAs wait for the epilogue)
            t += [dict(kind=4, threads=64, ntile=n, stages=st, parts=1) for n in (8, 40) for st in (2, 3)
                  if n <= max(8, (nrhs + 7) // 8 * 8) and mma4_fits(nb, n, 64, st)]
    return t


def ctx_with_int_links(lib, prec, link_prec, max_rhs, seed=91, **kw):
    cd = coarse_dims(DIMS, BLOCK)
    Vc, nb = int(np.prod(cd)), 2 * NVEC
    rng = np.random.default_rng(seed)
    A = (rng.integers(-3, 4, size=(9, Vc, nb, nb)) + 1j * rng.integers(-3, 4, size=(9, Vc, nb, nb))).astype(complex)
    p = lib.default_params(dims=DIMS, blocks=[BLOCK], nvec=[NVEC], max_rhs=max_rhs, inner_prec=prec,
                           coarse_link_prec=link_prec, **kw)
    ctx = lib.Context(p)
    ctx.set_coarse_links(1, dev(A))
    op = CoarseOperator(np.stack([to_grid(A[d], cd) for d in range(9)]), cd)
    return ctx, op, rng, cd, Vc, nb


def int_phi(rng, nrhs, Vc, nb):
    return (rng.integers(-2, 3, size=(nrhs, Vc, nb)) + 1j * rng.integers(-2, 3, size=(nrhs, Vc, nb))).astype(complex)


CASES = [("f64", 1), ("f64", 5), ("f32", 1), ("f32", 6), ("bf16", 1), ("bf16", 8), ("bf16", 37), ("f16", 3)]


@pytest.mark.parametrize("lk,nrhs", CASES)
def test_every_launch_shape_is_exact(lib, lk, nrhs):
    prec = lib.F64 if lk == "f64" else lib.F32
    lp = {"f64": lib.F32, "f32": lib.F32, "bf16": lib.BF16, "f16": lib.F16}[lk]
    ctx, op, rng, cd, Vc, nb = ctx_with_int_links(lib, prec, lp, 40)
    phi = int_phi(rng, nrhs, Vc, nb)
    want = [op(f).reshape(Vc, nb) for f in fields(phi, cd, nb)]
    tiles = candidate_tiles(nrhs, lk, nb)
    assert tiles
    for t in tiles:
        ctx.set_coarse_tile(1, nrhs, prec, **t)
        assert ctx.get_coarse_tile(1, nrhs, prec)["source"] == 2
        out = dev(np.zeros_like(phi))
        ctx.apply_coarse(1, dev(phi), out, nrhs=nrhs, prec=prec)
        got = host(out)
        for r in range(nrhs):
            assert np.array_equal(got[r], want[r]), (t, r)
    ctx.set_coarse_tile(1, nrhs, prec, kind=-1)
    assert ctx.get_coarse_tile(1, nrhs, prec)["source"] == 0


@pytest.mark.parametrize("lk,nrhs", [("f32", 1), ("f32", 24), ("bf16", 16), ("f64", 1)])
def test_autotuner_times_candidates_and_keeps_the_fastest(lib, lk, nrhs):
    prec = lib.F64 if lk == "f64" else lib.F32
    lp = lib.BF16 if lk == "bf16" else lib.F32
    ctx, op, rng, cd, Vc, nb = ctx_with_int_links(lib, prec, lp, 40, autotune=1)
    t = ctx.tune_coarse(1, nrhs, prec)
    assert t["source"] == 1 and t["candidates"] > 5
    assert 0.0 < t["us"] <= t["us_default"]
    assert ctx.get_coarse_tile(1, nrhs, prec) == t
    phi = int_phi(rng, nrhs, Vc, nb)
    out = dev(np.zeros_like(phi))
    ctx.apply_coarse(1, dev(phi), out, nrhs=nrhs, prec=prec)
    got = host(out)
    for r, f in enumerate(fields(phi, cd, nb)):
        assert np.array_equal(got[r], op(f).reshape(Vc, nb))


def test_autotune_on_first_use_inside_a_graph_solve(lib):
    from paper_1904_08678_gb300 import inputs
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    p = lib.default_params(dims=dims, blocks=[block], nvec=[8], m0=-0.1, csw=1.0, inner_prec=lib.F32,
                           use_graphs=1, autotune=1)
    ctx = lib.Context(p)
    ctx.set_gauge(dev(inputs.random_gauge(dims, 0.3, 1051)))
    ctx.setup(dev(inputs.setup_vectors(dims, 12, 8, 0, 1051)))
    b = inputs.source(dims, 0)
    sts = [ctx.solve(dev(b), dev(np.zeros_like(b))) for _ in range(3)]
    assert all(s.converged and s.true_residual <= 1e-10 for s in sts)
    assert [s.graph for s in sts] == [0, 1, 1]
    assert ctx.get_coarse_tile(1, 1, lib.F32)["source"] == 1
    # forcing another shape invalidates the captured graph; the next solve recaptures
    ctx.set_coarse_tile(1, 1, lib.F32, kind=1, rhs_per_cta=1, parts=2)
    st = ctx.solve(dev(b), dev(np.zeros_like(b)))
    assert st.graph == 1 and st.converged and abs(st.outer_iterations - sts[-1].outer_iterations) <= 1


def test_invalid_tiles_are_rejected(lib):
    ctx, *_ = ctx_with_int_links(lib, lib.F32, lib.F32, 8)
    bad = [(1, dict(kind=2, ntile=16)),                 # tensor cores need BF16 links
           (4, dict(kind=0, threads=512, parts=1)),     # one-rhs kernel with 4 rhs
           (4, dict(kind=1, rhs_per_cta=3, parts=1)),   # no such rhs tile
           (1, dict(kind=0, threads=48, parts=1)),      # threads not a multiple of 32
           (1, dict(kind=0, threads=512, parts=0)),
           (1, dict(kind=3, threads=256, parts=8, stages=1)),   # a pipeline needs >= 2 stages
           (1, dict(kind=0, threads=256, parts=1, stages=3)),   # one or two rows in flight
           (1, dict(kind=3, threads=96, parts=8, stages=4)),    # 128, 256 or 512 threads
           (4, dict(kind=3, threads=256, parts=8, stages=4)),   # one rhs only
           (1, dict(kind=3, threads=256, parts=48, stages=8)),  # beyond the shared-memory limit
           (8, dict(kind=4, threads=128, ntile=16, stages=4)),  # tensor cores need BF16 links
           (1, dict(kind=7))]
    for nrhs, t in bad:
        with pytest.raises(lib.WcmgError) as e:
            ctx.set_coarse_tile(1, nrhs, lib.F32, **t)
        assert e.value.code == lib.ERR_ARG, t


def test_autotuner_cold_mode_times_streamed_links(lib):
    """cold = 1: every timed apply follows an L2-evicting scratch write; the choice is
    still a valid shape that reproduces the oracle exactly."""
    ctx, op, rng, cd, Vc, nb = ctx_with_int_links(lib, lib.F32, lib.F32, 8)
    t = ctx.tune_coarse(1, 1, lib.F32, cold=1)
    assert t["source"] == 1 and t["candidates"] > 5 and 0.0 < t["us"] <= t["us_default"]
    phi = int_phi(rng, 1, Vc, nb)
    out = dev(np.zeros_like(phi))
    ctx.apply_coarse(1, dev(phi), out, nrhs=1, prec=lib.F32)
    assert np.array_equal(host(out)[0], op(fields(phi, cd, nb)[0]).reshape(Vc, nb))
    with pytest.raises(lib.WcmgError) as e:
        ctx.tune_coarse(1, 1, lib.F32, cold=2)
    assert e.value.code == lib.ERR_ARG
