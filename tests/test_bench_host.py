"""Host-side logic of bench.py's multi-rank path (barrier, max/sum over ranks,
replica timing) on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, l = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    bench.barrier(dist)
    mx = bench.max_over_ranks(dist, 10.0 + r)
    sm = bench.sum_over_ranks(dist, 3.0)
    bench.barrier(dist)
    q.put((r, w, mx, sm))
    dist.destroy_process_group()


def test_two_rank_reductions_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert out == [(0, 2, 11.0, 6.0), (1, 2, 11.0, 6.0)]


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(None, 4.5) == 4.5
    assert bench.sum_over_ranks(None, 4.5) == 4.5


def test_oracle_model_one_core():
    """cpu_baseline.one_core: the oracle's operator model timed in a child process with one
    BLAS / OpenMP thread.  The child reports one core used, and its value is the model's
    sum over the operators it timed (here a small count vector on the 16^3x32 workload)."""
    import bench
    counts = {"apply": [2, 3, 0, 0], "restrict": [1, 1, 0, 0], "prolong": [1, 1, 0, 0], "ortho": [1, 0, 0, 0],
              "coarsen": [1, 0, 0, 0]}
    one = bench.oracle_model_one_core(counts, "c2")
    assert one is not None
    assert one["cores"] == 1 and one["cores_measured"] == 1
    total, _ = bench.model_time(one["seconds_per_call"], counts, dict(bench.WORKLOADS["c2"]))
    assert one["value"] == pytest.approx(total, abs=0.5)
    assert one["value"] > 0
