"""The N > 1 host path of bench.py on CPU: world_size-2 gloo ranks (no GPU).

The scorer shards by file with no data-path collective (replicas); what runs
across ranks is the timing: a barrier, the slowest rank's time (all_reduce
MAX) and the whole-job rate.  A sharded fit would exchange only the integer
class counts, whose sum is exact; that merge is checked here too, with the
oracle's counts on each rank's shard."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        import synth
        out = {}
        # slowest rank's time and the job's rate
        dist.barrier()
        ms = [3.5, 4.25][rank]
        out["max_ms"] = bench.max_over_ranks(ms)
        out["rate"] = bench.job_rate(1000, out["max_ms"], world)
        # exact merge of per-shard class counts (the exchange of a sharded fit)
        n, F = 600, 32
        p = synth.dirichlet_profiles(5, 2, F, 0.2)
        y = synth.labels_bernoulli(6, n)
        T = synth.file_totals(7, n, 6.0, 1.0)
        X = synth.count_rows(8, p, y, T, 65535, out_dtype="float32").numpy()
        lo, hi = rank * n // world, (rank + 1) * n // world
        m = oracle.mn_fit(X[lo:hi], y[lo:hi], 2)
        c = torch.from_numpy(m["counts"].astype(np.int64))
        nc = torch.from_numpy(m["nc"].astype(np.int64))
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        dist.all_reduce(nc, op=dist.ReduceOp.SUM)
        full = oracle.mn_fit(X, y, 2)
        out["counts_equal"] = bool((c.numpy() == full["counts"].astype(np.int64)).all())
        out["nc_equal"] = bool((nc.numpy() == full["nc"].astype(np.int64)).all())
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_merge():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert res[r]["max_ms"] == 4.25
        assert res[r]["rate"] == pytest.approx(2 * 1000 / 4.25e-3)
        assert res[r]["counts_equal"] and res[r]["nc_equal"]


def test_single_process_helpers():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_rate(10, 2.0, 4) == pytest.approx(20000.0)
