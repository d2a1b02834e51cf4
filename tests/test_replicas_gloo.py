"""Multi-GPU replicas, host logic on CPU: two gloo ranks (world size 2).

The sampling path shards by sample index: each rank draws its own rows of the same Philox stream, so
there is no collective on the data path; the only cross-rank operations are a barrier and the
max-over-ranks of the timed region.  Checked here: the rank/step row ranges tile the sample space
without overlap, the max reduction, and that two ranks sampling disjoint ranges with the oracle
reproduce one rank sampling the union (the property the device path relies on).
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      BENCH_BACKEND="gloo")
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import gen
    import oracle

    r, w, _ = bench.dist_setup()
    assert (r, w) == (rank, ws)
    rows, steps = 64, 3
    ranges = [(bench.step_rows(i, r, w, rows), rows) for i in range(steps)]
    t = bench.max_over_ranks(float(10 + rank), w)
    bench.barrier(w)
    b, ts, _ = gen.mps_tensors(10, 3, 8, base_seed=3)
    mine = {n0: oracle.sample(b, ts, 99, n, n0=n0)[0] for n0, n in ranges}
    gathered = [None] * w
    dist.all_gather_object(gathered, {"ranges": ranges, "t": t, "samples": mine})
    if rank == 0:
        out.put(gathered)
    dist.destroy_process_group()


def test_two_replicas_tile_the_sample_space():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(g["t"] == 11.0 for g in gathered)  # max over ranks
    spans = sorted(n0 for g in gathered for n0, _ in g["ranges"])
    assert spans == [64 * i for i in range(6)]  # disjoint, contiguous tiling
    import gen
    import oracle

    b, ts, _ = gen.mps_tensors(10, 3, 8, base_seed=3)
    union, _ = oracle.sample(b, ts, 99, 6 * 64)
    for g in gathered:
        for n0, smp in g["samples"].items():
            assert np.array_equal(smp, union[n0:n0 + 64])
