"""The multi-GPU form is replicas only: every rank searches its own query
batch against its own copy of the index, and the job's time is the slowest
rank's. This checks the host side of that (the rank timing reduction and the
query split bench.py uses) with two gloo ranks on CPU; no GPU is involved."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    nq = 64
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    q0, qn = bench.replica_queries(rank, nq)
    q = synth.sift_like_10m().mix.queries(qn, start=q0)
    out.put((rank, ms, q0, qn, q.sum(dtype=np.float64)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time_and_own_batches():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time
    assert [r[1] for r in res] == [15.0, 15.0]
    # disjoint query batches, and each is the synthetic generator's own rows
    import synth
    assert [(r[2], r[3]) for r in res] == [(0, 64), (64, 64)]
    full = synth.sift_like_10m().mix.queries(128)
    assert res[0][4] == full[:64].sum(dtype=np.float64)
    assert res[1][4] == full[64:].sum(dtype=np.float64)
    assert res[0][4] != res[1][4]


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_queries(0, 100) == (0, 100)
