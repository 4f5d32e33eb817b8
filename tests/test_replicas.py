"""Host-side replica coordination with two gloo ranks on the CPU: the max over
ranks used for timing, barriers, balanced segment shards, and the job rate."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2311_03096_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, offsets, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = replicas.env()
        replicas.barrier()
        ms = replicas.max_over_ranks(10.0 + 5.0 * rank)
        s0, s1 = replicas.shard_segments(offsets, r, w)
        replicas.barrier()
        q.put((r, w, lr, ms, s0, s1))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    off = np.concatenate([[0], np.cumsum(np.random.default_rng(3).integers(1, 5000, 101))])
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, off, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(r[3] == 15.0 for r in res)   # the slowest rank's time
    (a0, a1), (b0, b1) = [(r[4], r[5]) for r in res]
    assert a0 == 0 and a1 == b0 and b1 == len(off) - 1
    share = off[a1] / off[-1]
    assert abs(share - 0.5) < 0.05


def test_shards_cover_all_segments():
    off = np.concatenate([[0], np.cumsum(np.random.default_rng(4).integers(0, 3000, 500))])
    for world in (1, 2, 3, 4, 8):
        cuts = [replicas.shard_segments(off, r, world) for r in range(world)]
        assert cuts[0][0] == 0 and cuts[-1][1] == 500
        assert all(cuts[i][1] == cuts[i + 1][0] for i in range(world - 1))
        sizes = [off[b] - off[a] for a, b in cuts]
        assert max(sizes) - min(sizes) <= 2 * 3000 + 1


def test_job_rate():
    assert replicas.job_rate(1000, 4, 2.0) == 2.0e6
