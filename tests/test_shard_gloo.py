"""The multi-process path on CPU: two gloo ranks shard the seeded shot stream, and the
timing / count reductions give the slowest rank's time and the job's total."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2406_18655_gb300 import inputs as I
from paper_2406_18655_gb300 import shard as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        h = I.bb72()[0]
        probs = np.full(h.shape[1], 0.05)
        first, count = S.shard(rank, world, 300)
        e = I.sample_errors(9, count, probs, first_shot=first)
        s = I.syndromes(h, e)
        # a rank's local "step time" and work count
        res = S.job_throughput(units_per_rank=count, ms_per_step_local=10.0 + 5.0 * rank)
        q.put((rank, e, s, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(world):
        rank, e, s, res = q.get(timeout=120)
        out[rank] = (e, s, res)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the shards are disjoint, contiguous pieces of the single-process stream
    h = I.bb72()[0]
    e_all = I.sample_errors(9, 600, np.full(h.shape[1], 0.05))
    assert np.array_equal(np.concatenate([out[0][0], out[1][0]]), e_all)
    assert np.array_equal(np.concatenate([out[0][1], out[1][1]]), I.syndromes(h, e_all))
    for r in range(world):
        res = out[r][2]
        assert res["ms_per_step"] == 15.0          # the slowest rank
        assert res["units"] == 600                 # all ranks' shots
        assert abs(res["per_s"] - 600 / 0.015) < 1e-6


def test_single_process_and_bad_requests():
    assert S.shard(0, 1, 10) == (0, 10)
    assert S.job_throughput(10, 2.0)["per_s"] == 5000.0
    for bad in [(2, 2, 1), (-1, 2, 1), (0, 0, 1), (0, 1, -1)]:
        try:
            S.shard(*bad)
        except ValueError:
            continue
        raise AssertionError(bad)
