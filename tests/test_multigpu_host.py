"""Multi-GPU host logic on CPU: gloo ranks (world size 2) reduce timing and work; the
environment partition is contiguous, complete and balanced by box count."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2207_06649_b300 import multigpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "ran" for 1 + r seconds and did 100 * (r + 1) env-steps
    t, w = multigpu.reduce_job(1.0 + rank, 100.0 * (rank + 1), device="cpu")
    q.put((rank, t, w, multigpu.rank_seed(3, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, w, seed in res:
        assert t == 2.0 and w == 300.0
    assert res[0][3] != res[1][3]


def test_single_process_reduction_is_identity():
    assert multigpu.reduce_job(1.5, 7.0) == (1.5, 7.0)


def test_partition_is_contiguous_complete_and_balanced():
    rng = np.random.default_rng(0)
    counts = rng.integers(5, 41, size=4096)
    for world in (1, 2, 4, 8):
        off = multigpu.partition_envs(counts, world)
        assert off[0] == 0 and off[-1] == len(counts) and np.all(np.diff(off) >= 0)
        loads = np.array([counts[off[r]:off[r + 1]].sum() for r in range(world)])
        assert loads.max() - loads.min() <= 2 * counts.max()
