"""Multi-rank host logic on CPU: two gloo ranks (world size 2).

Restarts shard across GPUs with no collective on the data path; the only
exchange is the final merge of the best restart and the max-over-ranks
timing of the benchmark. Both are exercised here with CPU tensors.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2606_06641_gb300 import solver
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank 0 found 3 violations at restart 5, rank 1 found a solution at restart 9
        unsat, restart = (3, 5) if rank == 0 else (0, 9)
        asg = np.full(7, rank + 1, dtype=np.int8) * (1 if rank == 0 else -1)
        win = solver.merge_across_ranks(unsat, restart, asg)
        # ties break to the lowest rank
        tie = solver.merge_across_ranks(2, 4 - rank, np.full(3, rank, dtype=np.int8))
        t = solver.max_over_ranks(1.5 if rank == 0 else 2.25)
        out[rank] = (win[0], win[1], win[2], list(win[3]), tie[1], tie[2], list(tie[3]), t)
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_and_timing():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        unsat, wr, wb, asg, tie_rank, tie_restart, tie_asg, t = out[r]
        assert (unsat, wr, wb) == (0, 1, 9)
        assert asg == [-2] * 7
        assert (tie_rank, tie_restart) == (0, 4) and tie_asg == [0, 0, 0]
        assert t == 2.25
