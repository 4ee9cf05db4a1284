"""Solve loops over the C ABI: plain CLS and the batched serving form.

Algorithm 1 (projected gradient descent with a fixed step) runs on the device;
this module only sequences the ABI calls and reads the solved flags.

* ``solve_plain``: one instance at a time, B restarts, one un-captured launch
  sequence per step, the solved flag read back after every step. This is the
  plain continuous local search the batched form is compared with.
* ``solve_batched``: many instances in one handle (one launch per length
  bucket covers all of them), the descent loop replayed as a captured CUDA
  graph of S steps, solved flags read back between replays.

Both report, per instance, whether it was solved, the steps taken and the
wall time from the start of the run until its solution was known; every
reported solution has been re-checked exactly (afs_round_and_verify).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

from . import binding as bd
from .synth import Instance


@dataclass
class SolveResult:
    solved: np.ndarray          # bool per instance
    steps: np.ndarray           # steps until solved (or the budget)
    seconds: np.ndarray         # wall time from run start until solved (or the end)
    total_seconds: float
    assignments: List[Optional[np.ndarray]] = field(default_factory=list)


def _verify_solution(inst: Instance, asg: np.ndarray) -> bool:
    """Host re-check of a +-1 assignment against the instance records."""
    lits = inst.lits
    var = np.abs(lits) - 1
    val = asg[var].astype(np.int64)
    lit_true = np.where(lits > 0, val < 0, val > 0)
    cs = np.concatenate([[0], np.cumsum(lit_true)])
    t = cs[inst.lit_off[1:]] - cs[inst.lit_off[:-1]]
    k = np.diff(inst.lit_off)
    ok = np.ones(inst.m, bool)
    for c in range(inst.m):
        ct, kk, tt = int(inst.ctype[c]), int(k[c]), int(t[c])
        if ct == 0:
            ok[c] = tt >= 1
        elif ct == 1:
            ok[c] = (tt % 2) == (1 if inst.parity[c] else 0)
        elif ct == 2:
            ok[c] = 0 < tt < kk
        elif ct == 3:
            ok[c] = tt <= 1
        elif ct == 4:
            ok[c] = tt == 1
        elif ct == 5:
            ok[c] = tt == inst.param[c]
        else:
            ok[c] = tt >= inst.param[c] if inst.op[c] == 0 else tt < inst.param[c]
    return bool(ok.all())


def solve_plain(insts: Sequence[Instance], B: int, eta: float, max_steps: int, seed: int = 0,
                x0s: Optional[Sequence] = None) -> SolveResult:
    """Instances one after another; each gets B restarts and up to max_steps steps."""
    import torch
    n = len(insts)
    solved = np.zeros(n, bool)
    steps = np.full(n, max_steps, np.int64)
    secs = np.zeros(n)
    asgs: List[Optional[np.ndarray]] = [None] * n
    sol_host = torch.empty(1, dtype=torch.int32).pin_memory()
    t_run = time.perf_counter()
    for i, inst in enumerate(insts):
        p = bd.default_params(eta=eta, use_graph=0, autotune=0, verify_every=1)
        h = bd.load_instance(inst, p)
        bd.init_restarts(h, B, seed=seed + i, x0=None if x0s is None else x0s[i])
        _, sol = bd.get_verify(h)
        for t in range(1, max_steps + 1):
            bd.step(h, 1)
            _, sol = bd.get_verify(h)
            sol_host.copy_(sol)
            if int(sol_host[0]) != 2 ** 31 - 1:
                solved[i] = True
                steps[i] = t
                break
        if solved[i]:
            _, best, asg, ok = bd.round_and_verify(h)
            if not ok[0] or not _verify_solution(inst, asg):
                raise RuntimeError(f"instance {i}: reported solution failed the host re-check")
            asgs[i] = asg
        torch.cuda.synchronize()
        secs[i] = time.perf_counter() - t_run
        h.free()
    return SolveResult(solved, steps, secs, time.perf_counter() - t_run, asgs)


def solve_batched(insts: Sequence[Instance], B: int, eta: float, max_steps: int, seed: int = 0,
                  steps_per_poll: int = 10, x0=None, line_search=None) -> SolveResult:
    """All instances in one handle; S-step graph replays, solved flags polled
    between them. line_search = (s, beta, c, trials) replaces the fixed step by
    Armijo backtracking (afs_step_ls, one iteration per poll)."""
    import torch
    n = len(insts)
    solved = np.zeros(n, bool)
    steps = np.full(n, max_steps, np.int64)
    secs = np.zeros(n)
    t_run = time.perf_counter()
    p = bd.default_params(eta=eta, use_graph=1, autotune=1, verify_every=1)
    h = bd.load_batch(insts, p)
    bd.init_restarts(h, B, seed=seed, x0=x0)
    sol_host = torch.empty(n, dtype=torch.int32).pin_memory()
    done_steps = 0
    S = max(1, steps_per_poll)
    while done_steps < max_steps:
        s = min(S, max_steps - done_steps)
        if line_search is None:
            bd.step(h, s)
        else:
            s = 1
            bd.step_ls(h, 1, *line_search)
        done_steps += s
        _, sol = bd.get_verify(h)
        sol_host.copy_(sol)
        now = time.perf_counter() - t_run
        flags = sol_host.numpy() != 2 ** 31 - 1
        new = flags & ~solved
        steps[new] = done_steps
        secs[new] = now
        solved |= flags
        if solved.all():
            break
    un, best, asg, ok = bd.round_and_verify(h)
    asgs: List[Optional[np.ndarray]] = [None] * n
    v0 = 0
    for i, inst in enumerate(insts):
        if solved[i]:
            a = asg[v0:v0 + inst.n]
            if not ok[i] or not _verify_solution(inst, a):
                raise RuntimeError(f"instance {i}: reported solution failed the host re-check")
            asgs[i] = a
        v0 += inst.n
    total = time.perf_counter() - t_run
    secs[~solved] = total
    h.free()
    return SolveResult(solved, steps, secs, total, asgs)


def merge_across_ranks(best_unsat: int, best_restart: int, assignment: np.ndarray):
    """Replicas on several GPUs solve the same instance from different
    restarts; the result is the restart with the fewest violated constraints
    (ties: lowest rank, then lowest restart). One all-reduce of a packed key
    picks the winner and one broadcast ships its +-1 assignment; this is the
    only exchange the data-parallel path needs. Works with any
    torch.distributed backend (CPU tensors with gloo)."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(), dist.get_world_size()
    key = torch.tensor([best_unsat * world * (1 << 31) + rank * (1 << 31) + best_restart], dtype=torch.int64)
    dist.all_reduce(key, op=dist.ReduceOp.MIN)
    k = int(key.item())
    win_unsat, rem = divmod(k, world * (1 << 31))
    win_rank, win_restart = divmod(rem, 1 << 31)
    buf = torch.from_numpy(np.ascontiguousarray(assignment, dtype=np.int8)).clone()
    dist.broadcast(buf, src=win_rank)
    return win_unsat, win_rank, win_restart, buf.numpy()


def max_over_ranks(value: float) -> float:
    """The slowest rank's time (bench timing rule)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def par2(res: SolveResult, timeout_s: float) -> float:
    """PAR-2: mean time with unsolved instances charged twice the timeout."""
    t = np.where(res.solved & (res.seconds <= timeout_s), res.seconds, 2.0 * timeout_s)
    return float(t.mean())


def median_tts(res: SolveResult, timeout_s: float) -> float:
    """Median time-to-solve with unsolved instances counted at twice the timeout."""
    t = np.where(res.solved & (res.seconds <= timeout_s), res.seconds, 2.0 * timeout_s)
    return float(np.median(t))
