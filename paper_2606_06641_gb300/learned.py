"""Learned initialiser: label harvesting, training and the paired evaluation.

The network, its gradient and Adam run in libafsat (afs_mpnn_*); this module
only sequences the calls:

* ``harvest``: solve instances with the plain batched descent (uniform
  starts) and turn the distinct satisfying assignments found per instance
  (up to ``max_solutions``) into soft labels y_v = fraction of them with v True.
* ``train``: mini-batch Adam over handles that each hold a group of labelled
  instances (the message passing runs over the disjoint union).
* ``evaluate``: the same held-out instances and the same step budget, solved
  from learned starts (the uniform starts nudged toward mu with a strength
  ramped over the restarts, or mu plus ramped noise with a share of restarts
  kept uniform) and from uniform starts.
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import binding as bd
from .synth import Instance


@dataclass
class Labels:
    y: np.ndarray        # soft labels per variable of the labelled instances (concatenated)
    insts: List[Instance]
    n_solutions: np.ndarray


def harvest(insts: Sequence[Instance], B: int, eta: float, steps: int, seed: int = 0,
            max_solutions: int = 8) -> Labels:
    """Soft labels from the distinct solutions the descent finds per instance."""
    import torch
    h = bd.load_batch(insts, bd.default_params(eta=eta, verify_every=1))
    bd.init_restarts(h, B, seed=seed)
    bd.step(h, steps)
    un, _ = bd.get_verify(h)
    x = bd.get_x(h).cpu().numpy()
    un = un.cpu().numpy()
    h.free()
    ys, kept, nsol = [], [], []
    v0 = 0
    for i, inst in enumerate(insts):
        cols = np.nonzero(un[i] == 0)[0]
        if cols.size:
            signs = (x[v0:v0 + inst.n, cols] < 0).T          # True where the variable is True
            uniq = np.unique(signs, axis=0)[:max_solutions]
            ys.append(uniq.mean(axis=0).astype(np.float32))
            kept.append(inst)
            nsol.append(uniq.shape[0])
        v0 += inst.n
    y = np.concatenate(ys) if ys else np.zeros(0, np.float32)
    return Labels(y, kept, np.asarray(nsol))


def make_batches(labels: Labels, group: int) -> List[Tuple[bd.Handle, "object"]]:
    """Handles of `group` labelled instances each, with their label tensors."""
    import torch
    out = []
    v0 = 0
    offs = np.cumsum([0] + [i.n for i in labels.insts])
    for g0 in range(0, len(labels.insts), group):
        gi = labels.insts[g0:g0 + group]
        h = bd.load_batch(gi, bd.default_params(autotune=0))
        y = torch.from_numpy(labels.y[offs[g0]:offs[g0 + len(gi)]]).cuda()
        out.append((h, y))
    return out


def train(net: bd.Mpnn, batches, epochs: int, lr: float, seed: int = 0, log_every: int = 0) -> List[float]:
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(batches))
        tot = 0.0
        for bi in order:
            h, y = batches[bi]
            loss, _ = net.loss_grad(h, y)
            net.adam_step(lr)
            tot += loss
        hist.append(tot / max(len(batches), 1))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {hist[-1]:.4f}", flush=True)
    return hist


# Starting points from the network: ("nudge", alpha_min, alpha_max) moves the
# uniform starts toward mu (x = clamp(u + alpha_b mu), alpha ramped over the
# restarts, the uniform draws the same as the plain form's); ("sample",
# uniform_frac, sigma_min, sigma_max) draws x = clamp(mu + sigma_b eps) for
# a share of the restarts and keeps the rest uniform.
DEFAULT_START = ("nudge", 0.0, 0.5)


def evaluate(net: Optional[bd.Mpnn], insts: Sequence[Instance], B: int, eta: float, max_steps: int,
             seed: int = 0, steps_per_poll: int = 10, start=DEFAULT_START):
    """Batched solve of `insts` from learned starts (net given) or uniform starts
    (net None). Returns (solved[bool], steps[int], seconds per instance, total)."""
    import torch
    n = len(insts)
    t0 = time.perf_counter()
    h = bd.load_batch(insts, bd.default_params(eta=eta, verify_every=1, autotune=0))
    bd.init_restarts(h, B, seed=seed)
    if net is not None:
        if start[0] == "nudge":
            net.nudge_restarts(h, alpha_min=start[1], alpha_max=start[2])
        else:
            net.init_restarts(h, B, seed=seed + 1, uniform_frac=start[1], sigma_min=start[2], sigma_max=start[3])
    solved = np.zeros(n, bool)
    steps = np.full(n, max_steps, np.int64)
    secs = np.zeros(n)
    sol_host = torch.empty(n, dtype=torch.int32).pin_memory()
    done = 0
    while done < max_steps:
        s = min(steps_per_poll, max_steps - done)
        bd.step(h, s)
        done += s
        _, sol = bd.get_verify(h)
        sol_host.copy_(sol)
        flags = sol_host.numpy() != 2 ** 31 - 1
        new = flags & ~solved
        steps[new] = done
        secs[new] = time.perf_counter() - t0
        solved |= flags
        if solved.all():
            break
    total = time.perf_counter() - t0
    secs[~solved] = total
    _, _, _, ok = bd.round_and_verify(h)
    if np.any(solved & (ok == 0)):
        raise RuntimeError("an instance flagged solved failed the final exact check")
    h.free()
    return solved, steps, secs, total
