"""Seeded synthetic instances and starting points for Fourier-expansion CLS.

This module is the only code shared by the CUDA path, the tests and the CPU
oracle. It draws instances and starting points; it holds none of the method's
arithmetic (no truth tables, coefficients, expansions or gradients).

Instance format (mirrors the hybrid DIMACS records of the paper's Appendix A):
  * ``ctype[c]``  constraint type code (``OR, XOR, NAE, AMO, EO, EK, CARD``)
  * ``op[c]``     CARD comparison, ``GE`` (t >= r) or ``LT`` (t < r)
  * ``param[c]``  threshold r for EK and CARD (ignored otherwise)
  * ``parity[c]`` XOR parity: 1 = odd number of true literals, 0 = even
  * ``lit_off``   CSR offsets, constraint c owns ``lits[lit_off[c]:lit_off[c+1]]``
  * ``lits``      DIMACS literals: +v is variable v (1-based), -v its negation

Workload recipes: uniform random 3-SAT at ratio 4.26 (n=50), a hybrid mixed-type instance
(n=2000), a long-constraint precision stress (n=10000, k in [64,512]), an
uneven batch of 256 instances, and the n=50 random 3-SAT distribution for the learned
initialiser. The paper's own benchmark files are not available; these
distributions stand in for their shapes.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

OR, XOR, NAE, AMO, EO, EK, CARD = range(7)
GE, LT = 0, 1
TYPE_NAMES = ("or", "xor", "nae", "amo", "eo", "ek", "card")


@dataclass
class Instance:
    n: int
    ctype: np.ndarray
    op: np.ndarray
    param: np.ndarray
    parity: np.ndarray
    lit_off: np.ndarray
    lits: np.ndarray

    @property
    def m(self) -> int:
        return int(self.ctype.shape[0])

    @property
    def n_lits(self) -> int:
        return int(self.lits.shape[0])

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.lit_off).astype(np.int32)

    def constraint(self, c: int) -> np.ndarray:
        return self.lits[self.lit_off[c]:self.lit_off[c + 1]]


class _Builder:
    """Accumulates constraint records and emits an :class:`Instance`."""

    def __init__(self, n: int):
        self.n = n
        self.ctype: List[int] = []
        self.op: List[int] = []
        self.param: List[int] = []
        self.parity: List[int] = []
        self.lens: List[int] = []
        self.lits: List[np.ndarray] = []

    def add(self, ctype: int, lits: Sequence[int], op: int = GE, param: int = 0,
            parity: int = 1) -> None:
        lits = np.asarray(lits, dtype=np.int32)
        self.ctype.append(ctype)
        self.op.append(op)
        self.param.append(param)
        self.parity.append(parity)
        self.lens.append(int(lits.shape[0]))
        self.lits.append(lits)

    def build(self) -> Instance:
        off = np.zeros(len(self.lens) + 1, dtype=np.int64)
        off[1:] = np.cumsum(np.asarray(self.lens, dtype=np.int64))
        off = off.astype(np.int32)
        lits = (np.concatenate(self.lits).astype(np.int32) if self.lits
                else np.zeros(0, dtype=np.int32))
        return Instance(
            n=self.n,
            ctype=np.asarray(self.ctype, dtype=np.int8),
            op=np.asarray(self.op, dtype=np.int8),
            param=np.asarray(self.param, dtype=np.int32),
            parity=np.asarray(self.parity, dtype=np.int8),
            lit_off=off,
            lits=lits,
        )


def rng_for(family: int, index: int, salt: int = 0) -> np.random.Generator:
    """Independent PCG64 stream per (workload family, instance index, salt)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([family, index, salt])))


def _draw_lits(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    """k distinct variables, uniform, each with a fair sign."""
    v = rng.choice(n, size=k, replace=False).astype(np.int32) + 1
    s = np.where(rng.random(k) < 0.5, -1, 1).astype(np.int32)
    return v * s


def _draw_lits_block(rng: np.random.Generator, n: int, count: int, k: int) -> np.ndarray:
    """``count`` rows of k distinct uniform variables with fair signs."""
    if k * 4 <= n:
        # rejection sampling of whole rows, vectorised
        out = np.empty((count, k), dtype=np.int32)
        todo = np.arange(count)
        while todo.size:
            cand = rng.integers(0, n, size=(todo.size, k), dtype=np.int64)
            srt = np.sort(cand, axis=1)
            ok = np.all(srt[:, 1:] != srt[:, :-1], axis=1) if k > 1 else np.ones(todo.size, bool)
            out[todo[ok]] = cand[ok]
            todo = todo[~ok]
        v = out + 1
    else:
        v = np.stack([rng.choice(n, size=k, replace=False) for _ in range(count)]) + 1
    s = np.where(rng.random((count, k)) < 0.5, -1, 1)
    return (v * s).astype(np.int32)


def random_ksat(n: int, m: int, k: int, rng: np.random.Generator) -> Instance:
    b = _Builder(n)
    rows = _draw_lits_block(rng, n, m, k)
    for r in rows:
        b.add(OR, r)
    return b.build()


def random_3sat_n50(index: int = 0) -> Instance:
    """Uniform random 3-SAT, n=50, m=213 (ratio 4.26)."""
    return random_ksat(50, 213, 3, rng_for(1, index))


def hybrid_n2000(index: int = 0) -> Instance:
    """Hybrid mixed-type instance, n=2000: 8000 3-clauses, 400 XOR(5) with a
    fair parity, 200 CARD(20) >= 10 and 100 NAE(4), in one shuffled list."""
    rng = rng_for(2, index)
    n = 2000
    b = _Builder(n)
    recs = []
    for r in _draw_lits_block(rng, n, 8000, 3):
        recs.append((OR, r, GE, 0, 1))
    par = rng.integers(0, 2, size=400)
    for r, p in zip(_draw_lits_block(rng, n, 400, 5), par):
        recs.append((XOR, r, GE, 0, int(p)))
    for r in _draw_lits_block(rng, n, 200, 20):
        recs.append((CARD, r, GE, 10, 1))
    for r in _draw_lits_block(rng, n, 100, 4):
        recs.append((NAE, r, GE, 0, 1))
    for i in rng.permutation(len(recs)):
        t, r, op, prm, p = recs[i]
        b.add(t, r, op, prm, p)
    return b.build()


def long_card_n10000(index: int = 0, n: int = 10000, n_clauses: int = 30000, n_long: int = 500,
            kmin: int = 64, kmax: int = 512) -> Instance:
    """Long-constraint stress: 3-clauses plus CARD(>= r) / EK(= r) constraints of
    length uniform in [kmin, kmax], r uniform in [ceil(k/4), floor(3k/4)],
    half CARD and half EK."""
    rng = rng_for(3, index)
    b = _Builder(n)
    for r in _draw_lits_block(rng, n, n_clauses, 3):
        b.add(OR, r)
    for j in range(n_long):
        k = int(rng.integers(kmin, kmax + 1))
        r = int(rng.integers(-(-k // 4), (3 * k) // 4 + 1))
        lits = _draw_lits(rng, n, k)
        if j % 2 == 0:
            b.add(CARD, lits, GE, r)
        else:
            b.add(EK, lits, GE, r)
    return b.build()


def batch_instance(index: int, nmin: int = 100, nmax: int = 20000) -> Instance:
    """One member of the uneven batch: n log-uniform in [nmin, nmax], m = ratio*n
    with ratio uniform in [4.0, 4.3]; 90% 3-clauses, 5% XOR of length 3..8,
    5% CARD (>= r) of length 10..100 with r uniform in [k/4, 3k/4]."""
    rng = rng_for(4, index)
    n = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
    m = int(round(rng.uniform(4.0, 4.3) * n))
    n_x = int(round(0.05 * m))
    n_c = int(round(0.05 * m))
    n_o = m - n_x - n_c
    b = _Builder(n)
    recs = [(OR, r, GE, 0, 1) for r in _draw_lits_block(rng, n, n_o, 3)]
    for _ in range(n_x):
        k = int(rng.integers(3, 9))
        recs.append((XOR, _draw_lits(rng, n, k), GE, 0, int(rng.integers(0, 2))))
    for _ in range(n_c):
        k = int(rng.integers(10, min(100, n) + 1))
        r = int(rng.integers(-(-k // 4), (3 * k) // 4 + 1))
        recs.append((CARD, _draw_lits(rng, n, k), GE, r, 1))
    for i in rng.permutation(len(recs)):
        t, r, op, prm, p = recs[i]
        b.add(t, r, op, prm, p)
    return b.build()


def instance_batch(count: int = 256, nmin: int = 100, nmax: int = 20000) -> List[Instance]:
    return [batch_instance(i, nmin, nmax) for i in range(count)]


def learned_split(index: int, split: str = "train") -> Instance:
    """Random 3-SAT n=50, m=213; training and held-out instances use disjoint streams."""
    salt = 0 if split == "train" else 1
    return random_ksat(50, 213, 3, rng_for(5, index, salt))


def mixed_small(index: int, n: int = 40, m: int = 60, kmax: int = 12) -> Instance:
    """Small instance mixing every constraint type and several lengths, used by
    parity tests that must cover all truth-table shapes."""
    rng = rng_for(100, index)
    b = _Builder(n)
    for _ in range(m):
        t = int(rng.integers(0, 7))
        k = int(rng.integers(1, min(kmax, n) + 1))
        lits = _draw_lits(rng, n, k)
        if t == EK:
            b.add(EK, lits, GE, int(rng.integers(0, k + 1)))
        elif t == CARD:
            b.add(CARD, lits, int(rng.integers(0, 2)), int(rng.integers(0, k + 2)))
        elif t == XOR:
            b.add(XOR, lits, GE, 0, int(rng.integers(0, 2)))
        else:
            b.add(t, lits)
    return b.build()


def single_type(ctype: int, k: int, count: int, n: int, index: int = 0, op: int = GE,
                param: int = 0, parity: int = 1) -> Instance:
    """``count`` constraints of one type and length over n variables."""
    rng = rng_for(101, index, ctype * 1000 + k)
    b = _Builder(n)
    for r in _draw_lits_block(rng, n, count, k):
        b.add(ctype, r, op, param, parity)
    return b.build()


def uniform_x0(n: int, B: int, seed: int) -> np.ndarray:
    """Starting points x[n][B] uniform on [-1, 1], float32, restart-major."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([7, seed])))
    return rng.uniform(-1.0, 1.0, size=(n, B)).astype(np.float32)


def near_vertex_x0(n: int, B: int, seed: int, spread: float = 0.05) -> np.ndarray:
    """Starting points near hypercube vertices (|x| in [1-spread, 1])."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([8, seed])))
    s = np.where(rng.random((n, B)) < 0.5, -1.0, 1.0)
    return (s * (1.0 - spread * rng.random((n, B)))).astype(np.float32)


def vertex_x0(n: int, B: int, seed: int) -> np.ndarray:
    """Exact hypercube vertices, with a few exact zeros to exercise tie rounding."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([9, seed])))
    x = np.where(rng.random((n, B)) < 0.5, -1.0, 1.0).astype(np.float32)
    return x


def concat_instances(insts: Sequence[Instance]) -> Instance:
    """Disjoint union: variables of instance i are shifted past those of 0..i-1."""
    b = _Builder(sum(i.n for i in insts))
    shift = 0
    for inst in insts:
        for c in range(inst.m):
            l = inst.constraint(c)
            l = np.where(l > 0, l + shift, l - shift)
            b.add(int(inst.ctype[c]), l, int(inst.op[c]), int(inst.param[c]), int(inst.parity[c]))
        shift += inst.n
    return b.build()
