"""CPU FP64 oracle for Fourier-expansion continuous local search (CLS).

TEST INFRASTRUCTURE ONLY. This module is imported by ``tests/``, by the
package's ``smoke()`` check and by the CPU-baseline leg of ``bench.py``; the
product path never imports, links or runs it. It shares no code with the CUDA
path (no kernels, headers, tables or coefficient generators). It takes
instances as plain arrays with the attributes ``n, ctype, op, param, parity,
lit_off, lits`` (the hybrid DIMACS records of the paper's Appendix A) and
starting points as numpy arrays ``x[n][B]``.

What it computes, and from which passage:
  * Truth tables f(t) of every symmetric constraint type: Table 1 and the
    type table of Appendix A (OR, XOR, NAE, AMO, EO, EK, CARD), with True
    mapped to -1 and False to +1 (Sec. 2.1, Eq. 1).
  * The Fourier expansion (Eq. 1) of a symmetric constraint at a point
    l in [-1,1]^k. Eq. 1 is the multilinear extension of f, which equals the
    expectation of f(T), where T counts independent literals that are true
    with probability p_i = (1 - l_i)/2. The distribution of T is built by the
    Poisson-binomial recurrence, O(k^2) per constraint.
  * Its exact gradient dFE/dl_i = (E f(T_{-i}) - E f(T_{-i} + 1)) / 2, from a
    backward message over the same recurrence, O(k^2) per constraint.
  * The objective sum_c FE_c and its gradient in x (Sec. 2.1.1), one projected
    gradient step with a fixed step size (Algorithm 1: step, then projection
    onto [-1,1]^n), and the unsatisfied-constraint count at the sign-rounded
    point (Algorithm 1's returned unsat count), in exact integers.
  * Brute-force references: Eq. 1 summed over all subsets with Walsh
    coefficients taken from their definition (k <= 12), exhaustive
    satisfiability for n <= 20, and a plain DPLL for labelling small
    instances.
  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for the counter-based
    starting points, so the device generator can be checked bit for bit.

Readings of the paper taken here (where it is silent or ambiguous):
  * A literal is True when l_i = -1. The sign-rounded point takes x_v < 0 as
    True and x_v >= 0 (including -0.0) as False.
  * CARD is normalised to ">= r" or "< r"; a plain positive threshold means
    ">= r" and a negative one "< |r|" (Appendix A).
  * XOR with parity 1 is satisfied by an odd count, parity 0 by an even count.
  * NAE is satisfied iff 0 < t < k.
  * Repeated variables inside one constraint are independent literals.
  * A constraint counts as unsatisfied at a vertex iff f(t) = +1 (the "FE > 0"
    test of Algorithm 1 evaluated exactly at the rounded point).
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Optional, Tuple

import numpy as np

# Constraint type codes of the instance records (Appendix A type identifiers).
T_OR, T_XOR, T_NAE, T_AMO, T_EO, T_EK, T_CARD = range(7)
OP_GE, OP_LT = 0, 1


# --------------------------------------------------------------------------
# Truth tables (Table 1; Appendix A type table)
# --------------------------------------------------------------------------
def satisfied(ctype: int, k: int, t: int, op: int = OP_GE, param: int = 0,
              parity: int = 1) -> bool:
    """Whether a symmetric constraint of length k holds when t literals are true."""
    if ctype == T_OR:
        return t >= 1
    if ctype == T_XOR:
        return (t % 2) == (1 if parity else 0)
    if ctype == T_NAE:
        return 0 < t < k
    if ctype == T_AMO:
        return t <= 1
    if ctype == T_EO:
        return t == 1
    if ctype == T_EK:
        return t == param
    if ctype == T_CARD:
        return t >= param if op == OP_GE else t < param
    raise ValueError(f"unknown constraint type {ctype}")


def truth_table(ctype: int, k: int, op: int = OP_GE, param: int = 0,
                parity: int = 1) -> np.ndarray:
    """f(t) for t = 0..k: -1 where the constraint holds, +1 where it fails."""
    return np.array([-1.0 if satisfied(ctype, k, t, op, param, parity) else 1.0
                     for t in range(k + 1)], dtype=np.float64)


def instance_tables(inst) -> List[np.ndarray]:
    k = np.diff(inst.lit_off)
    return [truth_table(int(inst.ctype[c]), int(k[c]), int(inst.op[c]), int(inst.param[c]),
                        int(inst.parity[c])) for c in range(len(k))]


def normalise_card(threshold: int, op: Optional[str]) -> Tuple[int, int]:
    """Appendix A: map a CARD threshold (and optional operator) to (op, r) with
    op in {GE, LT}: no operator -> positive r means >= r, negative means < |r|;
    '>' r -> >= r+1; '<=' r -> < r+1; '>=' and '<' are kept."""
    if op is None:
        return (OP_GE, threshold) if threshold > 0 else (OP_LT, -threshold)
    if op == ">=":
        return OP_GE, threshold
    if op == ">":
        return OP_GE, threshold + 1
    if op == "<":
        return OP_LT, threshold
    if op == "<=":
        return OP_LT, threshold + 1
    raise ValueError(op)


# --------------------------------------------------------------------------
# Fourier expansion as an expectation (Eq. 1), Poisson-binomial recurrence
# --------------------------------------------------------------------------
def count_distribution(ell: np.ndarray) -> np.ndarray:
    """P(T = t), t = 0..k, for T = number of true literals; ell[..., k] in
    [-1,1], each literal true with probability (1 - l)/2, independently."""
    k = ell.shape[-1]
    p = (1.0 - ell) / 2.0
    q = 1.0 - p
    dist = np.zeros(ell.shape[:-1] + (k + 1,), dtype=np.float64)
    dist[..., 0] = 1.0
    for i in range(k):
        new = dist * q[..., i:i + 1]
        new[..., 1:] += dist[..., :-1] * p[..., i:i + 1]
        dist = new
    return dist


def fe(f: np.ndarray, ell: np.ndarray) -> np.ndarray:
    """Fourier expansion of a symmetric constraint with truth table f[..., k+1]
    (broadcast against ell[..., k]): E[f(T)]."""
    dist = count_distribution(np.asarray(ell, dtype=np.float64))
    return np.sum(dist * f, axis=-1)


def fe_and_dfe(f: np.ndarray, ell: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """FE and dFE/dl_i for every literal.

    With pre_{i-1} the count distribution of literals 1..i-1 and
    h_i(a) = E[f(a + T_{>i}) - f(a + 1 + T_{>i})], the derivative is
    dFE/dl_i = 1/2 * sum_a pre_{i-1}(a) h_i(a). h is propagated backwards with
    h_{i-1}(a) = q_i h_i(a) + p_i h_i(a + 1), starting from h_k(a) = f(a) - f(a+1).
    """
    ell = np.asarray(ell, dtype=np.float64)
    k = ell.shape[-1]
    lead = ell.shape[:-1]
    f = np.broadcast_to(f, lead + (k + 1,))
    p = (1.0 - ell) / 2.0
    q = 1.0 - p
    pres = []
    dist = np.zeros(lead + (k + 1,), dtype=np.float64)
    dist[..., 0] = 1.0
    for i in range(k):
        pres.append(dist)
        new = dist * q[..., i:i + 1]
        new[..., 1:] += dist[..., :-1] * p[..., i:i + 1]
        dist = new
    value = np.sum(dist * f, axis=-1)
    grad = np.empty(lead + (k,), dtype=np.float64)
    h = f[..., :-1] - f[..., 1:]          # h_k(a), a = 0..k-1
    for i in range(k, 0, -1):              # literal i (1-based)
        pre = pres[i - 1][..., :i]         # pre_{i-1}(a), a = 0..i-1
        grad[..., i - 1] = 0.5 * np.sum(pre * h[..., :i], axis=-1)
        if i > 1:
            h = q[..., i - 1:i] * h[..., :i - 1] + p[..., i - 1:i] * h[..., 1:i]
    return value, grad


# --------------------------------------------------------------------------
# Whole-instance objective, gradient, PGD step, exact verification
# --------------------------------------------------------------------------
def _groups(inst) -> Dict[int, np.ndarray]:
    k = np.diff(inst.lit_off)
    out: Dict[int, np.ndarray] = {}
    for kk in np.unique(k):
        out[int(kk)] = np.nonzero(k == kk)[0]
    return out


def literal_values(inst, x: np.ndarray, cons: np.ndarray, k: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """l[g, b, i] = s_i * x[v_i, b] for the constraints ``cons`` (all of length k)."""
    idx = inst.lit_off[cons][:, None] + np.arange(k)[None, :]
    lits = inst.lits[idx]
    var = np.abs(lits) - 1
    sgn = np.where(lits < 0, -1.0, 1.0)
    xv = x.astype(np.float64)[var]                     # [G, k, B]
    ell = np.transpose(xv * sgn[:, :, None], (0, 2, 1))  # [G, B, k]
    return ell, var, sgn


def evaluate(inst, x: np.ndarray, want_grad: bool = True):
    """FE of every constraint, fe[m][B], and if asked the per-occurrence
    derivative go[L][B] = s_i * dFE_c/dl_i and the gradient of the objective
    g[n][B] = sum over occurrences of v of s_i * dFE_c/dl_i."""
    x = np.asarray(x)
    n, B = x.shape
    m = len(inst.lit_off) - 1
    fe_out = np.zeros((m, B), dtype=np.float64)
    go = np.zeros((inst.lits.shape[0], B), dtype=np.float64) if want_grad else None
    g = np.zeros((n, B), dtype=np.float64) if want_grad else None
    tables = instance_tables(inst)
    for k, cons in _groups(inst).items():
        f = np.stack([tables[c] for c in cons])[:, None, :]   # [G, 1, k+1]
        if k == 0:
            fe_out[cons] = f[:, :, 0]
            continue
        ell, var, sgn = literal_values(inst, x, cons, k)
        if want_grad:
            val, d = fe_and_dfe(f, ell)                          # d [G, B, k]
            fe_out[cons] = val
            contrib = np.transpose(d, (0, 2, 1)) * sgn[:, :, None]   # [G, k, B]
            occ = inst.lit_off[cons][:, None] + np.arange(k)[None, :]
            go[occ.ravel()] = contrib.reshape(-1, B)
            np.add.at(g, var.ravel(), contrib.reshape(-1, B))
        else:
            fe_out[cons] = fe(f, ell)
    return fe_out, go, g


def objective(inst, x: np.ndarray) -> np.ndarray:
    fe_out, _, _ = evaluate(inst, x, want_grad=False)
    return fe_out.sum(axis=0)


def pgd_step(inst, x: np.ndarray, eta: float) -> np.ndarray:
    """One step of Algorithm 1 with a fixed step: x <- proj_[-1,1](x - eta * grad)."""
    _, _, g = evaluate(inst, x, want_grad=True)
    return np.clip(x.astype(np.float64) - eta * g, -1.0, 1.0)


def armijo_step(inst, x: np.ndarray, s: float, beta: float, c: float, trials: int):
    """One projected-gradient step with Armijo backtracking per restart (the
    line search Algorithm 1 leaves unspecified, read as): g = grad F(x); trial
    i = 0, 1, .. tries eta_i = s * beta**i and x_i = proj_[-1,1](x - eta_i g),
    and the first trial with F(x_i) <= F(x) + c * sum_v g_v (x_i,v - x_v) is
    taken; a restart that accepts none takes the last trial. Returns the new
    state and the chosen trial per restart (-1 where none was accepted)."""
    x = np.asarray(x, dtype=np.float64)
    fe0, _, g = evaluate(inst, x, want_grad=True)
    f0 = fe0.sum(axis=0)
    out = np.empty_like(x)
    chosen = np.full(x.shape[1], -1, dtype=np.int64)
    done = np.zeros(x.shape[1], dtype=bool)
    for i in range(trials):
        xi = np.clip(x - (s * beta ** i) * g, -1.0, 1.0)
        fi = objective(inst, xi)
        dec = (g * (xi - x)).sum(axis=0)
        ok = (fi <= f0 + c * dec) & ~done
        out[:, ok] = xi[:, ok]
        chosen[ok] = i
        done |= ok
        if i == trials - 1:
            out[:, ~done] = xi[:, ~done]
    return out, chosen


def round_signs(x: np.ndarray) -> np.ndarray:
    """Sign rounding: True (-1) where x < 0, False (+1) otherwise."""
    return np.where(np.asarray(x) < 0, -1, 1).astype(np.int8)


def true_counts(inst, sigma: np.ndarray) -> np.ndarray:
    """t[c][b] = number of true literals of constraint c under sigma[n][B] (+-1)."""
    lits = inst.lits.astype(np.int64)
    var = np.abs(lits) - 1
    sgn = np.where(lits < 0, -1, 1)
    lit_true = (sgn[:, None] * sigma[var].astype(np.int64)) == -1        # [L, B]
    cs = np.concatenate([np.zeros((1, sigma.shape[1]), np.int64),
                         np.cumsum(lit_true, axis=0, dtype=np.int64)])
    return cs[inst.lit_off[1:]] - cs[inst.lit_off[:-1]]


def unsat_mask(inst, x: np.ndarray) -> np.ndarray:
    """unsat[c][b] = 1 where constraint c fails at the sign-rounded point."""
    sigma = round_signs(x)
    t = true_counts(inst, sigma)
    k = np.diff(inst.lit_off)
    out = np.zeros(t.shape, dtype=np.int32)
    for c in range(len(k)):
        tab = truth_table(int(inst.ctype[c]), int(k[c]), int(inst.op[c]), int(inst.param[c]),
                          int(inst.parity[c]))
        out[c] = (tab[t[c]] > 0).astype(np.int32)
    return out


def unsat_count(inst, x: np.ndarray) -> np.ndarray:
    """Per-restart number of unsatisfied constraints at the rounded point."""
    return unsat_mask(inst, x).sum(axis=0).astype(np.int32)


def pgd(inst, x0: np.ndarray, eta: float, steps: int):
    """Algorithm 1 with a fixed step size and no early stop: returns the
    trajectory end point and the unsat count after every step."""
    x = x0.astype(np.float64)
    hist = []
    for _ in range(steps):
        x = pgd_step(inst, x, eta)
        hist.append(unsat_count(inst, x))
    return x, np.stack(hist) if hist else np.zeros((0, x0.shape[1]), np.int32)


# --------------------------------------------------------------------------
# Brute-force references
# --------------------------------------------------------------------------
def walsh_coefficients(f: np.ndarray) -> np.ndarray:
    """f_hat(S) for every subset S of {0..k-1} (bitmask order), from the
    definition f_hat(S) = 2^-k sum_{L in {+-1}^k} F(L) prod_{i in S} L_i with
    F(L) = f(#{i : L_i = -1})."""
    k = len(f) - 1
    pts = np.array(list(itertools.product([1.0, -1.0], repeat=k)), dtype=np.float64).reshape(-1, k)
    F = f[(pts < 0).sum(axis=1)]
    masks = np.arange(1 << k)
    bits = ((masks[:, None] >> np.arange(k)[None, :]) & 1).astype(bool)      # [2^k, k]
    chi = np.ones((1 << k, pts.shape[0]), dtype=np.float64)
    for i in range(k):
        chi[bits[:, i]] *= pts[:, i][None, :]
    return chi @ F / float(1 << k)


def fe_walsh(f: np.ndarray, ell: np.ndarray) -> np.ndarray:
    """Eq. 1 summed directly: sum_S f_hat(S) prod_{i in S} l_i, for ell[B, k]."""
    k = len(f) - 1
    fhat = walsh_coefficients(f)
    ell = np.atleast_2d(np.asarray(ell, dtype=np.float64))
    masks = np.arange(1 << k)
    bits = ((masks[:, None] >> np.arange(k)[None, :]) & 1).astype(bool)
    mono = np.ones((ell.shape[0], 1 << k), dtype=np.float64)
    for i in range(k):
        mono[:, bits[:, i]] *= ell[:, i][:, None]
    return mono @ fhat


def exhaustive_sat(inst) -> Tuple[bool, Optional[np.ndarray]]:
    """Enumerate all 2^n assignments (n <= 20). Returns (sat, one model as +-1)."""
    n = inst.n
    if n > 20:
        raise ValueError("exhaustive check limited to n <= 20")
    k = np.diff(inst.lit_off)
    tabs = [truth_table(int(inst.ctype[c]), int(k[c]), int(inst.op[c]), int(inst.param[c]),
                        int(inst.parity[c])) for c in range(len(k))]
    chunk = 1 << min(n, 16)
    for start in range(0, 1 << n, chunk):
        a = np.arange(start, min(start + chunk, 1 << n), dtype=np.int64)
        sigma = np.where(((a[None, :] >> np.arange(n)[:, None]) & 1) == 1, -1, 1).astype(np.int8)
        t = true_counts(inst, sigma)
        ok = np.ones(a.shape[0], dtype=bool)
        for c in range(len(k)):
            ok &= tabs[c][t[c]] < 0
        if ok.any():
            j = int(np.nonzero(ok)[0][0])
            return True, sigma[:, j].copy()
    return False, None


def dpll(inst, max_nodes: int = 2_000_000) -> Optional[bool]:
    """Plain DPLL for clause-only (OR) instances with unit propagation.
    Returns True (SAT), False (UNSAT) or None if the node budget ran out."""
    if np.any(inst.ctype != T_OR):
        raise ValueError("dpll handles OR constraints only")
    clauses = [list(map(int, inst.lits[inst.lit_off[c]:inst.lit_off[c + 1]]))
               for c in range(len(inst.lit_off) - 1)]
    nodes = [0]

    def simplify(cls, lit):
        out = []
        for cl in cls:
            if lit in cl:
                continue
            if -lit in cl:
                cl = [l for l in cl if l != -lit]
                if not cl:
                    return None
            out.append(cl)
        return out

    def solve(cls):
        nodes[0] += 1
        if nodes[0] > max_nodes:
            raise TimeoutError
        while True:
            unit = next((cl[0] for cl in cls if len(cl) == 1), None)
            if unit is None:
                break
            cls = simplify(cls, unit)
            if cls is None:
                return False
        if not cls:
            return True
        counts: Dict[int, int] = {}
        for cl in cls:
            for l in cl:
                counts[l] = counts.get(l, 0) + 1
        lit = max(counts, key=lambda l: (counts[l] + counts.get(-l, 0), counts[l], -abs(l)))
        for choice in (lit, -lit):
            sub = simplify(cls, choice)
            if sub is not None and solve(sub):
                return True
        return False

    try:
        return solve(clauses)
    except TimeoutError:
        return None


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11) and the counter-based starting points
# --------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32 with 10 rounds. ctr[..., 4] and key[..., 2] are uint32
    arrays; returns uint32[..., 4]. Each round multiplies words 0 and 2 by the
    round constants, swaps in the high halves xor-ed with words 1, 3 and the
    key, and the key advances by the Weyl constants between rounds."""
    c = np.asarray(ctr, dtype=np.uint64) & _MASK32
    k = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for r in range(10):
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK32, lo1, (hi0 ^ c3 ^ k1) & _MASK32, lo0
        if r < 9:
            k0 = (k0 + _PHILOX_W0) & _MASK32
            k1 = (k1 + _PHILOX_W1) & _MASK32
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def philox_uniform_x0(seed: int, n: int, B: int, stream: int = 0) -> np.ndarray:
    """Counter-based starting points x[v][b] in [-1, 1): counter
    (b // 4, v, stream, 0), key (seed low word, seed high word); word b % 4 of
    the output is mapped to (2 * (w >> 8) * 2^-24) - 1, which is exact in FP32."""
    v = np.arange(n, dtype=np.uint64)[:, None]
    b = np.arange(B, dtype=np.uint64)[None, :]
    ctr = np.zeros((n, B, 4), dtype=np.uint64)
    ctr[..., 0] = b // np.uint64(4)
    ctr[..., 1] = v
    ctr[..., 2] = np.uint64(stream)
    key = np.zeros((n, B, 2), dtype=np.uint64)
    key[..., 0] = np.uint64(seed & 0xFFFFFFFF)
    key[..., 1] = np.uint64((seed >> 32) & 0xFFFFFFFF)
    out = philox4x32_10(ctr, key)
    word = np.take_along_axis(out, (np.arange(B) % 4)[None, :, None].repeat(n, 0).astype(np.int64),
                              axis=-1)[..., 0]
    u = (word >> np.uint32(8)).astype(np.float64) * (2.0 ** -24)
    return (2.0 * u - 1.0).astype(np.float32)
