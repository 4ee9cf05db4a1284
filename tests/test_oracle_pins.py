"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something other than itself: Eq. 1 summed
over all subsets with Walsh coefficients from their definition, closed forms
of the constraint types, the vertex property of the expansion, exact finite
differences (the expansion is multilinear), exhaustive satisfiability, the
paper's worked input-format examples (Appendix A), and the published
Philox4x32-10 known-answer vectors.
"""
import math
import os

import numpy as np
import pytest

from oracle import fe_oracle as O
from paper_2606_06641_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TYPES = [O.T_OR, O.T_XOR, O.T_NAE, O.T_AMO, O.T_EO, O.T_EK, O.T_CARD]


def _tables_for(k):
    """A spread of truth tables of length k covering every type and operator."""
    out = [O.truth_table(O.T_OR, k), O.truth_table(O.T_XOR, k, parity=1),
           O.truth_table(O.T_XOR, k, parity=0), O.truth_table(O.T_NAE, k),
           O.truth_table(O.T_AMO, k), O.truth_table(O.T_EO, k)]
    for r in sorted({0, 1, k // 2, k}):
        out.append(O.truth_table(O.T_EK, k, param=r))
        out.append(O.truth_table(O.T_CARD, k, O.OP_GE, r))
        out.append(O.truth_table(O.T_CARD, k, O.OP_LT, r))
    return out


# --- Eq. 1 by brute force -------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 8, 10])
def test_fe_equals_walsh_expansion(k):
    rng = np.random.default_rng(k)
    ell = np.concatenate([rng.uniform(-1, 1, (6, k)),
                          np.clip(np.sign(rng.uniform(-1, 1, (3, k))) * (1 - 0.01 * rng.random((3, k))), -1, 1),
                          np.zeros((1, k))])
    for f in _tables_for(k):
        np.testing.assert_allclose(O.fe(f, ell), O.fe_walsh(f, ell), atol=1e-13, rtol=0)


@pytest.mark.parametrize("k", [1, 3, 6, 9])
def test_gradient_equals_walsh_derivative(k):
    """d/dl_i of sum_S f_hat(S) prod_{j in S} l_j = sum_{S containing i} f_hat(S) prod_{S \\ i} l_j."""
    rng = np.random.default_rng(100 + k)
    ell = rng.uniform(-1, 1, (5, k))
    masks = np.arange(1 << k)
    bits = ((masks[:, None] >> np.arange(k)[None, :]) & 1).astype(bool)
    for f in _tables_for(k):
        fhat = O.walsh_coefficients(f)
        _, d = O.fe_and_dfe(f, ell)
        for i in range(k):
            sel = bits[:, i]
            mono = np.ones((ell.shape[0], int(sel.sum())))
            for j in range(k):
                if j != i:
                    mono *= np.where(bits[sel, j][None, :], ell[:, j][:, None], 1.0)
            ref = mono @ fhat[sel]
            np.testing.assert_allclose(d[:, i], ref, atol=1e-13, rtol=0)


def test_walsh_coefficients_of_parity_and_or():
    """Textbook spectra: odd XOR of k bits is the single character prod x_i
    (f_hat = 1 on the full set); OR = -1 + 2 * prod (1 + x_i)/2 puts weight
    2^{1-k} on every non-empty set and 2^{1-k} - 1 on the empty set."""
    k = 5
    fx = O.walsh_coefficients(O.truth_table(O.T_XOR, k, parity=1))
    want = np.zeros(1 << k)
    want[(1 << k) - 1] = 1.0
    np.testing.assert_allclose(fx, want, atol=1e-15)
    fo = O.walsh_coefficients(O.truth_table(O.T_OR, k))
    want = np.full(1 << k, 2.0 ** (1 - k))
    want[0] = 2.0 ** (1 - k) - 1
    np.testing.assert_allclose(fo, want, atol=1e-15)


# --- closed forms -----------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 7, 20, 64, 200])
def test_closed_forms(k):
    rng = np.random.default_rng(7 * k)
    ell = rng.uniform(-1, 1, (4, k))
    p = (1 - ell) / 2
    q = 1 - p
    np.testing.assert_allclose(O.fe(O.truth_table(O.T_OR, k), ell), -1 + 2 * q.prod(-1), atol=1e-12)
    np.testing.assert_allclose(O.fe(O.truth_table(O.T_XOR, k, parity=1), ell), ell.prod(-1), atol=1e-12)
    np.testing.assert_allclose(O.fe(O.truth_table(O.T_XOR, k, parity=0), ell), -ell.prod(-1), atol=1e-12)
    np.testing.assert_allclose(O.fe(O.truth_table(O.T_NAE, k), ell),
                               -1 + 2 * (q.prod(-1) + p.prod(-1)), atol=1e-12)


@pytest.mark.parametrize("k", [1, 4, 17, 64, 301, 512])
def test_equal_literals_are_binomial(k):
    """With every l_i equal, T ~ Binomial(k, p); CARD, EK, AMO and EO reduce to
    binomial tail and point probabilities."""
    for lv in [-0.9, -0.3, 0.0, 0.45, 0.99]:
        p = (1 - lv) / 2
        ell = np.full((1, k), lv)
        pmf = np.array([math.comb(k, t) * p ** t * (1 - p) ** (k - t) for t in range(k + 1)])
        for r in sorted({0, 1, k // 3, k // 2, k}):
            got = O.fe(O.truth_table(O.T_CARD, k, O.OP_GE, r), ell)[0]
            assert abs(got - (1 - 2 * pmf[r:].sum())) < 1e-11
            got = O.fe(O.truth_table(O.T_CARD, k, O.OP_LT, r), ell)[0]
            assert abs(got - (1 - 2 * pmf[:r].sum())) < 1e-11
            got = O.fe(O.truth_table(O.T_EK, k, param=r), ell)[0]
            assert abs(got - (1 - 2 * pmf[r])) < 1e-11
        assert abs(O.fe(O.truth_table(O.T_AMO, k), ell)[0] - (1 - 2 * pmf[:2].sum())) < 1e-11
        assert abs(O.fe(O.truth_table(O.T_EO, k), ell)[0] - (1 - 2 * pmf[1])) < 1e-11


@pytest.mark.parametrize("k", [1, 5, 33, 128])
def test_center_is_uniform_mean(k):
    for f in _tables_for(k):
        want = sum(math.comb(k, t) * f[t] for t in range(k + 1)) / 2.0 ** k
        assert abs(O.fe(f, np.zeros((1, k)))[0] - want) < 1e-12


# --- vertex property and multilinearity ------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 8, 31, 100])
def test_vertex_values_are_exact(k):
    """At l in {+-1}^k the expansion equals f(t) exactly (Sec. 2.1.1)."""
    rng = np.random.default_rng(k + 3)
    ell = np.where(rng.random((16, k)) < 0.5, -1.0, 1.0)
    t = (ell < 0).sum(-1)
    for f in _tables_for(k):
        assert np.array_equal(O.fe(f, ell), f[t])


@pytest.mark.parametrize("k", [2, 3, 9, 20, 65])
def test_gradient_is_exact_difference(k):
    """The expansion is affine in each l_i, so dFE/dl_i = (FE|l_i=1 - FE|l_i=-1)/2
    and also equals the central difference at any step h."""
    rng = np.random.default_rng(11 * k)
    ell = rng.uniform(-1, 1, (3, k))
    for f in _tables_for(k)[:8]:
        _, d = O.fe_and_dfe(f, ell)
        for i in range(k):
            hi, lo = ell.copy(), ell.copy()
            hi[:, i], lo[:, i] = 1.0, -1.0
            np.testing.assert_allclose(d[:, i], (O.fe(f, hi) - O.fe(f, lo)) / 2, atol=1e-12)
            h = 0.37
            hi[:, i], lo[:, i] = ell[:, i] + h, ell[:, i] - h
            np.testing.assert_allclose(d[:, i], (O.fe(f, hi) - O.fe(f, lo)) / (2 * h), atol=1e-11)


# --- instance level ---------------------------------------------------------
def test_instance_gradient_is_central_difference_in_x():
    """Variables are distinct inside each constraint, so the objective is affine
    in each x_v: its exact central difference checks the sign handling and the
    scatter over occurrences."""
    inst = synth.mixed_small(1, n=14, m=25, kmax=7)
    x = synth.uniform_x0(inst.n, 3, 5).astype(np.float64)
    _, go, g = O.evaluate(inst, x)
    h = 0.25
    for v in range(inst.n):
        xp, xm = x.copy(), x.copy()
        xp[v] += h
        xm[v] -= h
        fd = (O.objective(inst, xp) - O.objective(inst, xm)) / (2 * h)
        np.testing.assert_allclose(g[v], fd, atol=1e-12)
    # per-occurrence values sum to the per-variable gradient
    var = np.abs(inst.lits) - 1
    acc = np.zeros_like(g)
    np.add.at(acc, var, go)
    np.testing.assert_allclose(acc, g, atol=1e-14)


def test_unsat_count_matches_objective_at_vertices():
    """At a vertex every FE_c is -1 or +1, so sum_c FE_c = -m + 2 * unsat."""
    for idx in range(4):
        inst = synth.mixed_small(idx, n=30, m=50, kmax=9)
        x = synth.vertex_x0(inst.n, 8, idx)
        obj = O.objective(inst, x)
        un = O.unsat_count(inst, x)
        np.testing.assert_array_equal(obj, -inst.m + 2 * un.astype(np.float64))


def test_unsat_count_by_plain_loop():
    inst = synth.mixed_small(9, n=12, m=30, kmax=6)
    x = synth.uniform_x0(inst.n, 5, 2)
    x[0, 0] = 0.0
    x[1, 1] = -0.0
    un = O.unsat_count(inst, x)
    for b in range(x.shape[1]):
        cnt = 0
        for c in range(inst.m):
            t = 0
            for lit in inst.constraint(c):
                val = x[abs(lit) - 1, b]
                is_true = (val < 0) if lit > 0 else not (val < 0)
                t += int(is_true)
            k = len(inst.constraint(c))
            ok = O.satisfied(int(inst.ctype[c]), k, t, int(inst.op[c]), int(inst.param[c]),
                             int(inst.parity[c]))
            cnt += 0 if ok else 1
        assert un[b] == cnt


def test_sat_criterion_on_exhaustive_models():
    """A model found by enumeration has unsat = 0 and objective exactly -m."""
    for idx in range(6):
        inst = synth.random_ksat(12, 40, 3, synth.rng_for(200, idx))
        sat, model = O.exhaustive_sat(inst)
        if sat:
            x = model.astype(np.float32)[:, None]
            assert O.unsat_count(inst, x)[0] == 0
            assert O.objective(inst, x)[0] == -inst.m


def test_dpll_agrees_with_enumeration():
    seen = set()
    for idx in range(24):
        n = 10 + idx % 8
        inst = synth.random_ksat(n, int(round(4.6 * n)), 3, synth.rng_for(201, idx))
        sat, _ = O.exhaustive_sat(inst)
        assert O.dpll(inst) == sat
        seen.add(sat)
    assert seen == {True, False}


def test_pgd_step_single_clause_closed_form():
    """One clause (x1 or x2 or x3): FE = -1 + 2 prod (1 + x_i)/2, so at x = 0 the
    gradient is 1/4 per variable and a unit step lands at -1/4."""
    b = synth._Builder(3)
    b.add(synth.OR, [1, 2, 3])
    inst = b.build()
    x = np.zeros((3, 1))
    np.testing.assert_allclose(O.pgd_step(inst, x, 1.0), np.full((3, 1), -0.25), atol=1e-15)
    # projection: a huge step is clamped to the box
    np.testing.assert_allclose(O.pgd_step(inst, x, 100.0), np.full((3, 1), -1.0))


# --- golden fixtures from the paper and from the RNG's publication ----------
def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_appendix_a_semantics():
    names = {n: i for i, n in enumerate(synth.TYPE_NAMES)}
    rows = _read_golden("appendix_a_semantics.txt")
    assert len(rows) == 11
    for row in rows:
        ctype, k, thr, opstr, parity = names[row[0]], int(row[1]), int(row[2]), row[3], int(row[4])
        want = np.array([float(v) for v in row[5:]])
        assert want.shape == (k + 1,)
        op, r = O.OP_GE, thr
        if ctype == O.T_CARD:
            op, r = O.normalise_card(thr, None if opstr == "none" else opstr)
        got = O.truth_table(ctype, k, op, r, parity)
        np.testing.assert_array_equal(got, want)


def test_philox_known_answers():
    rows = _read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for row in rows:
        vals = [int(v, 16) for v in row]
        ctr = np.array(vals[0:4], dtype=np.uint64)
        key = np.array(vals[4:6], dtype=np.uint64)
        out = O.philox4x32_10(ctr, key)
        assert [int(v) for v in out] == vals[6:10]


def test_philox_uniform_x0_properties():
    x = O.philox_uniform_x0(12345, 64, 40)
    assert x.dtype == np.float32 and x.shape == (64, 40)
    assert x.min() >= -1.0 and x.max() < 1.0
    assert abs(float(x.mean())) < 0.05
    # exact 24-bit grid: (x + 1) / 2 * 2^24 is an integer
    u = (x.astype(np.float64) + 1) / 2 * 2 ** 24
    assert np.all(u == np.round(u))
    # different seeds and streams give different points
    assert not np.array_equal(x, O.philox_uniform_x0(12346, 64, 40))
    assert not np.array_equal(x, O.philox_uniform_x0(12345, 64, 40, stream=1))


# ---- the line-search step -------------------------------------------------------
def test_armijo_single_trial_is_the_fixed_step():
    inst = synth.mixed_small(1)
    x = synth.uniform_x0(inst.n, 12, 3).astype(np.float64)
    got, chosen = O.armijo_step(inst, x, 0.07, 0.5, 1e-4, 1)
    np.testing.assert_allclose(got, O.pgd_step(inst, x, 0.07), rtol=0, atol=1e-15)
    assert np.all(chosen <= 0)


def test_armijo_choice_satisfies_and_previous_violates_the_condition():
    """The accepted trial meets the sufficient-decrease inequality, every larger
    trial breaks it, and accepted steps never increase the objective."""
    inst = synth.mixed_small(4)
    x = synth.uniform_x0(inst.n, 40, 4).astype(np.float64)
    s, beta, c, T = 30.0, 0.5, 1e-4, 8   # large first steps, so that some restarts backtrack
    got, chosen = O.armijo_step(inst, x, s, beta, c, T)
    _, _, g = O.evaluate(inst, x)
    f0 = O.objective(inst, x)

    def cond(i):
        xi = np.clip(x - s * beta ** i * g, -1, 1)
        return O.objective(inst, xi) <= f0 + c * (g * (xi - x)).sum(axis=0)

    conds = np.stack([cond(i) for i in range(T)])
    for b in range(x.shape[1]):
        if chosen[b] >= 0:
            assert conds[chosen[b], b] and not conds[:chosen[b], b].any()
            assert O.objective(inst, got[:, [b]])[0] <= f0[b] + 1e-12
        else:
            assert not conds[:, b].any()
    assert np.any(chosen > 0) and np.any(chosen == 0)
