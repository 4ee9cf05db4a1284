"""CPU tests of the C-ABI library's host logic (no device work).

The library must load and export every symbol that include/afsat.h declares;
its load-time coefficient tables, evaluated here in FP64 exactly as the
kernels combine them, must reproduce the oracle's expansion and gradient; its
exact-integer ESP coefficients must equal the Walsh coefficients computed from
their definition; and malformed records must be rejected before any CUDA call.
"""
import os
import re

import numpy as np
import pytest

from oracle import fe_oracle as O
from paper_2606_06641_gb300 import binding as bd
from paper_2606_06641_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_2606_06641_gb300 import build
    build.build()
    yield


def _header_symbols():
    txt = open(os.path.join(ROOT, "include", "afsat.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(afs_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    syms = _header_symbols()
    assert len(syms) >= 20
    lib = bd.lib()
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(bd.SIGNATURES), set(syms) ^ set(bd.SIGNATURES)
    assert "sm_103a" in bd.version()


def test_library_resolves_every_symbol_at_load():
    """Loading the library with immediate binding (RTLD_NOW, a fresh process)
    resolves every symbol it uses: a declaration with the wrong linkage or a
    missing definition fails here instead of at its first call under lazy
    binding."""
    import subprocess
    import sys
    path = bd.lib()._name
    code = "import ctypes, os, sys; ctypes.CDLL(sys.argv[1], mode=os.RTLD_NOW)"
    r = subprocess.run([sys.executable, "-c", code, path], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]


def _eval_short(tab, k, esp, ell):
    """FE and dFE/dl for ell[B, k] from a short-form table, in float64."""
    t = tab.astype(np.float64).reshape(-1, 4)
    fe = np.full(ell.shape[0], t[0, 0])
    grad = np.zeros_like(ell)
    nreal = (k & 1) + (1 if esp else 0)
    for q in range(nreal):
        alpha, E = t[1 + q, 0], t[1 + q, 1]
        f = ell + alpha
        fe += E * f.prod(axis=1)
        for i in range(k):
            grad[:, i] += E * np.delete(f, i, axis=1).prod(axis=1)
    n_scaled = 0 if esp else int(t[0, 1])
    # scaled tables (PGF, k <= 24) store only their nonzero complex roots
    n_complex = n_scaled if (not esp and k <= 24) else k // 2
    for j in range(n_complex):
        if j < n_scaled:  # factor (w + i), w = l / gamma, stored as 1/gamma
            inv_gam, _, er, ei = t[1 + nreal + j]
            E = er + 1j * ei
            f = ell * inv_gam + 1j
            fe += np.real(E * f.prod(axis=1))
            for i in range(k):
                grad[:, i] += np.real(E * inv_gam * np.delete(f, i, axis=1).prod(axis=1))
            continue
        alpha, gam, er, ei = t[1 + nreal + j]
        E = er + 1j * ei
        f = ell + alpha + 1j * gam
        fe += np.real(E * f.prod(axis=1))
        for i in range(k):
            grad[:, i] += np.real(E * np.delete(f, i, axis=1).prod(axis=1))
    return fe, grad


def _eval_long_pgf(tab, k, ell):
    """The long probability-generating table walked the way the kernel walks
    it, in FP64: per kept complex root the factor g = p l + i (form A) or
    l + i p (form B, roots from the head's first form-B index on), segments
    of 16 literals with the stored s^16 after each full one; the value
    Re(E' P) and each literal's derivative Re(E' P g'(l_i) / g(l_i)), its
    factor divided out of the full product (g' = p in form A, 1 in form B);
    the real root (odd k) as c_mid prod l."""
    t = tab.astype(np.float64).reshape(-1, 4)
    c0, nr, cmid, has_real = t[0]
    first_b = int(t[1, 0])
    rows = ell.shape[0]
    nseg = (k + 15) // 16
    fe = np.full(rows, c0)
    grad = np.zeros_like(ell)
    for j in range(int(nr)):
        g0, g1 = t[2 + 2 * j], t[3 + 2 * j]
        p, s16, E = g0[0], g0[1] + 1j * g0[2], g1[0] + 1j * g1[1]
        fb = j >= first_b
        g = (ell + 1j * p) if fb else (p * ell + 1j)
        P = np.ones(rows, dtype=np.complex128)
        for sg in range(nseg):
            i0 = 16 * sg
            P = P * g[:, i0:min(k, i0 + 16)].prod(axis=1)
            if sg < nseg - 1:
                P = P * s16
        T = E * P
        fe += np.real(T)
        grad += np.real((T * (1.0 if fb else p))[:, None] / g)
    if has_real > 0.5:
        fe += cmid * ell.prod(axis=1)
        for i in range(k):
            grad[:, i] += cmid * np.delete(ell, i, axis=1).prod(axis=1)
    return fe, grad


def _eval_long(tab, k, esp, ell):
    if not esp:
        return _eval_long_pgf(tab, k, ell)
    t = tab.astype(np.float64).reshape(-1, 4)
    fe = np.full(ell.shape[0], t[0, 0])
    grad = np.zeros_like(ell)
    nroots = k // 2 + (k & 1) + (1 if esp else 0)
    for j in range(nroots):
        Ar, Ai, br, bi = t[1 + 2 * j]
        dr, di, er, ei = t[2 + 2 * j]
        f = (Ar + 1j * Ai) - (br + 1j * bi) * (1.0 - ell)
        fe += np.real((er + 1j * ei) * f.prod(axis=1))
        for i in range(k):
            grad[:, i] += np.real((dr + 1j * di) * np.delete(f, i, axis=1).prod(axis=1))
    return fe, grad


def _shapes(k):
    out = [(O.T_OR, 0, 0, 1), (O.T_XOR, 0, 0, 1), (O.T_XOR, 0, 0, 0), (O.T_NAE, 0, 0, 1), (O.T_AMO, 0, 0, 1),
           (O.T_EO, 0, 0, 1)]
    for r in sorted({0, 1, k // 2, k}):
        out += [(O.T_EK, 0, r, 1), (O.T_CARD, O.OP_GE, r, 1), (O.T_CARD, O.OP_LT, r, 1)]
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 13, 20, 24, 25, 32])
def test_short_pgf_table_reproduces_oracle(k):
    rng = np.random.default_rng(k)
    ell = np.concatenate([rng.uniform(-1, 1, (5, k)), np.sign(rng.uniform(-1, 1, (2, k)))])
    for (ct, op, r, par) in _shapes(k):
        tab = bd.coef_table(ct, k, op, r, par, basis=bd.BASIS_PGF, form=0)
        f = O.truth_table(ct, k, op, r, par)
        fe, g = _eval_short(tab, k, False, ell)
        ref_fe, ref_g = O.fe_and_dfe(f, ell)
        np.testing.assert_allclose(fe, ref_fe, atol=2e-6, rtol=0)
        np.testing.assert_allclose(g, ref_g, atol=2e-6, rtol=0)


@pytest.mark.parametrize("k", [1, 3, 16, 17, 33, 64, 101, 128, 129, 160, 255, 300, 512])
def test_long_pgf_table_reproduces_oracle(k):
    """The FP32 long table, walked in FP64 as the kernel walks it, against the
    oracle at interior, near-vertex and vertex points: with the coefficients
    solved for the FP32 nodes the error stays at FP32 rounding of the table,
    not k times it."""
    rng = np.random.default_rng(50 + k)
    ell = np.concatenate([rng.uniform(-1, 1, (2, k)), np.sign(rng.uniform(-1, 1, (2, k))),
                          np.sign(rng.uniform(-1, 1, (1, k))) * (1 - 1e-3 * rng.uniform(0, 1, (1, k)))])
    shapes = _shapes(k)
    if k > 128:
        shapes = shapes[:2] + shapes[6:]
    for (ct, op, r, par) in shapes:
        tab = bd.coef_table(ct, k, op, r, par, basis=bd.BASIS_PGF, form=1)
        f = O.truth_table(ct, k, op, r, par)
        fe, g = _eval_long(tab, k, False, ell)
        ref_fe, ref_g = O.fe_and_dfe(f, ell)
        np.testing.assert_allclose(fe, ref_fe, atol=1e-6, rtol=0, err_msg=str((ct, op, r, par)))
        np.testing.assert_allclose(g, ref_g, atol=1e-6, rtol=0, err_msg=str((ct, op, r, par)))


@pytest.mark.parametrize("k", [1, 2, 3, 6, 9, 12])
def test_esp_tables_reproduce_oracle_at_small_k(k):
    """The paper's basis: prod (1 + w^j l) combined with the DFT of f_hat(|S|=d)."""
    rng = np.random.default_rng(90 + k)
    ell = rng.uniform(-1, 1, (4, k))
    for (ct, op, r, par) in _shapes(k):
        f = O.truth_table(ct, k, op, r, par)
        ref_fe, ref_g = O.fe_and_dfe(f, ell)
        for form, ev in ((0, _eval_short), (1, _eval_long)):
            tab = bd.coef_table(ct, k, op, r, par, basis=bd.BASIS_ESP, form=form)
            fe, g = ev(tab, k, True, ell)
            np.testing.assert_allclose(fe, ref_fe, atol=2e-5, rtol=0)
            np.testing.assert_allclose(g, ref_g, atol=2e-5, rtol=0)


@pytest.mark.parametrize("k", [1, 2, 5, 8, 10])
def test_esp_coefficients_equal_walsh_definition(k):
    for (ct, op, r, par) in _shapes(k):
        f = O.truth_table(ct, k, op, r, par)
        fhat = O.walsh_coefficients(f)
        c = bd.esp_coefficients(ct, k, op, r, par)
        masks = np.arange(1 << k)
        sizes = np.array([bin(mm).count("1") for mm in masks])
        for d in range(k + 1):
            np.testing.assert_allclose(fhat[sizes == d], c[d], atol=1e-15)


def test_esp_coefficients_exact_at_large_k():
    """f_hat(|S| = d) of odd parity is 1 at d = k and 0 elsewhere; of CARD >= 1
    (OR) it is 2^(1-k) for d >= 1 and 2^(1-k) - 1 at d = 0 - exact at any k."""
    for k in (40, 127, 300):
        c = bd.esp_coefficients(O.T_XOR, k, 0, 0, 1)
        want = np.zeros(k + 1)
        want[k] = 1.0
        np.testing.assert_array_equal(c, want)
        c = bd.esp_coefficients(O.T_OR, k)
        want = np.full(k + 1, 2.0 ** (1 - k))
        want[0] -= 1.0
        np.testing.assert_array_equal(c, want)


def test_pgf_table_has_exact_conjugate_roots():
    """Short-form roots: gamma_j = cot(pi j/(k+1)) (stored as tan for the scaled
    form up to k = 24, as cot beyond), and the mirrored middle root of an odd
    length has a purely real weight."""
    for k in (5, 9, 23, 25, 31):
        t = bd.coef_table(O.T_CARD, k, O.OP_GE, k // 2).reshape(-1, 4)
        ang = np.pi * np.arange(1, k // 2 + 1) / (k + 1)
        if k <= 24:
            # the stored roots are a subsequence of j = 1..k/2 (zero ones dropped)
            assert 1 <= t[0, 1] <= k // 2 and t.shape[0] == 2 + int(t[0, 1])
            tans = np.tan(ang).astype(np.float32)
            idx = [int(np.argmin(np.abs(tans - v))) for v in t[2:, 0]]
            assert idx == sorted(set(idx))
            np.testing.assert_allclose(t[2:, 0], tans[idx], rtol=2e-7)
            assert np.all(t[2:, 1] == 0.0)
        else:
            assert t[0, 1] == 0
            np.testing.assert_allclose(t[2:, 1], (1.0 / np.tan(ang)).astype(np.float32), rtol=2e-7)
            assert np.all(t[2:, 0] == 0.0)
        assert t[1, 0] == 0.0 and t[1, 2] == 0.0 and t[1, 3] == 0.0


def _bad(inst_kw):
    b = synth._Builder(5)
    for rec in inst_kw:
        b.add(*rec)
    return b.build()


@pytest.mark.parametrize("records,code", [
    ([(synth.OR, [1, 2, 6])], -2),       # variable beyond n
    ([(synth.OR, [1, 0, 2])], -2),       # literal zero
    ([(synth.OR, [])], -3),              # empty constraint
    ([(9, [1, 2])], -4),                 # unknown type
    ([(synth.CARD, [1, 2], 7, 1)], -4),  # unknown CARD operator
])
def test_invalid_records_rejected_before_device_work(records, code):
    inst = _bad(records)
    with pytest.raises(bd.AfsError) as ei:
        bd.load_instance(inst, stream=0)
    assert ei.value.code == code


def test_overlong_constraint_rejected():
    b = synth._Builder(2000)
    b.add(synth.CARD, list(range(1, bd.MAX_LEN + 2)), synth.GE, 3)
    with pytest.raises(bd.AfsError) as ei:
        bd.load_instance(b.build(), stream=0)
    assert ei.value.code == -3


def test_parity_tables_keep_only_the_nonzero_root():
    """The spectrum of an odd-length parity constraint is the single root
    w = -1: a scaled table stores no complex root whose coefficient is zero,
    and it still reproduces the oracle."""
    rng = np.random.default_rng(7)
    for k in (3, 5, 7, 9):
        for par in (0, 1):
            tab = bd.coef_table(O.T_XOR, k, 0, 0, par, basis=bd.BASIS_PGF, form=0)
            t = tab.reshape(-1, 4)
            assert t[0, 1] == 0 and t.shape[0] == 2   # head and the real root only
            ell = rng.uniform(-1, 1, (4, k))
            fe, g = _eval_short(tab, k, False, ell)
            ref_fe, ref_g = O.fe_and_dfe(O.truth_table(O.T_XOR, k, 0, 0, par), ell)
            np.testing.assert_allclose(fe, ref_fe, atol=2e-6, rtol=0)
            np.testing.assert_allclose(g, ref_g, atol=2e-6, rtol=0)


def test_tile_spec_round_trip():
    spec = "1024:3=4x2,4=2x1,5=4x1,20=1x1"
    chunk, tiles = bd.parse_tiles(spec)
    assert chunk == 1024 and tiles == {3: (4, 2), 4: (2, 1), 5: (4, 1), 20: (1, 1)}
    assert bd.format_tiles(chunk, tiles) == spec
    assert bd.parse_tiles("0:") == (0, {})


def test_length3_level_expansion_derivative():
    """The fused pass's derivative of a length-3 constraint in its first
    variable, x1 (A x2 + B1) + B2 x2 + C with A = s c3 s1 s2, B1 = s c2 s1,
    B2 = s c2 s2, C = s c1 (c_d the library's level coefficients, l = s x),
    equals the oracle's s * dFE/dl for every shape and sign pattern."""
    rng = np.random.default_rng(33)
    x = rng.uniform(-1, 1, (6, 3))
    for (ct, op, r, par) in _shapes(3):
        f = O.truth_table(ct, 3, op, r, par)
        c = bd.esp_coefficients(ct, 3, op, r, par)
        for signs in ((1, 1, 1), (-1, 1, -1), (1, -1, -1), (-1, -1, 1)):
            s = np.array(signs, dtype=np.float64)
            _, g = O.fe_and_dfe(f, x * s)
            want = s[0] * g[:, 0]
            A, B1, B2, C = s[0] * c[3] * s[1] * s[2], s[0] * c[2] * s[1], s[0] * c[2] * s[2], s[0] * c[1]
            got = x[:, 1] * (A * x[:, 2] + B1) + B2 * x[:, 2] + C
            np.testing.assert_allclose(got, want, atol=1e-14, rtol=0)


@pytest.mark.parametrize("k", list(range(33, 513, 29)) + [63, 64, 65, 100, 101, 128, 255, 256, 257, 480, 511, 512])
def test_long_pgf_table_forms_stay_in_range(k):
    """Layout of a long probability-generating table: the kept roots are
    exactly those with a nonzero coefficient (an odd-length parity keeps only
    the real root), form B starts at a multiple of 32 (so 8-, 16- and 32-root
    passes never straddle it), and for |l| <= 1 each root's factor modulus
    |g| <= 1/|s| (the true factor |s g| <= 1) while the per-segment power
    s^16 stays a normal FP32 number (|s|^16 >= 2^-100), so the forward walk's
    running product stays within 2^100 of its true size inside a segment."""
    for (ct, op, r, par) in [(O.T_CARD, O.OP_GE, k // 2, 1), (O.T_EK, 0, k // 3, 1), (O.T_XOR, 0, 0, 1),
                             (O.T_OR, 0, 0, 1)]:
        t = bd.coef_table(ct, k, op, r, par, basis=bd.BASIS_PGF, form=1).astype(np.float64).reshape(-1, 4)
        n, has_real, fb = int(t[0, 1]), t[0, 3], int(t[1, 0])
        nx, nc = int(t[1, 1]), int(t[1, 2])
        assert t.shape[0] == 2 + 2 * n + nx * nc // 4
        # kept roots = nonzero exact spectrum (pairs j = 1..k/2); the real root w = -1 (odd k)
        f = O.truth_table(ct, k, op, r, par).astype(np.float64)
        N = k + 1
        spec = np.fft.fft(f) / N
        assert has_real == (1.0 if k % 2 == 1 and abs(spec[N // 2]) > 1e-13 else 0.0)
        if ct == O.T_XOR and k % 2 == 1:
            assert n == 0 and has_real == 1.0   # odd-length parity: only the real root
        assert n == int(np.sum(np.abs(spec[1:k // 2 + 1]) > 1e-13))
        assert fb == n or fb % 32 == 0
        for j in range(n):
            p = t[2 + 2 * j, 0]
            s16 = t[2 + 2 * j, 1] + 1j * t[2 + 2 * j, 2]
            s_mod = abs(s16) ** (1 / 16)
            gmax = np.sqrt(1 + p * p)   # |p l + i| (form A) or |l + i p| (form B) at |l| <= 1
            assert gmax <= 1.0 / s_mod * (1 + 1e-5)        # |g| <= 1/|s| (|f| <= 1)
            assert abs(s16) >= 2.0 ** -100
        # expanded roots: a multiple of 32, all in form A, 16 or 32 terms
        assert nx % 32 == 0 and nx <= fb and (nc in (16, 32) if nx else nc == 0)


@pytest.mark.parametrize("k", [100, 130, 200, 256, 300, 401, 512])
def test_long_pgf_expansion_terms_approximate_the_derivative_factor(k):
    """The expanded roots' stored terms c_n: sum_n c_n T_n(2u - 1) evaluated
    by numpy's Chebyshev series in FP64 equals 1 / (p^2 u + 1), the form-A
    derivative term's denominator, on u in [0, 1] to the FP32 rounding of the
    stored terms (relative to the function's smallest value there, 1 / (p^2 +
    1))."""
    t = bd.coef_table(O.T_CARD, k, O.OP_GE, k // 2, 1, basis=bd.BASIS_PGF, form=1).astype(np.float64).reshape(-1, 4)
    n, nx, nc = int(t[0, 1]), int(t[1, 1]), int(t[1, 2])
    if k >= 200:
        assert nx >= 64  # long tables expand most roots
    c = t[2 + 2 * n:].reshape(-1)
    assert c.size == nx * nc
    u = np.linspace(0.0, 1.0, 1001)
    for j in range(nx):
        p = t[2 + 2 * j, 0]
        exact = 1.0 / (p * p * u + 1.0)
        approx = np.polynomial.chebyshev.chebval(2.0 * u - 1.0, c[j * nc:(j + 1) * nc])
        assert np.max(np.abs(approx - exact)) * (p * p + 1.0) < 4e-7


def _paper_basis_fp64(c, ell):
    """Sec. 2.1.2's products in the paper's basis in FP64: the DFT over d of
    f_hat(|S| = d) combined with prod_i (1 + w^j l_i) at the k+1 roots."""
    k = ell.size
    N = k + 1
    w = np.exp(2j * np.pi * np.arange(N) / N)
    d = np.arange(k + 1)
    chat = np.array([np.sum(c * w[j] ** (-d)) for j in range(N)]) / N
    return float(np.real(np.sum(chat * np.prod(1 + np.outer(w, ell), axis=1))))


def _pgf_basis_fp64(f, ell):
    """The probability-generating basis in FP64: DFT of the truth table
    combined with prod_i (q_i + p_i w^j)."""
    k = ell.size
    N = k + 1
    w = np.exp(2j * np.pi * np.arange(N) / N)
    ft = np.fft.fft(f.astype(np.float64)) / N          # sum_t f(t) w^{-jt} / N
    p = (1 - ell) / 2
    return float(np.real(np.sum(ft * np.prod((1 - p)[None, :] + np.outer(w, p), axis=1))))


def test_paper_basis_fp64_ceiling():
    """Sec. 3.4's floating-point limit, reproduced from the library's exact
    ESP coefficients: evaluated in FP64, the paper's basis loses accuracy as
    the products reach 2^k near the all-false vertex (the satisfying region of
    an at-most-one constraint), from about 1e-5 at k = 40 to a degenerate
    1e-2 at k = 48 and worse beyond; the probability-generating basis stays
    at rounding level at the same points."""
    rng = np.random.default_rng(0)
    worst = {}
    for k in (32, 40, 48, 56, 64):
        c = bd.esp_coefficients(O.T_AMO, k)
        f = O.truth_table(O.T_AMO, k)
        e_paper, e_pgf = [], []
        for _ in range(10):
            ell = 1.0 - 0.05 * rng.random(k)
            ref = O.fe(f, ell[None])[0]
            e_paper.append(abs(_paper_basis_fp64(c, ell) - ref))
            e_pgf.append(abs(_pgf_basis_fp64(f, ell) - ref))
        worst[k] = max(e_paper)
        assert max(e_pgf) < 1e-12, (k, max(e_pgf))
    assert worst[32] < 1e-5 and worst[40] < 1e-3
    assert worst[48] > 1e-3 and worst[56] > 1e-1 and worst[64] > 1.0
    assert worst[32] < worst[40] < worst[48] < worst[56] < worst[64]
