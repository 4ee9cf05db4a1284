"""GPU parity of the CUDA path against the FP64 CPU oracle (through the C ABI).

Tolerances (FP32 arithmetic against FP64): an expansion value must lie within
1e-5 * max(1, |FE_ref|) of the oracle; a variable's gradient within
1e-5 * max(1, sum over its occurrences of |s_i dFE/dl_i|). With BF16 storage
of x the arithmetic is checked at the dequantised point against the same 1e-5
and the end-to-end value at the original FP32 point against 2e-2. Integer
work (unsat counts, sign rounding, the counter-based starting points) must be
bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe_oracle as O
from paper_2606_06641_gb300 import binding as bd
from paper_2606_06641_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06641_gb300 import build
    build.build()
    yield


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _grad_scale(inst, go_ref):
    var = np.abs(inst.lits) - 1
    acc = np.zeros((inst.n, go_ref.shape[1]))
    np.add.at(acc, var, np.abs(go_ref))
    return np.maximum(1.0, acc)


def _check_eval(inst, x, params=None, tol=TOL, x_dtype=torch.float32, x_ref=None):
    h = bd.load_instance(inst, params)
    xd = _dev(x, x_dtype)
    fe, g = bd.eval_fe_grad(h, xd)
    torch.cuda.synchronize()
    xr = x if x_ref is None else x_ref
    fe_ref, go_ref, g_ref = O.evaluate(inst, xr.astype(np.float64))
    fe = fe.cpu().numpy()
    g = g.cpu().numpy()
    fe_err = np.abs(fe - fe_ref) / np.maximum(1.0, np.abs(fe_ref))
    g_err = np.abs(g - g_ref) / _grad_scale(inst, go_ref)
    assert fe_err.max() <= tol, f"FE error {fe_err.max():.3e}"
    assert g_err.max() <= tol, f"gradient error {g_err.max():.3e}"
    return fe_err.max(), g_err.max()


# ---- expansion and gradient ------------------------------------------------
@pytest.mark.parametrize("idx", range(4))
def test_mixed_types_eval(idx):
    inst = synth.mixed_small(idx, n=60, m=120, kmax=12)
    for B, gen in ((37, synth.uniform_x0), (70, synth.near_vertex_x0), (5, synth.vertex_x0)):
        _check_eval(inst, gen(inst.n, B, idx))


@pytest.mark.parametrize("k", list(range(1, 33)))
def test_every_short_length(k):
    """All 32 register-kernel lengths, several types, ragged restart counts."""
    for t, op, r, par in ((synth.OR, 0, 0, 1), (synth.XOR, 0, 0, k % 2), (synth.CARD, synth.GE, (k + 1) // 2, 1),
                          (synth.EK, 0, k // 3, 1), (synth.NAE, 0, 0, 1)):
        inst = synth.single_type(t, k, 9, max(2 * k, 12), index=k, op=op, param=r, parity=par)
        _check_eval(inst, synth.uniform_x0(inst.n, 45, k))


@pytest.mark.parametrize("k", [33, 40, 47, 48, 63, 64, 65, 100, 101, 128, 129, 255, 256, 257, 480, 511, 512])
def test_long_lengths(k):
    """Every length class of the long kernel up to AFS_MAX_LEN = 512 (the
    longest constraints of the workloads), tails of 1..16 literals in the last
    segment, at uniform, near-vertex and vertex points: within 1e-5."""
    for t, op, r in ((synth.CARD, synth.GE, k // 2), (synth.EK, 0, k // 3), (synth.AMO, 0, 0),
                     (synth.CARD, synth.LT, 3 * k // 4)):
        inst = synth.single_type(t, k, 3, k + 7, index=k, op=op, param=r)
        _check_eval(inst, synth.uniform_x0(inst.n, 19, k))
        _check_eval(inst, synth.near_vertex_x0(inst.n, 11, k, spread=0.02))
        _check_eval(inst, synth.vertex_x0(inst.n, 6, k))


@pytest.mark.parametrize("k", [64, 101, 256, 301, 512])
def test_long_lengths_at_exact_zeros(k):
    """The long kernel divides each literal's factor out of the root's full
    product. Points where literal values are exactly 0 make the second-form
    factors l + i p as small as they get (i p), and the real root's factor
    (odd k) exactly 0; points mixing 0 with the vertices -1, +1 and interior
    values must still match the oracle within 1e-5."""
    rng = np.random.default_rng(700 + k)
    for t, op, r, par in ((synth.CARD, synth.GE, k // 2, 1), (synth.XOR, 0, 0, 1), (synth.EK, 0, k // 3, 1),
                          (synth.NAE, 0, 0, 1)):
        inst = synth.single_type(t, k, 2, k + 3, index=k + 3 * t, op=op, param=r, parity=par)
        B = 12
        x = rng.choice(np.array([0.0, -1.0, 1.0, 0.3, -0.7]), size=(inst.n, B), p=[0.4, 0.15, 0.15, 0.15, 0.15])
        x[:, 0] = 0.0                      # every literal exactly 0
        x[: inst.n // 2, 1] = 0.0          # half of them 0, the rest interior
        x[inst.n // 2:, 1] = rng.uniform(-1, 1, inst.n - inst.n // 2)
        _check_eval(inst, x.astype(np.float32))


@pytest.mark.parametrize("k", [100, 101, 102, 127, 200, 393, 480])
def test_long_form_boundaries(k):
    """Lengths where the long tables switch the passes of roots near pi/2 to
    the second factor form (from about k = 100 on), for parity (odd k keeps
    only the real root, even k every complex root), NAE, EO and a threshold,
    at uniform and near-vertex points."""
    for t, op, r, par in ((synth.XOR, 0, 0, 1), (synth.XOR, 0, 0, 0), (synth.NAE, 0, 0, 1), (synth.EO, 0, 0, 1),
                          (synth.CARD, synth.GE, k // 2, 1)):
        inst = synth.single_type(t, k, 2, k + 5, index=k + t, op=op, param=r, parity=par)
        _check_eval(inst, synth.uniform_x0(inst.n, 13, k))
        _check_eval(inst, synth.near_vertex_x0(inst.n, 7, k, spread=0.02))


def test_every_long_tile():
    """Every tile of the long kernel (8, 16 or 32 lanes per restart; 2, 4 or 8
    warps per CTA) on a mix of long lengths and types, ragged restart count:
    lengths 43..406 cover tables without expanded roots, with 16 and with 32
    Chebyshev terms (a slot of 8 lanes takes the 32-term tables' roots
    exactly, one of 16 holds two terms a lane)."""
    inst = synth.long_card_n10000(3, n=600, n_clauses=200, n_long=10, kmin=33, kmax=512)
    x = synth.uniform_x0(inst.n, 29, 5)
    h = bd.load_instance(inst)
    groups = bd.long_tiles(h)
    assert groups and all(t[2] > 32 for t in groups)
    fe_ref, go_ref, g_ref = O.evaluate(inst, x.astype(np.float64))
    for tile in ((32, 4), (32, 8), (16, 2), (16, 4), (8, 2)):
        bd.set_long_tiles(h, [tile] * len(groups))
        assert all(t[:2] == tile for t in bd.long_tiles(h))
        fe, g = bd.eval_fe_grad(h, _dev(x))
        fe_err = np.abs(fe.cpu().numpy() - fe_ref) / np.maximum(1.0, np.abs(fe_ref))
        g_err = np.abs(g.cpu().numpy() - g_ref) / _grad_scale(inst, go_ref)
        assert fe_err.max() <= TOL and g_err.max() <= TOL, (tile, fe_err.max(), g_err.max())
    with pytest.raises(bd.AfsError):
        bd.set_long_tiles(h, [(8, 4)] * len(groups))


def test_bf16_storage_long():
    """BF16 state with long constraints (k = 100 and 300): arithmetic at the
    dequantised point within 1e-5."""
    for k in (100, 300):
        inst = synth.single_type(synth.CARD, k, 2, k + 9, index=k, op=synth.GE, param=k // 2)
        x = synth.uniform_x0(inst.n, 24, k)
        x_deq = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
        _check_eval(inst, x_deq, x_dtype=torch.bfloat16, x_ref=x_deq)


def test_mixed_short_and_long_in_one_instance():
    inst = synth.long_card_n10000(0, n=2000, n_clauses=3000, n_long=12, kmin=33, kmax=300)
    _check_eval(inst, synth.uniform_x0(inst.n, 41, 3))


def test_duplicate_and_complementary_literals():
    """Repeated variables are independent literals on both sides."""
    b = synth._Builder(6)
    b.add(synth.OR, [1, 1, 2])
    b.add(synth.XOR, [3, -3, 4, 5], parity=0)
    b.add(synth.CARD, [1, -1, 2, 2, 6] * 8, synth.GE, 17)
    _check_eval(b.build(), synth.uniform_x0(6, 33, 1))


def test_bf16_storage_variant():
    inst = synth.mixed_small(7, n=50, m=90, kmax=20)
    x = synth.uniform_x0(inst.n, 64, 3)
    xb = torch.from_numpy(x).to(torch.bfloat16)
    x_deq = xb.to(torch.float32).numpy()
    # arithmetic at the dequantised point
    _check_eval(inst, x_deq, x_dtype=torch.bfloat16, x_ref=x_deq)
    # end to end against the original FP32 point
    _check_eval(inst, x_deq, x_dtype=torch.bfloat16, x_ref=x, tol=2e-2)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 12])
def test_esp_basis_short(k):
    """The paper's elementary-symmetric basis is accurate for short constraints."""
    p = bd.default_params(basis=bd.BASIS_ESP)
    inst = synth.single_type(synth.CARD, k, 7, 2 * k + 3, index=k, op=synth.GE, param=(k + 1) // 2)
    _check_eval(inst, synth.uniform_x0(inst.n, 33, k), params=p, tol=5e-5)


def test_esp_basis_long_runs_and_degrades():
    """Long constraints in the paper's basis: scaled products keep every value
    finite up to k = 100 (no FP32 overflow), while cancellation makes the
    error grow with k, as the paper's floating-point section describes."""
    p = bd.default_params(basis=bd.BASIS_ESP)
    errs = {}
    for k in (40, 100):
        inst = synth.single_type(synth.CARD, k, 2, k + 3, index=k, op=synth.GE, param=k // 2)
        x = synth.uniform_x0(inst.n, 16, k)
        h = bd.load_instance(inst, p)
        fe, g = bd.eval_fe_grad(h, _dev(x))
        fe = fe.cpu().numpy()
        ref, _, _ = O.evaluate(inst, x.astype(np.float64))
        errs[k] = np.nanmax(np.abs(fe - ref))
        if k == 40:
            assert np.all(np.isfinite(fe))
    assert errs[100] > errs[40]


# ---- exact check ------------------------------------------------------------
@pytest.mark.parametrize("idx", range(3))
def test_unsat_counts_bit_exact(idx):
    inst = synth.mixed_small(idx + 10, n=40, m=150, kmax=40)
    for B, x in ((50, synth.uniform_x0(inst.n, 50, idx)), (33, synth.vertex_x0(inst.n, 33, idx))):
        x = x.copy()
        x[0, :5] = 0.0
        x[1, :5] = -0.0
        h = bd.load_instance(inst)
        bd.init_restarts(h, B, x0=_dev(x))
        un, best, asg, sol = bd.round_and_verify(h)
        ref = O.unsat_count(inst, x)
        np.testing.assert_array_equal(un[0], ref)
        assert best[0] == int(np.argmin(ref))
        np.testing.assert_array_equal(asg, O.round_signs(x[:, best[0]]))
        assert sol[0] == int(ref.min() == 0)


def test_philox_starting_points_bit_exact():
    inst = synth.random_3sat_n50(3)
    h = bd.load_instance(inst)
    bd.init_restarts(h, 37, seed=0x1234_5678_9ABC)
    x = bd.get_x(h).cpu().numpy()
    np.testing.assert_array_equal(x, O.philox_uniform_x0(0x1234_5678_9ABC, inst.n, 37))


def test_batch_starting_points_and_counts_per_instance():
    insts = [synth.random_3sat_n50(i) for i in range(3)] + [synth.mixed_small(5, n=30, m=40, kmax=9)]
    h = bd.load_batch(insts)
    B = 24
    bd.init_restarts(h, B, seed=99)
    x = bd.get_x(h).cpu().numpy()
    un, best, asg, sol = bd.round_and_verify(h)
    v0 = 0
    for i, inst in enumerate(insts):
        xi = x[v0:v0 + inst.n]
        np.testing.assert_array_equal(xi, O.philox_uniform_x0(99, inst.n, B, stream=i))
        np.testing.assert_array_equal(un[i], O.unsat_count(inst, xi))
        v0 += inst.n


# ---- descent steps ---------------------------------------------------------
@pytest.mark.parametrize("graph", [0, 1])
def test_few_steps_match_oracle(graph):
    inst = synth.mixed_small(21, n=50, m=100, kmax=24)
    x0 = synth.uniform_x0(inst.n, 40, 8)
    eta = 0.05
    p = bd.default_params(eta=eta, use_graph=graph, autotune=1)
    h = bd.load_instance(inst, p)
    bd.init_restarts(h, 40, x0=_dev(x0))
    x = x0.astype(np.float64)
    for t in range(3):
        bd.step(h, 1)
        x = O.pgd_step(inst, x, eta)
        got = bd.get_x(h).cpu().numpy()
        assert np.abs(got - x).max() <= 4 * TOL * (t + 1), np.abs(got - x).max()
        un, _ = bd.get_verify(h)
        np.testing.assert_array_equal(un.cpu().numpy()[0], O.unsat_count(inst, got))


def test_chunked_step_equals_single_chunk():
    """Restart chunks only change the launch shape, not the arithmetic."""
    inst = synth.hybrid_n2000(1)
    x0 = synth.uniform_x0(inst.n, 200, 4)
    outs = []
    for chunk in (32, 96, 256):
        p = bd.default_params(eta=0.1, chunk=chunk, autotune=0)
        h = bd.load_instance(inst, p)
        bd.init_restarts(h, 200, x0=_dev(x0))
        bd.step(h, 2)
        outs.append(bd.get_x(h).cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_fixed_tiles_match_autotuned_and_oracle():
    """Every tile shape a caller may fix computes the same step: x after two
    steps agrees across shapes and with the oracle, and the unsat counts of
    each are the oracle's for its own state."""
    inst = synth.hybrid_n2000(1)
    B = 256
    x0 = synth.uniform_x0(inst.n, B, 5)
    ks = sorted(set(int(k) for k in inst.lengths))
    ref = O.pgd_step(inst, O.pgd_step(inst, x0.astype(np.float64), 0.1), 0.1)
    outs = []
    for chunk, rpl, cpw in ((0, None, None), (64, 1, 1), (256, 4, 8), (128, 2, 3)):
        h = bd.load_instance(inst, bd.default_params(eta=0.1, autotune=0 if rpl else 1))
        bd.init_restarts(h, B, x0=_dev(x0))
        if rpl:
            tiles = {k: (min(rpl, 4 if k <= 8 else 2 if k <= 16 else 1), cpw) for k in ks if k <= 32}
            bd.set_tiles(h, chunk, tiles)
            c, got = bd.tiles(h)
            assert c == chunk and got == tiles
        bd.step(h, 2)
        x = bd.get_x(h).cpu().numpy()
        un, _ = bd.get_verify(h)
        np.testing.assert_array_equal(un.cpu().numpy()[0], O.unsat_count(inst, x))
        assert np.abs(x - ref).max() <= 0.1 * 4 * TOL
        outs.append(x)
        h.free()
    for x in outs[1:]:
        assert np.abs(x - outs[0]).max() <= 1e-6


def test_set_tiles_rejects_bad_shapes():
    inst = synth.hybrid_n2000(1)
    h = bd.load_instance(inst, bd.default_params(autotune=0))
    with pytest.raises(RuntimeError):
        bd.set_tiles(h, 64, {3: (1, 1)})            # before init_restarts
    bd.init_restarts(h, 64, seed=1)
    before = bd.tiles(h)
    with pytest.raises(RuntimeError):
        bd.set_tiles(h, 0, {20: (2, 1)})            # k=20 allows one restart per lane
    with pytest.raises(RuntimeError):
        bd.set_tiles(h, 0, {3: (3, 1)})             # not a power of two
    with pytest.raises(RuntimeError):
        bd.set_tiles(h, 0, {3: (1, 65)})
    assert bd.tiles(h) == before


def test_config2_full_size_sampled():
    """The hybrid n=2000 instance at B=1024 in the launch configuration of the
    benchmark (autotuned tiles and chunk, graph replay): one step checked on
    sampled restarts against the oracle, unsat counts for every restart."""
    inst = synth.hybrid_n2000(0)
    B = 1024
    eta = 0.1
    x0 = synth.uniform_x0(inst.n, B, 11)
    h = bd.load_instance(inst, bd.default_params(eta=eta))
    bd.init_restarts(h, B, x0=_dev(x0))
    bd.step(h, 1)
    x1 = bd.get_x(h).cpu().numpy()
    un, _ = bd.get_verify(h)
    np.testing.assert_array_equal(un.cpu().numpy()[0], O.unsat_count(inst, x1))
    cols = np.array([0, 1, 31, 32, 255, 256, 511, 777, 1000, 1023])
    ref = O.pgd_step(inst, x0[:, cols].astype(np.float64), eta)
    assert np.abs(x1[:, cols] - ref).max() <= eta * 2 * TOL
    fe, g = bd.eval_fe_grad(h, _dev(x0[:, cols]))
    fe_ref, go_ref, g_ref = O.evaluate(inst, x0[:, cols].astype(np.float64))
    assert np.abs(fe.cpu().numpy() - fe_ref).max() <= TOL
    assert (np.abs(g.cpu().numpy() - g_ref) / _grad_scale(inst, go_ref)).max() <= TOL


def _check_step_columns(inst, x0, x1, cols, eta, tol=TOL):
    """x1 = one step from x0, checked on the sampled restarts `cols` against
    the oracle: the update within eta * tol of the variable's gradient scale,
    and the exact unsat counts of the new state."""
    _, go_ref, g_ref = O.evaluate(inst, x0[:, cols].astype(np.float64))
    ref = np.clip(x0[:, cols].astype(np.float64) - eta * g_ref, -1.0, 1.0)
    bound = eta * tol * _grad_scale(inst, go_ref) + 1e-6
    assert np.all(np.abs(x1[:, cols] - ref) <= bound)


def test_config3_full_size_sampled():
    """The long-constraint instance (n = 10000, 30000 3-OR + 500 CARD/EK of
    length 64..512) at B = 4096 in the launch configuration of the benchmark:
    one step checked on sampled restarts, and the exact counts of the new
    state on them."""
    inst = synth.long_card_n10000(0)
    B, eta = 4096, 0.1
    x0 = synth.uniform_x0(inst.n, B, 12)
    h = bd.load_instance(inst, bd.default_params(eta=eta))
    bd.init_restarts(h, B, x0=_dev(x0))
    bd.step(h, 1)
    x1 = bd.get_x(h).cpu().numpy()
    un, _ = bd.get_verify(h)
    h.free()
    cols = np.array([0, 1, 31, 32, 1000, 2047, 2048, 4095])
    _check_step_columns(inst, x0, x1, cols, eta)   # lengths up to 512: the 1e-5 bar
    np.testing.assert_array_equal(un.cpu().numpy()[0][cols], O.unsat_count(inst, x1[:, cols]))


def test_config4_full_size_sampled():
    """The uneven batch (256 instances, n log-uniform in 100..20000, B = 64 each)
    in one handle as the benchmark loads it: one step, checked for the
    smallest, a middle and the largest instance on every restart (counts) and
    on sampled restarts (update)."""
    insts = synth.instance_batch(256)
    B, eta = 64, 0.1
    h = bd.load_batch(insts, bd.default_params(eta=eta))
    bd.init_restarts(h, B, seed=21)
    x0 = bd.get_x(h).cpu().numpy()
    bd.step(h, 1)
    x1 = bd.get_x(h).cpu().numpy()
    un, _ = bd.get_verify(h)
    un = un.cpu().numpy()
    h.free()
    offs = np.concatenate([[0], np.cumsum([i.n for i in insts])])
    sizes = np.array([i.n for i in insts])
    order = np.argsort(sizes)
    cols = np.array([0, 1, 31, 32, 63])
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        inst = insts[i]
        a, b = offs[i], offs[i + 1]
        np.testing.assert_array_equal(un[i], O.unsat_count(inst, x1[a:b]), err_msg=f"instance {i}")
        _check_step_columns(inst, x0[a:b], x1[a:b], cols, eta)


# ---- solver behaviour and edge cases ---------------------------------------
def test_never_reports_sat_on_unsat_instances():
    seen = {True: 0, False: 0}
    for idx in range(10):
        inst = synth.random_ksat(14, 70, 3, synth.rng_for(300, idx))
        sat, _ = O.exhaustive_sat(inst)
        seen[sat] += 1
        h = bd.load_instance(inst, bd.default_params(eta=0.2))
        bd.init_restarts(h, 64, seed=idx)
        bd.step(h, 100)
        _, flag = bd.get_verify(h)
        un, best, asg, sol = bd.round_and_verify(h)
        if not sat:
            assert sol[0] == 0 and un.min() > 0
            assert int(flag.cpu()[0]) == 2 ** 31 - 1  # "no solved restart" is INT32_MAX
        if sol[0]:
            assert O.unsat_count(inst, asg.astype(np.float32)[:, None])[0] == 0
    assert seen[True] > 0 and seen[False] > 0


def test_solved_restarts_are_frozen():
    inst = synth.random_ksat(20, 60, 3, synth.rng_for(301, 0))
    h = bd.load_instance(inst, bd.default_params(eta=0.2))
    bd.init_restarts(h, 32, seed=5)
    bd.step(h, 200)
    un, sol = bd.get_verify(h)
    x_a = bd.get_x(h).cpu().numpy()
    bd.step(h, 20)
    x_b = bd.get_x(h).cpu().numpy()
    solved = un.cpu().numpy()[0] == 0
    assert solved.any()
    np.testing.assert_array_equal(x_a[:, solved], x_b[:, solved])
    assert sol.cpu().numpy()[0] == int(np.nonzero(solved)[0][0])


def test_single_restart_and_single_literal():
    b = synth._Builder(3)
    b.add(synth.OR, [1])
    b.add(synth.CARD, [-2], synth.LT, 1)
    b.add(synth.XOR, [3], parity=0)
    inst = b.build()
    _check_eval(inst, synth.uniform_x0(3, 1, 0))


def test_empty_constraint_set():
    b = synth._Builder(4)
    inst = b.build()
    h = bd.load_instance(inst)
    bd.init_restarts(h, 8, seed=1)
    x0 = bd.get_x(h).cpu().numpy()
    bd.step(h, 3)
    np.testing.assert_array_equal(bd.get_x(h).cpu().numpy(), x0)
    un, best, asg, sol = bd.round_and_verify(h)
    assert sol[0] == 1 and un.max() == 0


def test_step_before_init_is_an_error():
    h = bd.load_instance(synth.random_3sat_n50(0))
    with pytest.raises(bd.AfsError) as ei:
        bd.step(h, 1)
    assert ei.value.code == -8


@pytest.mark.parametrize("B,xs", [(64, bd.X_F32), (50, bd.X_F32), (50, bd.X_BF16)])
def test_step_host_matches_device_step(B, xs):
    """The whole-state host-buffer step (FP32 copies straight into the state's
    rows, 2D when the row pitch exceeds B; BF16 through a stage) equals the
    device step."""
    inst = synth.random_3sat_n50(2)
    x0 = synth.uniform_x0(inst.n, B, 9)
    p = bd.default_params(eta=0.1, x_storage=xs)
    h1 = bd.load_instance(inst, p)
    bd.init_restarts(h1, B, x0=_dev(x0))
    bd.step(h1, 1)
    x_dev = bd.get_x(h1).cpu().numpy()
    un_dev, _ = bd.get_verify(h1)
    h2 = bd.load_instance(inst, p)
    bd.init_restarts(h2, B, seed=0)
    xh = torch.from_numpy(x0).pin_memory()
    xo = torch.empty_like(xh).pin_memory()
    un = bd.step_host(h2, xh, xo)
    np.testing.assert_array_equal(xo.numpy(), x_dev)
    np.testing.assert_array_equal(un.numpy(), un_dev.cpu().numpy())


@pytest.mark.parametrize("case", ["f32_1024", "f32_840", "bf16_1024"])
def test_pipelined_step_host_matches_device_steps(case):
    """States of 32 MB and more take afs_step_host in restart chunks whose
    host copies overlap the other chunks' kernels (4 chunks of 256 restarts;
    a ragged last chunk at B = 840; BF16 storage), here on short and long
    constraints together. Two chained host-buffer steps must give the device
    steps' states and exact counts bit for bit, and leave the handle's check
    and count consistent."""
    inst = synth.long_card_n10000(1, n=10000, n_clauses=20000, n_long=24, kmin=40, kmax=160)
    B = 840 if case.endswith("840") else 1024
    xs = bd.X_BF16 if case.startswith("bf16") else bd.X_F32
    assert inst.n * B * 4 >= 32 << 20
    x0 = synth.uniform_x0(inst.n, B, 31)
    p = bd.default_params(eta=0.1, x_storage=xs)
    h1 = bd.load_instance(inst, p)
    bd.init_restarts(h1, B, x0=_dev(x0))
    h2 = bd.load_instance(inst, p)
    bd.init_restarts(h2, B, seed=0)
    xh = torch.from_numpy(x0).pin_memory()
    xo = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        bd.step(h1, 1)
        x_dev = bd.get_x(h1).cpu().numpy()
        un_dev, sol_dev = bd.get_verify(h1)
        un = bd.step_host(h2, xh, xo)
        np.testing.assert_array_equal(xo.numpy(), x_dev)
        np.testing.assert_array_equal(un.numpy(), un_dev.cpu().numpy())
        un2, sol2 = bd.get_verify(h2)
        np.testing.assert_array_equal(un2.cpu().numpy(), un_dev.cpu().numpy())
        np.testing.assert_array_equal(sol2.cpu().numpy(), sol_dev.cpu().numpy())
        np.testing.assert_array_equal(bd.get_step_check(h2).cpu().numpy(), bd.get_step_check(h1).cpu().numpy())
        xh.copy_(xo)
    h1.free()
    h2.free()


# ---- 3-literal constraints: derivatives recomputed in the gather --------------
def test_fused_gradient_without_fe_values():
    """Gradient-only evaluation (no FE kernel for the k = 3 bucket) equals the
    oracle and the gradient of the full evaluation."""
    inst = synth.mixed_small(2, n=30, m=80, kmax=5)
    x = synth.uniform_x0(inst.n, 70, 21)
    h = bd.load_instance(inst)
    _, g_only = bd.eval_fe_grad(h, _dev(x), want_fe=False)
    fe, g_full = bd.eval_fe_grad(h, _dev(x))
    fe_ref, go_ref, g_ref = O.evaluate(inst, x.astype(np.float64))
    assert torch.equal(g_only, g_full)
    assert (np.abs(g_only.cpu().numpy() - g_ref) / _grad_scale(inst, go_ref)).max() <= TOL
    assert np.abs(fe.cpu().numpy() - fe_ref).max() <= TOL


@pytest.mark.parametrize("k", [1, 2, 3])
def test_fused_lengths_with_repeated_variables(k):
    """Short lengths around the fused one (k = 1, 2 through the FE kernels, k = 3
    fused), with repeated and complementary literals, through the step and evaluation paths."""
    b = synth._Builder(6)
    rng = np.random.default_rng(k)
    for _ in range(40):
        lits = rng.integers(1, 7, size=k) * np.where(rng.random(k) < 0.5, -1, 1)
        b.add(int(rng.integers(0, 7)) if k > 1 else synth.OR, lits, synth.GE, int(rng.integers(0, k + 1)),
              int(rng.integers(0, 2)))
    inst = b.build()
    x0 = synth.uniform_x0(inst.n, 40, 30 + k)
    _check_eval(inst, x0)
    h = bd.load_instance(inst, bd.default_params(eta=0.1, verify_every=0, autotune=0))
    bd.init_restarts(h, 40, x0=_dev(x0))
    bd.step(h, 1)
    ref = O.pgd_step(inst, x0.astype(np.float64), 0.1)
    assert np.abs(bd.get_x(h).cpu().numpy() - ref).max() <= 0.1 * 2 * TOL


@pytest.mark.parametrize("B", [64, 256, 1024])
def test_fused_and_unfused_steps_agree(monkeypatch, B):
    """The same steps with the k = 3 derivatives recomputed in the fused pass
    and with them written as occurrence rows by the FE kernel (at chunks that
    take the prefetching and the plain fused sums); the fused steps also
    follow the FP64 oracle's projected steps."""
    inst = synth.hybrid_n2000(1)
    x0 = synth.uniform_x0(inst.n, B, 17)
    outs = []
    for fuse in ("1", "0"):
        monkeypatch.setenv("AFS_FUSE", fuse)
        h = bd.load_instance(inst, bd.default_params(eta=0.1, autotune=0))
        bd.init_restarts(h, B, x0=_dev(x0))
        bd.step(h, 3)
        outs.append(bd.get_x(h).cpu().numpy())
        h.free()
    assert np.abs(outs[0] - outs[1]).max() <= 1e-5
    x = x0[:, :8].astype(np.float64)
    for _ in range(3):
        x = O.pgd_step(inst, x, 0.1)
    assert np.abs(outs[0][:, :8] - x).max() <= 1e-4


def test_parsed_hybrid_file_end_to_end():
    """An instance read from the hybrid format runs through the library: FE,
    gradient and the exact check agree with the oracle."""
    from paper_2606_06641_gb300 import dimacs
    text = "\n".join([
        "p cnf 12 9",
        "h 1 -2 3 0", "x 2 4 -5 6 0", "nae 1 7 8 0", "amo -3 9 10 0", "e 4 11 12 0",
        "ek 2 1 5 9 12 0", "card >=3 2 3 6 7 8 0", "card <=1 10 11 -12 0", "d -2 1 4 8 0",
    ])
    inst = dimacs.parse(text).inst
    x = synth.uniform_x0(inst.n, 64, 77)
    _check_eval(inst, x)
    h = bd.load_instance(inst, bd.default_params(eta=0.1, autotune=0))
    bd.init_restarts(h, 64, x0=_dev(x))
    bd.step(h, 20)
    un, best, asg, sol = bd.round_and_verify(h)
    np.testing.assert_array_equal(un[0], O.unsat_count(inst, bd.get_x(h).cpu().numpy()))


# ---- partial assignments ------------------------------------------------------
def test_fixed_variables_hold_and_the_rest_follow_the_oracle():
    """A fixed variable sits at -1 (True) / +1 (False) from the moment it is
    fixed and is never moved; the free variables take the oracle's projected
    step of the state with the fixed values in place."""
    inst = synth.hybrid_n2000(3)
    B = 96
    rng = np.random.default_rng(4)
    fix = np.zeros(inst.n, np.int8)
    idx = rng.choice(inst.n, size=300, replace=False)
    fix[idx] = np.where(rng.random(300) < 0.5, 1, -1)
    x0 = synth.uniform_x0(inst.n, B, 8)
    h = bd.load_instance(inst, bd.default_params(eta=0.1, verify_every=0, autotune=0))
    bd.init_restarts(h, B, x0=_dev(x0))
    bd.set_fixed(h, fix)
    xf = bd.get_x(h).cpu().numpy()
    want = x0.copy()
    want[fix != 0] = np.where(fix[fix != 0] > 0, -1.0, 1.0)[:, None]
    np.testing.assert_array_equal(xf, want)
    bd.step(h, 1)
    x1 = bd.get_x(h).cpu().numpy()
    ref = O.pgd_step(inst, want.astype(np.float64), 0.1)
    free = fix == 0
    assert np.abs(x1[free] - ref[free]).max() <= 0.1 * 2 * TOL
    np.testing.assert_array_equal(x1[~free], want[~free])
    bd.step(h, 5)
    np.testing.assert_array_equal(bd.get_x(h).cpu().numpy()[~free], want[~free])


def test_fixed_assignments_per_restart_group_and_clearing():
    inst = synth.mixed_small(5)
    B = 64
    fix = np.zeros((2, inst.n), np.int8)
    fix[0, :5] = 1
    fix[1, 5:10] = -1
    h = bd.load_instance(inst, bd.default_params(eta=0.1, autotune=0))
    bd.init_restarts(h, B, seed=9)
    bd.set_fixed(h, fix)
    bd.step(h, 3)
    x = bd.get_x(h).cpu().numpy()
    assert np.all(x[:5, :32] == -1.0) and np.all(x[5:10, 32:] == 1.0)
    bd.init_restarts(h, B, seed=10)      # the assignments survive a re-initialisation
    x = bd.get_x(h).cpu().numpy()
    assert np.all(x[:5, :32] == -1.0) and np.all(x[5:10, 32:] == 1.0)
    bd.set_fixed(h, None)
    bd.step(h, 1)
    assert np.any(bd.get_x(h).cpu().numpy()[:5, :32] != -1.0)


def test_reader_units_as_partial_assignment():
    from paper_2606_06641_gb300 import dimacs
    text = "\n".join(["p cnf 8 6", "1 0", "e -2 0", "ek 3 3 4 5 0", "h 6 7 8 0", "x 1 6 8 0",
                      "card <=1 2 6 7 0"])
    p = dimacs.parse(text)
    assert p.units == {1: True, 2: False, 3: True, 4: True, 5: True}
    h = bd.load_instance(p.inst, bd.default_params(eta=0.1, autotune=0))
    bd.init_restarts(h, 32, seed=2)
    bd.set_fixed(h, p.units)
    bd.step(h, 50)
    un, best, asg, sol = bd.round_and_verify(h)
    assert sol[0] == 1
    for v, val in p.units.items():
        assert asg[v - 1] == (-1 if val else 1)   # the sign of x: -1 = True


# ---- line search ---------------------------------------------------------------
@pytest.mark.parametrize("which", ["mixed", "long"])
def test_line_search_step_matches_the_oracle(which):
    """One Armijo step: the trial each restart takes is the oracle's (except
    where the sufficient-decrease test is within FP32 noise of its bound), and
    the new state equals the oracle's for those restarts. "long" adds
    constraints of length 100..300 (both long-table layouts), whose FE values
    enter the objective the trials are judged by."""
    if which == "mixed":
        inst = synth.mixed_small(4)
    else:
        inst = synth.long_card_n10000(0, n=400, n_clauses=600, n_long=6, kmin=100, kmax=300)
    B = 40
    x0 = synth.uniform_x0(inst.n, B, 4)
    # (a stricter decrease constant makes the long instance backtrack too)
    s, beta, c, T = 30.0, 0.5, (1e-4 if which == "mixed" else 0.5), 8
    ref, ref_chosen = O.armijo_step(inst, x0.astype(np.float64), s, beta, c, T)
    h = bd.load_instance(inst, bd.default_params(autotune=0))
    bd.init_restarts(h, B, x0=_dev(x0))
    chosen = bd.step_ls(h, 1, s, beta, c, T).cpu().numpy()[0]
    x1 = bd.get_x(h).cpu().numpy()
    # the margin of each trial's test, from the oracle
    _, _, g = O.evaluate(inst, x0.astype(np.float64))
    f0 = O.objective(inst, x0.astype(np.float64))
    close = np.zeros(B, bool)
    for i in range(T):
        xi = np.clip(x0 - s * beta ** i * g, -1, 1)
        margin = O.objective(inst, xi) - (f0 + c * (g * (xi - x0)).sum(axis=0))
        close |= np.abs(margin) < 1e-4 * np.maximum(1.0, np.abs(f0))
    same = chosen == ref_chosen
    assert np.all(same | close)
    assert same.sum() >= B - 2
    assert np.abs(x1[:, same] - ref[:, same]).max() <= 1e-4
    assert np.any(ref_chosen > 0)
    un, _ = bd.get_verify(h)
    np.testing.assert_array_equal(un.cpu().numpy()[0], O.unsat_count(inst, x1))


def test_line_search_then_fixed_steps_with_partial_assignment():
    inst = synth.hybrid_n2000(2)
    B = 64
    fix = np.zeros(inst.n, np.int8)
    fix[:50] = 1
    h = bd.load_instance(inst, bd.default_params(eta=0.1, autotune=0))
    bd.init_restarts(h, B, seed=5)
    bd.set_fixed(h, fix)
    f_before = O.objective(inst, bd.get_x(h).cpu().numpy().astype(np.float64))
    chosen = bd.step_ls(h, 3, 1.0, 0.5, 1e-4, 6).cpu().numpy()
    x = bd.get_x(h).cpu().numpy()
    assert np.all(x[:50] == -1.0)
    assert np.all(O.objective(inst, x.astype(np.float64))[chosen[0] >= 0] <= f_before[chosen[0] >= 0] + 1e-3)
    bd.step(h, 2)   # the checked fixed-step path runs on after the line-search steps
    x2 = bd.get_x(h).cpu().numpy()
    un, _ = bd.get_verify(h)
    np.testing.assert_array_equal(un.cpu().numpy()[0], O.unsat_count(inst, x2))
    assert np.all(x2[:50] == -1.0)


def test_line_search_graph_replay_equals_direct_launches():
    """The captured line-search graph (replayed across calls and parities)
    gives bit-identical states, trial choices and counts to direct launches."""
    inst = synth.hybrid_n2000(3)
    B = 96
    x0 = synth.uniform_x0(inst.n, B, 8)
    out = {}
    for use_graph in (0, 1):
        h = bd.load_instance(inst, bd.default_params(eta=0.1, autotune=0, use_graph=use_graph))
        bd.init_restarts(h, B, x0=_dev(x0))
        ch = []
        # per (nsteps, start parity): direct launches, then capture, then replays
        for _ in range(6):
            ch.append(bd.step_ls(h, 1, 2.0, 0.5, 1e-3, 5).cpu().numpy())
        for _ in range(3):
            ch.append(bd.step_ls(h, 2, 2.0, 0.5, 1e-3, 5).cpu().numpy())
        un, _ = bd.get_verify(h)
        out[use_graph] = (bd.get_x(h).cpu().numpy(), np.stack(ch), un.cpu().numpy())
        h.free()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])
    np.testing.assert_array_equal(out[1][2][0], O.unsat_count(inst, out[1][0]))
