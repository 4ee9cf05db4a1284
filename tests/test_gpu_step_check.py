"""The exact check inside the step (Algorithm 1's is_sat at the sign-rounded
state), read back per restart with get_step_check and compared with the
oracle's unsat counts element by element.

States are built so that satisfied and violated restarts both occur: for one
constraint per instance every true count t = 0..k appears; for multi-constraint
instances the constraints are drawn around a planted assignment, some
restarts sit exactly on it and the others have a few variables flipped.
Zeros of both signs are planted (a variable at +0 or -0 rounds to False).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fe_oracle as O
from paper_2606_06641_gb300 import binding as bd
from paper_2606_06641_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06641_gb300 import build
    build.build()
    yield


def _values(true_var, rng):
    """x for a 0/1 'variable is True' array: True -> negative, False -> +-0 or positive."""
    mag = rng.uniform(0.05, 1.0, size=true_var.shape).astype(np.float32)
    x = np.where(true_var, -mag, mag).astype(np.float32)
    z = (~true_var) & (rng.random(true_var.shape) < 0.15)
    x[z] = np.where(rng.random(int(z.sum())) < 0.5, np.float32(0.0), np.float32(-0.0))
    return x


def _single_constraint_case(ctype, k, B, rng, op=synth.GE, param=0, parity=1):
    """One constraint over all k variables; restart b has t = b mod (k+1) true literals."""
    b = synth._Builder(k)
    lits = (rng.permutation(k) + 1) * np.where(rng.random(k) < 0.5, -1, 1)
    b.add(ctype, lits, op, param, parity)
    inst = b.build()
    true_lit = np.zeros((k, B), bool)
    for col in range(B):
        t = col % (k + 1)
        true_lit[rng.permutation(k)[:t], col] = True
    # literal i on variable v: true iff (v True) xor negated
    var = np.abs(lits) - 1
    neg = (lits < 0)[:, None]
    true_var = np.zeros((k, B), bool)
    true_var[var] = true_lit ^ neg
    return inst, _values(true_var, rng)


def _planted_case(n, m, kmax, B, rng):
    """Constraints of every type that all hold at a planted assignment sigma."""
    sigma = rng.random(n) < 0.5
    b = synth._Builder(n)
    for _ in range(m):
        ctype = int(rng.integers(0, 7))
        k = int(rng.integers(2, kmax + 1))
        var = rng.choice(n, size=k, replace=False)
        if ctype == synth.OR:
            t = int(rng.integers(1, k + 1))
        elif ctype == synth.NAE:
            t = int(rng.integers(1, k))
        elif ctype == synth.AMO:
            t = int(rng.integers(0, 2))
        elif ctype == synth.EO:
            t = 1
        else:
            t = int(rng.integers(0, k + 1))
        want = np.zeros(k, bool)
        want[rng.permutation(k)[:t]] = True
        # literal true iff sigma_v xor negated  ->  negated = sigma_v xor want
        negated = sigma[var] ^ want
        lits = (var + 1) * np.where(negated, -1, 1)
        if ctype == synth.XOR:
            b.add(ctype, lits, synth.GE, 0, t % 2)
        elif ctype == synth.EK:
            b.add(ctype, lits, synth.GE, t)
        elif ctype == synth.CARD:
            if rng.random() < 0.5:
                b.add(ctype, lits, synth.GE, int(rng.integers(0, t + 1)))
            else:
                b.add(ctype, lits, synth.LT, int(rng.integers(t + 1, k + 2)))
        else:
            b.add(ctype, lits)
    inst = b.build()
    true_var = np.repeat(sigma[:, None], B, axis=1)
    for col in range(B):
        if col % 3:
            flips = rng.choice(n, size=int(rng.integers(1, 4)), replace=False)
            true_var[flips, col] ^= True
    return inst, _values(true_var, rng)


def _run_check(insts, xs, B):
    h = bd.load_batch(insts, bd.default_params(eta=0.0, verify_every=1, autotune=0))
    x0 = np.concatenate(xs, axis=0)
    bd.init_restarts(h, B, x0=torch.from_numpy(x0).cuda())
    bd.step(h, 1)
    got = bd.get_step_check(h).cpu().numpy()
    un, _ = bd.get_verify(h)
    un = un.cpu().numpy()
    h.free()
    for i, (inst, x) in enumerate(zip(insts, xs)):
        ref = O.unsat_count(inst, x)
        np.testing.assert_array_equal(got[i], ref == 0, err_msg=f"instance {i}")
        np.testing.assert_array_equal(un[i], ref, err_msg=f"instance {i} (final check)")
    return got


@pytest.mark.parametrize("ctype,kw", [
    (synth.OR, {}), (synth.XOR, {"parity": 1}), (synth.XOR, {"parity": 0}), (synth.NAE, {}),
    (synth.AMO, {}), (synth.EO, {}), (synth.EK, {"param": -1}), (synth.CARD, {"op": synth.GE, "param": -1}),
    (synth.CARD, {"op": synth.LT, "param": -1}),
])
def test_every_count_of_every_length(ctype, kw):
    """All counts t = 0..k for k across the short, 62/63/64 boundary and staged long sizes."""
    rng = np.random.default_rng(100 + ctype)
    B = 200
    insts, xs = [], []
    for k in (1, 2, 3, 5, 20, 31, 32, 33, 61, 62, 63, 64, 65, 100, 129, 197):
        args = dict(kw)
        if args.get("param") == -1:
            args["param"] = int(rng.integers(0, k + 1))
        inst, x = _single_constraint_case(ctype, k, B, rng, **args)
        insts.append(inst)
        xs.append(x)
    got = _run_check(insts, xs, B)
    assert got.any() and not got.all()


@pytest.mark.parametrize("B", [200, 300])
@pytest.mark.parametrize("ctype,kw", [
    (synth.OR, {}), (synth.XOR, {"parity": 1}), (synth.NAE, {}), (synth.EO, {}), (synth.EK, {"param": -1}),
    (synth.CARD, {"op": synth.GE, "param": -1}), (synth.CARD, {"op": synth.LT, "param": -1}),
])
def test_every_count_up_to_62_literals(ctype, kw, B):
    """All counts t = 0..k for k <= 62, where the checks of up to 8 restart
    words (B = 200) take one constraint per lane and wider ones (B = 300) one
    word per lane: both must give the oracle's counts."""
    rng = np.random.default_rng(300 + ctype + B)
    insts, xs = [], []
    for k in (1, 2, 3, 5, 20, 31, 32, 33, 61, 62):
        args = dict(kw)
        if args.get("param") == -1:
            args["param"] = int(rng.integers(0, k + 1))
        inst, x = _single_constraint_case(ctype, k, B, rng, **args)
        insts.append(inst)
        xs.append(x)
    got = _run_check(insts, xs, B)
    assert got.any() and not got.all()


@pytest.mark.parametrize("B", [32, 64, 250])
def test_planted_runs_of_long_short_constraints(B):
    """Runs of many constraints up to 62 literals (several runs of up to 31
    constraints and 256 literals per instance) in the lane-per-constraint check."""
    rng = np.random.default_rng(40 + B)
    insts, xs = [], []
    for i in range(4):
        inst, x = _planted_case(int(rng.integers(70, 120)), int(rng.integers(60, 140)), 62, B, rng)
        insts.append(inst)
        xs.append(x)
    got = _run_check(insts, xs, B)
    assert got[:, 0].all()


def test_longest_constraint_all_counts():
    rng = np.random.default_rng(7)
    B = 1100
    insts, xs = [], []
    for ctype, args in ((synth.CARD, {"op": synth.GE, "param": 300}), (synth.EK, {"param": 500}),
                        (synth.XOR, {"parity": 1})):
        inst, x = _single_constraint_case(ctype, 512, B, rng, **args)
        insts.append(inst)
        xs.append(x)
    _run_check(insts, xs, B)


@pytest.mark.parametrize("B", [1, 31, 33, 100, 256])
def test_planted_mixed_instances(B):
    """Multi-constraint ranges, several instances per launch, ragged restart counts."""
    rng = np.random.default_rng(B)
    insts, xs = [], []
    for i in range(5):
        inst, x = _planted_case(int(rng.integers(20, 90)), int(rng.integers(5, 120)), 12, B, rng)
        insts.append(inst)
        xs.append(x)
    got = _run_check(insts, xs, B)
    assert got[:, 0].all()  # restart 0 sits on the planted assignment


def test_planted_hybrid_size_instance():
    """A hybrid-workload-sized planted instance (8000+ constraints, one instance) at B=1024."""
    rng = np.random.default_rng(11)
    inst, x = _planted_case(2000, 8700, 20, 1024, rng)
    _run_check([inst], [x], 1024)


def test_frozen_restarts_match_the_check():
    """With eta > 0 exactly the restarts the check marked satisfied keep their state."""
    rng = np.random.default_rng(5)
    B = 96
    inst, x = _planted_case(60, 150, 8, B, rng)
    h = bd.load_instance(inst, bd.default_params(eta=0.1, verify_every=1, autotune=0))
    bd.init_restarts(h, B, x0=torch.from_numpy(x).cuda())
    bd.step(h, 1)
    solved = bd.get_step_check(h).cpu().numpy()[0]
    x1 = bd.get_x(h).cpu().numpy()
    np.testing.assert_array_equal(solved, O.unsat_count(inst, x) == 0)
    assert np.array_equal(x1[:, solved], x[:, solved])
    moved = np.any(x1 != x, axis=0)
    assert moved[~solved].all()


def test_check_of_each_step_across_calls_and_chunks():
    """Several calls of one step each (alternating parities), with and without
    graphs and with restart chunks: every step's check is the oracle's
    verdict on the state that step read."""
    rng = np.random.default_rng(9)
    B = 160
    inst, x = _planted_case(80, 200, 10, B, rng)
    for use_graph, chunk in ((1, 0), (0, 64), (1, 96)):
        p = bd.default_params(eta=0.05, verify_every=1, autotune=0, use_graph=use_graph, chunk=chunk)
        h = bd.load_instance(inst, p)
        bd.init_restarts(h, B, x0=torch.from_numpy(x).cuda())
        for _ in range(4):
            before = bd.get_x(h).cpu().numpy()
            bd.step(h, 1)
            got = bd.get_step_check(h).cpu().numpy()[0]
            np.testing.assert_array_equal(got, O.unsat_count(inst, before) == 0)
        h.free()


def test_step_check_unavailable_after_unchecked_step():
    inst = synth.mixed_small(0)
    h = bd.load_instance(inst, bd.default_params(verify_every=0, autotune=0))
    bd.init_restarts(h, 32, seed=1)
    bd.step(h, 1)
    with pytest.raises(RuntimeError):
        bd.get_step_check(h)


def test_count_follows_every_state_write():
    """get_verify counts the current state: right after init_restarts, after
    steps, after set_x and after set_fixed, and a repeated call agrees."""
    rng = np.random.default_rng(13)
    B = 64
    inst, x = _planted_case(70, 180, 9, B, rng)
    h = bd.load_instance(inst, bd.default_params(eta=0.07, verify_every=1, autotune=0))
    bd.init_restarts(h, B, x0=torch.from_numpy(x).cuda())

    def agree():
        un, _ = bd.get_verify(h)
        un2, _ = bd.get_verify(h)
        ref = O.unsat_count(inst, bd.get_x(h).cpu().numpy())
        np.testing.assert_array_equal(un.cpu().numpy()[0], ref)
        np.testing.assert_array_equal(un2.cpu().numpy()[0], ref)

    agree()
    bd.step(h, 3)
    agree()
    x2 = np.where(rng.random(x.shape) < 0.5, -x, x).astype(np.float32)
    bd.set_x(h, torch.from_numpy(x2).cuda())
    agree()
    fix = np.zeros((1, inst.n), np.int8)
    fix[0, :10] = 1
    bd.set_fixed(h, fix)
    agree()
    bd.step(h, 2)
    agree()
    h.free()
