"""The persistent step mode: S steps of Algorithm 1 in one cooperative launch.

For handles whose constraints are all short, afs_step can run its steps as one
persistent launch (phases separated by a grid barrier) instead of the per-step
launches of the length buckets, the check and the CSR pass. Every unit does
the same arithmetic in the same order as the per-launch kernels, so the two
modes must produce bit-identical trajectories, step checks and solved flags;
the trajectories also follow the FP64 oracle's projected steps.
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


def _run(insts, B, persistent, steps, x0=None, fixed=None, **params):
    p = bd.default_params(eta=0.1, persistent=persistent, **params)
    h = bd.load_instance(insts[0], p) if len(insts) == 1 else bd.load_batch(insts, p)
    bd.init_restarts(h, B, seed=5, x0=x0)
    if fixed is not None:
        bd.set_fixed(h, fixed)
    mode, blocks = bd.step_mode(h)
    xs = []
    for s in steps:
        bd.step(h, s)
        xs.append(bd.get_x(h).cpu().numpy())
    un, sol = bd.get_verify(h)
    chk = bd.get_step_check(h).cpu().numpy() if params.get("verify_every", 1) else None
    out = (mode, blocks, xs, un.cpu().numpy(), sol.cpu().numpy(), chk)
    h.free()
    return out


@pytest.mark.parametrize("B", [32, 64, 200])
def test_persistent_matches_per_launch_steps_bit_for_bit(B):
    inst = synth.hybrid_n2000(1)   # buckets of length 3 (fused), 4, 5 and 20
    on = _run([inst], B, 1, (1, 7, 10))
    off = _run([inst], B, -1, (1, 7, 10))
    assert on[0] and on[1] > 0 and not off[0]
    for a, b in zip(on[2], off[2]):
        assert np.array_equal(a, b)
    assert np.array_equal(on[3], off[3]) and np.array_equal(on[4], off[4]) and np.array_equal(on[5], off[5])


def test_persistent_follows_the_oracle():
    inst = synth.mixed_small(3, n=60, m=150, kmax=20)
    B = 40
    x0 = synth.uniform_x0(inst.n, B, 2)
    mode, _, xs, _, _, _ = _run([inst], B, 1, (3,), x0=torch.from_numpy(x0).cuda())
    assert mode
    x = x0.astype(np.float64)
    for _ in range(3):
        x = O.pgd_step(inst, x, 0.1)
    assert np.abs(xs[0] - x).max() <= 1e-4


def test_persistent_batch_bf16_and_fixed_variables():
    insts = [synth.random_3sat_n50(i) for i in range(6)] + [synth.mixed_small(1, n=40, m=70, kmax=12)]
    n = sum(i.n for i in insts)
    fixed = np.zeros((2, n), np.int8)
    fixed[0, 3] = 1
    fixed[1, 10] = -1
    for xs in (bd.X_F32, bd.X_BF16):
        on = _run(insts, 96, 1, (4, 9), fixed=fixed, x_storage=xs)
        off = _run(insts, 96, -1, (4, 9), fixed=fixed, x_storage=xs)
        assert on[0]
        for a, b in zip(on[2], off[2]):
            assert np.array_equal(a, b)
        assert np.array_equal(on[3], off[3]) and np.array_equal(on[4], off[4])
        assert np.all(on[2][-1][3, :48] == -1.0) and np.all(on[2][-1][10, 48:] == 1.0)


def test_persistent_without_the_per_step_check():
    inst = synth.random_3sat_n50(4)
    on = _run([inst], 64, 1, (12,), verify_every=0)
    off = _run([inst], 64, -1, (12,), verify_every=0)
    assert on[0] and np.array_equal(on[2][0], off[2][0]) and np.array_equal(on[3], off[3])


def test_persistent_solves_and_flags_like_per_launch():
    insts = [synth.random_3sat_n50(i) for i in range(32)]
    on = _run(insts, 32, 1, (60,))
    off = _run(insts, 32, -1, (60,))
    assert on[0]
    assert np.array_equal(on[4], off[4]) and (on[4] != 2 ** 31 - 1).any()
    assert np.array_equal(on[2][0], off[2][0])


def test_long_constraints_keep_per_launch_steps():
    inst = synth.long_card_n10000(0, n=800, n_clauses=500, n_long=3, kmin=40, kmax=80)
    on = _run([inst], 32, 1, (2,))
    assert not on[0]
