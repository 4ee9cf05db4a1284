"""What the trained initialiser gains over uniform starts.

The learned-initialiser configuration at full size: 10000 training instances
of the n=50, m=213 random 3-SAT distribution labelled with the distinct
solutions the descent itself finds, 512 held-out instances, B=256 restarts,
500 steps. Held-out instances are solved from uniform starts and from the same
uniform starts nudged toward the network's proposal (x = clamp(u + alpha_b mu),
alpha ramped from 0 to 0.5 over the restarts). The learned starts must solve
at least as many held-out instances and take fewer steps on the instances both
forms solve; the network must also fit the held-out labels better than an
untrained one. Every reported solution is re-checked exactly by the solver.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06641_gb300 import binding as bd
from paper_2606_06641_gb300 import learned, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06641_gb300 import build
    build.build()
    yield


def _held_out_loss(net, batches):
    return float(np.mean([net.loss_grad(h, y)[0] for h, y in batches]))


def test_learned_starts_gain_over_uniform():
    eta, steps, B = 0.1, 500, 256
    train = [synth.learned_split(i, "train") for i in range(10000)]
    test = [synth.learned_split(i, "test") for i in range(512)]
    lab_tr = learned.harvest(train, 64, eta, steps, seed=1)
    lab_te = learned.harvest(test, 64, eta, steps, seed=2)
    assert len(lab_tr.insts) > 2000 and len(lab_te.insts) > 100
    tr_b = learned.make_batches(lab_tr, 64)
    te_b = learned.make_batches(lab_te, 64)
    untrained = bd.Mpnn(layers=3, seed=7)
    net = bd.Mpnn(layers=3, seed=7)
    loss0 = _held_out_loss(untrained, te_b)
    hist = learned.train(net, tr_b, 30, 3e-3)
    loss1 = _held_out_loss(net, te_b)
    assert hist[-1] < hist[0] and loss1 < loss0, (hist[0], hist[-1], loss0, loss1)
    s_u, st_u, _, _ = learned.evaluate(None, test, B, eta, steps, seed=3)
    s_l, st_l, _, _ = learned.evaluate(net, test, B, eta, steps, seed=3, start=learned.DEFAULT_START)
    both = s_u & s_l
    gain = st_u[both] - st_l[both]
    print(f"\nheld-out BCE untrained {loss0:.4f} trained {loss1:.4f}; solved uniform {int(s_u.sum())} "
          f"learned {int(s_l.sum())} of {len(test)}; median steps uniform {np.median(st_u[s_u])} learned "
          f"{np.median(st_l[s_l])}; paired step gain median {np.median(gain)} mean {gain.mean():.2f}")
    assert s_l.sum() >= s_u.sum()
    assert np.median(gain) > 0 and gain.mean() > 0
