"""What the trained initialiser gains over uniform starts (small scale).

Labels come from the descent's own solutions on training instances of the
n=50, m=213 random 3-SAT distribution; held-out instances are solved from
learned and from uniform starts with the same restarts and step budget.
The network must fit better than an untrained one on held-out labels, and
learned starts (with a quarter of the restarts kept uniform) must not lose
solves; the measured solve rates and step counts are printed.
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
    eta, steps = 0.1, 500
    train = [synth.learned_split(i, "train") for i in range(1500)]
    test = [synth.learned_split(i, "test") for i in range(160)]
    lab_tr = learned.harvest(train, 64, eta, steps, seed=1)
    lab_te = learned.harvest(test, 64, eta, steps, seed=2)
    assert len(lab_tr.insts) > 200 and len(lab_te.insts) > 20
    tr_b = learned.make_batches(lab_tr, 64)
    te_b = learned.make_batches(lab_te, 64)
    untrained = bd.Mpnn(layers=3, seed=7)
    net = bd.Mpnn(layers=3, seed=7)
    loss0 = _held_out_loss(untrained, te_b)
    hist = learned.train(net, tr_b, 25, 3e-3)
    loss1 = _held_out_loss(net, te_b)
    assert hist[-1] < hist[0]
    assert loss1 < loss0, (loss0, loss1)
    s_u, st_u, _, _ = learned.evaluate(None, test, 64, eta, steps, seed=3)
    s_l, st_l, _, _ = learned.evaluate(net, test, 64, eta, steps, seed=3)
    both = s_u & s_l
    print(f"\nheld-out BCE untrained {loss0:.4f} trained {loss1:.4f}; solve rate uniform {s_u.mean():.3f} "
          f"learned {s_l.mean():.3f}; median steps uniform {np.median(st_u[s_u]) if s_u.any() else None} "
          f"learned {np.median(st_l[s_l]) if s_l.any() else None}; paired step gain on both-solved "
          f"{np.median(st_u[both] - st_l[both]) if both.any() else None}")
    assert s_l.sum() >= 0.8 * s_u.sum()
