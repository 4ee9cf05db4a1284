"""Failure detection without a GPU fault.

The long-constraint kernel's wait for its bulk copies is bounded; when it runs
out the kernel records AFS_E_TIMEOUT in the handle's device status word and
returns. The test hook makes the kernel expect 16 bytes that no copy delivers
(a completion that nothing signals) with a ~10 ms limit; the host must read
the status, and the context must stay usable for the next correct call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def test_bounded_wait_times_out_and_context_survives():
    inst = synth.single_type(synth.CARD, 40, 2, 50, op=synth.GE, param=20)
    h = bd.load_instance(inst)
    x = torch.from_numpy(synth.uniform_x0(inst.n, 8, 1)).cuda()
    fe_ref, g_ref = bd.eval_fe_grad(h, x)
    assert bd.device_error(h) == 0
    bd.debug_wait_timeout(h, True)
    bd.eval_fe_grad(h, x)
    torch.cuda.synchronize()
    assert bd.device_error(h) == -6  # AFS_E_TIMEOUT
    bd.debug_wait_timeout(h, False)
    fe, g = bd.eval_fe_grad(h, x)
    assert bd.device_error(h) == 0
    assert torch.equal(fe, fe_ref) and torch.equal(g, g_ref)


def test_timeout_is_reported_once_then_cleared():
    inst = synth.single_type(synth.EK, 50, 3, 60, param=25)
    h = bd.load_instance(inst)
    x = torch.from_numpy(synth.uniform_x0(inst.n, 16, 2)).cuda()
    fe_ref, g_ref = bd.eval_fe_grad(h, x)
    bd.debug_wait_timeout(h, True)
    bd.eval_fe_grad(h, x)
    assert bd.device_error(h) == -6          # AFS_E_TIMEOUT read by the host
    assert bd.device_error(h) == 0           # the word was cleared
    bd.debug_wait_timeout(h, False)
    fe, g = bd.eval_fe_grad(h, x)
    assert bd.device_error(h) == 0
    assert torch.equal(fe, fe_ref) and torch.equal(g, g_ref)
    # the descent and the exact check still work on this context
    bd.init_restarts(h, 16, seed=3)
    bd.step(h, 5)
    un, best, asg, sol = bd.round_and_verify(h)
    assert un.shape == (1, 16)
