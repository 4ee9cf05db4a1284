"""The evaluation entry point that allocates no device memory.

afs_eval_fe_grad_noalloc is for callers that cannot call cudaMalloc when they
evaluate (cudaMalloc and cudaFree synchronise the device and take a
driver-wide lock, or all device memory is reserved by another allocator). It
keeps its scratch in a fixed 16 MiB array inside the library instead of a
buffer it allocates. Its results must match afs_eval_fe_grad, the entry point
that allocates its own buffer, on consecutive calls that reuse the shared
array; instances too large for the array must be rejected with a clear error.
This file is collected last so that a stop at the first failure has already
run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2606_06641_gb300 import binding as bd
from paper_2606_06641_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the FE / gradient tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_06641_gb300 import build
    build.build()
    yield


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float32)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    inst = synth.hybrid_n2000(3)  # 30400 occurrences: several column chunks of the array
    h = bd.load_instance(inst)
    for call, (B, seed) in enumerate(((300, 1), (77, 2))):
        x = _dev(synth.uniform_x0(inst.n, B, seed))
        fe_ref, g_ref = bd.eval_fe_grad(h, x)
        fe = torch.full((inst.m, B), float("nan"), device="cuda")
        g = torch.full((inst.n, B), float("nan"), device="cuda")
        bd.eval_fe_grad_noalloc(h, x, fe, g)
        torch.cuda.synchronize()
        fe_err = (fe - fe_ref).abs().max().item()
        g_err = (g - g_ref).abs().max().item()
        assert fe_err <= TOL and g_err <= TOL, (call, fe_err, g_err)


def test_noalloc_mixed_long_constraints():
    inst = synth.long_card_n10000(1, n=1500, n_clauses=2000, n_long=6, kmin=40, kmax=300)
    h = bd.load_instance(inst)
    x = _dev(synth.near_vertex_x0(inst.n, 45, 4))
    fe_ref, g_ref = bd.eval_fe_grad(h, x)
    fe = torch.empty((inst.m, 45), device="cuda")
    g = torch.empty((inst.n, 45), device="cuda")
    for _ in range(2):
        bd.eval_fe_grad_noalloc(h, x, fe, g)
        torch.cuda.synchronize()
        assert (fe - fe_ref).abs().max().item() <= TOL
        assert (g - g_ref).abs().max().item() <= TOL


def test_noalloc_rejects_instances_beyond_the_array():
    # 180000 occurrences of 6-clauses (each with a derivative row) x 32
    # restarts x 4 bytes > 16 MiB
    inst = synth.random_ksat(20000, 30000, 6, synth.rng_for(400, 0))
    assert inst.n_lits > 131072
    h = bd.load_instance(inst)
    x = _dev(synth.uniform_x0(inst.n, 32, 0))
    g = torch.empty((inst.n, 32), device="cuda")
    with pytest.raises(bd.AfsError) as ei:
        bd.eval_fe_grad_noalloc(h, x, None, g)
    assert ei.value.code == -1 and "scratch" in str(ei.value)


def test_noalloc_takes_large_instances_of_short_constraints():
    """160000 occurrences of 3-clauses need no derivative rows (the gather
    recomputes them), so the fixed array is not a limit for them; results
    equal the allocating entry point's."""
    inst = synth.random_ksat(20000, 53334, 3, synth.rng_for(400, 1))
    assert inst.n_lits > 131072
    h = bd.load_instance(inst)
    x = _dev(synth.uniform_x0(inst.n, 64, 3))
    fe_ref, g_ref = bd.eval_fe_grad(h, x)
    fe = torch.empty_like(fe_ref)
    g = torch.empty_like(g_ref)
    bd.eval_fe_grad_noalloc(h, x, fe, g)
    torch.cuda.synchronize()
    assert torch.equal(fe, fe_ref) and torch.equal(g, g_ref)


def test_noalloc_shrinks_chunks_to_the_array():
    """40000 occurrences of 4-clauses (each with a derivative row): a chunk of
    256 restarts would need 40 MB, so the entry point shrinks its chunks to 96
    restarts (96 x 40000 x 4 bytes fits 16 MiB) and walks B = 300 restarts in
    four chunks (96, 96, 96, 12); results equal the allocating entry point's."""
    inst = synth.random_ksat(5000, 10000, 4, synth.rng_for(400, 2))
    assert 16384 < inst.n_lits <= 131072
    h = bd.load_instance(inst)
    B = 300
    for call, seed in enumerate((5, 6)):
        x = _dev(synth.uniform_x0(inst.n, B, seed))
        fe_ref, g_ref = bd.eval_fe_grad(h, x)
        fe = torch.full((inst.m, B), float("nan"), device="cuda")
        g = torch.full((inst.n, B), float("nan"), device="cuda")
        bd.eval_fe_grad_noalloc(h, x, fe, g)
        torch.cuda.synchronize()
        fe_err = (fe - fe_ref).abs().max().item()
        g_err = (g - g_ref).abs().max().item()
        assert fe_err <= TOL and g_err <= TOL, (call, fe_err, g_err)
