"""Pins of the learned initialiser's FP64 reference (CPU only)."""
import numpy as np

from oracle import mpnn_oracle as M
from paper_2606_06641_gb300 import synth


def _setup(H=8, L=2, seed=0):
    inst = synth.mixed_small(3, n=12, m=20, kmax=5)
    n_par = sum(int(np.prod(s)) for _, s in M.param_shapes(H, L))
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.4, n_par)
    y = rng.uniform(0, 1, inst.n)
    w = (rng.random(inst.n) < 0.8).astype(np.float64)
    return inst, theta, y, w


def test_gradient_matches_central_differences():
    H, L = 8, 2
    inst, theta, y, w = _setup(H, L)
    loss, g, _ = M.loss_and_grad(inst, theta, y, w, H, L)
    rng = np.random.default_rng(1)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss_and_grad(inst, tp, y, w, H, L)[0] - M.loss_and_grad(inst, tm, y, w, H, L)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_is_bce_of_tanh_output():
    inst, theta, y, w = _setup()
    mu, cache = M.forward(inst, theta, 8, 2)
    p = (1 - mu) / 2
    ref = -np.sum(w * (y * np.log(p) + (1 - y) * np.log(1 - p))) / w.sum()
    loss, _ = M.loss_and_dz(cache["z"], y, w)
    assert abs(loss - ref) < 1e-10


def test_message_means_respect_signs():
    """A single clause (x1 or -x2): the constraint message is the mean of
    s_e P[v_e] over its two literals."""
    b = synth._Builder(2)
    b.add(synth.OR, [1, -2])
    inst = b.build()
    cons, var, sgn = M.edges(inst)
    assert list(var) == [0, 1] and list(sgn) == [1.0, -1.0] and list(cons) == [0, 0]
    fv, fc = M.features(inst)
    np.testing.assert_allclose(fv[:, 1], [1.0, -1.0])
    assert fc[0, 0] == 1.0 and fc[0, 7] == 2 / 8


def test_bf16_rounding_is_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-3])
    r = M.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                     # halfway, ties to even
    assert r[2] == 1.0 + 2 ** -6           # halfway, ties to even (up)
    assert r[3] == -2.5
    assert abs(r[4] - 3.0e-3) <= 3.0e-3 * 2 ** -8


def test_adam_first_step_is_sign_times_lr():
    th = np.zeros(3)
    g = np.array([0.5, -2.0, 1e-3])
    new, m, v = M.adam_step(th, g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(new, -0.01 * np.sign(g), rtol=1e-4)


def test_gradient_criteria_detect_planted_errors():
    """The element-wise criteria the GPU test applies accept the bfloat16-operand
    reference against the plain FP64 one (the FP64 criterion) and reject a
    gradient with one large entry's sign flipped or a weight gradient
    transposed (both planted in the oracle's own gradient)."""
    from mpnn_criteria import BF16_REF, FP64_REF, grad_mismatches
    H, L = 64, 3
    inst = synth.concat_instances([synth.random_3sat_n50(i) for i in range(2)])
    shapes = M.param_shapes(H, L)
    n_par = sum(int(np.prod(s)) for _, s in shapes)
    rng = np.random.default_rng(3)
    theta = np.concatenate([rng.uniform(-1, 1, int(np.prod(s))) * np.sqrt(3.0 / (s[-1] if len(s) > 1 else H))
                            for _, s in shapes])
    assert theta.size == n_par
    y = rng.uniform(0, 1, inst.n)
    w = (rng.random(inst.n) < 0.7).astype(np.float64)
    _, g_bf, _ = M.loss_and_grad(inst, theta, y, w, H, L, bf16=True)
    _, g64, _ = M.loss_and_grad(inst, theta, y, w, H, L, bf16=False)
    assert grad_mismatches(g_bf, g_bf, shapes, **BF16_REF) == []
    assert grad_mismatches(g_bf, g64, shapes, **FP64_REF) == []
    at = 0
    for name, shp in shapes:
        size = int(np.prod(shp))
        seg = g_bf[at:at + size]
        if np.abs(seg).max() > 0:
            bad = g_bf.copy()
            i = at + int(np.argmax(np.abs(seg)))
            bad[i] = -bad[i]
            assert name in grad_mismatches(bad, g_bf, shapes, **BF16_REF), name
            if len(shp) == 2 and shp[0] == shp[1]:
                bad = g_bf.copy()
                bad[at:at + size] = seg.reshape(shp).T.ravel()
                assert name in grad_mismatches(bad, g_bf, shapes, **BF16_REF), name
        at += size
