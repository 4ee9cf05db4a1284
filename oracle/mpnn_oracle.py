"""FP64 reference of the learned initialiser's message-passing network.

TEST INFRASTRUCTURE ONLY (imported by tests/ and never by the product path).
The paper has no learned component; this network is the bipartite
variable-constraint message passing the benchmark plan specifies, written out
plainly so the CUDA forward and backward kernels can be checked against it.
Its own gradient is pinned by central finite differences.

Graph: variables v, constraints c, edges e = literal occurrences (c_e, v_e, s_e)
with s_e = +1 for a positive literal and -1 for a negated one.
Features (also computed by the library from the instance records):
  f_v = [deg_v / 8, (pos_v - neg_v) / max(deg_v, 1), 1, 0]              (4)
  f_c = [onehot(type, 7), k / 8, param / max(k, 1), parity, op, 1, 0...]  (16)
Network (hidden H, L layers):
  h_v = relu(f_v A_v^T + a_v),  h_c = relu(f_c A_c^T + a_c)
  per layer l:
    P = h_v U_l^T;   m_c = mean_{e in c} s_e P[v_e]
    h_c = relu([h_c, m_c] Wc_l^T + bc_l)
    Q = h_c V_l^T;   q_v = mean_{e at v} s_e Q[c_e]   (0 for an isolated v)
    h_v = relu([h_v, q_v] Wv_l^T + bv_l)
  z = h_v w + b;  mu = tanh(z)   (x ~ mu: True when mu < 0)
Loss: p_v = P(v True) = (1 - mu_v)/2 = sigmoid(-2 z_v); mean over labelled
variables of the binary cross-entropy against the soft label y_v.
With ``bf16=True`` every matrix-product operand is rounded to bfloat16
(round to nearest even) before an exact product, as the tensor-core path does.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

FV, FC = 4, 16


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def edges(inst) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    k = np.diff(inst.lit_off)
    cons = np.repeat(np.arange(len(k)), k)
    var = np.abs(inst.lits).astype(np.int64) - 1
    sgn = np.where(inst.lits > 0, 1.0, -1.0)
    return cons, var, sgn


def features(inst) -> Tuple[np.ndarray, np.ndarray]:
    cons, var, sgn = edges(inst)
    n, m = inst.n, len(inst.lit_off) - 1
    deg = np.bincount(var, minlength=n).astype(np.float64)
    bal = np.bincount(var, weights=sgn, minlength=n)
    fv = np.zeros((n, FV))
    fv[:, 0] = deg / 8.0
    fv[:, 1] = bal / np.maximum(deg, 1.0)
    fv[:, 2] = 1.0
    k = np.diff(inst.lit_off).astype(np.float64)
    fc = np.zeros((m, FC))
    fc[np.arange(m), inst.ctype.astype(np.int64)] = 1.0
    fc[:, 7] = k / 8.0
    fc[:, 8] = np.where(np.isin(inst.ctype, (5, 6)), inst.param, 0) / np.maximum(k, 1.0)
    fc[:, 9] = np.where(inst.ctype == 1, inst.parity, 0)
    fc[:, 10] = np.where(inst.ctype == 6, inst.op, 0)
    fc[:, 11] = 1.0
    return fv, fc


def param_shapes(H: int = 64, L: int = 3) -> List[Tuple[str, Tuple[int, ...]]]:
    """Parameter order of the flat vector (shared with the library's layout)."""
    out = [("Av", (H, FV)), ("av", (H,)), ("Ac", (H, FC)), ("ac", (H,))]
    for l in range(L):
        out += [(f"U{l}", (H, H)), (f"V{l}", (H, H)), (f"Wc{l}", (H, 2 * H)), (f"bc{l}", (H,)),
                (f"Wv{l}", (H, 2 * H)), (f"bv{l}", (H,))]
    out += [("w", (H,)), ("b", (1,))]
    return out


def unflatten(theta: np.ndarray, H: int = 64, L: int = 3) -> Dict[str, np.ndarray]:
    out, at = {}, 0
    for name, shp in param_shapes(H, L):
        size = int(np.prod(shp))
        out[name] = np.asarray(theta[at:at + size], dtype=np.float64).reshape(shp)
        at += size
    assert at == theta.size
    return out


def _mm(a, b, bf16):
    if bf16:
        a, b = bf16_round(a), bf16_round(b)
    return a @ b


def forward(inst, theta, H=64, L=3, bf16=False):
    """Returns mu [n] and the cache the backward pass needs."""
    p = unflatten(theta, H, L)
    cons, var, sgn = edges(inst)
    n, m = inst.n, len(inst.lit_off) - 1
    k = np.bincount(cons, minlength=m).astype(np.float64)
    deg = np.bincount(var, minlength=n).astype(np.float64)
    fv, fc = features(inst)
    hv = np.maximum(_mm(fv, p["Av"].T, bf16) + p["av"], 0.0)
    hc = np.maximum(_mm(fc, p["Ac"].T, bf16) + p["ac"], 0.0)
    cache = {"fv": fv, "fc": fc, "hv0": hv, "hc0": hc, "layers": [], "k": k, "deg": deg}
    for l in range(L):
        P = _mm(hv, p[f"U{l}"].T, bf16)
        mc = np.zeros((m, H))
        np.add.at(mc, cons, sgn[:, None] * P[var])
        mc /= np.maximum(k, 1.0)[:, None]
        Xc = np.concatenate([hc, mc], axis=1)
        hc_new = np.maximum(_mm(Xc, p[f"Wc{l}"].T, bf16) + p[f"bc{l}"], 0.0)
        Q = _mm(hc_new, p[f"V{l}"].T, bf16)
        qv = np.zeros((n, H))
        np.add.at(qv, var, sgn[:, None] * Q[cons])
        qv /= np.maximum(deg, 1.0)[:, None]
        Xv = np.concatenate([hv, qv], axis=1)
        hv_new = np.maximum(_mm(Xv, p[f"Wv{l}"].T, bf16) + p[f"bv{l}"], 0.0)
        cache["layers"].append({"hv_in": hv, "Xc": Xc, "hc": hc_new, "Xv": Xv, "hv": hv_new})
        hv, hc = hv_new, hc_new
    z = hv @ p["w"] + p["b"][0]
    cache["hv_out"] = hv
    cache["z"] = z
    return np.tanh(z), cache


def loss_and_dz(z, y, wmask):
    """Mean masked BCE of p = sigmoid(-2 z) against y, and dloss/dz."""
    t = -2.0 * z
    wsum = max(float(wmask.sum()), 1.0)
    sp = np.maximum(t, 0.0) + np.log1p(np.exp(-np.abs(t)))
    loss = float(np.sum(wmask * (sp - y * t)) / wsum)
    sig = 1.0 / (1.0 + np.exp(-t))
    dz = wmask * (-2.0) * (sig - y) / wsum
    return loss, dz


def backward(inst, theta, cache, dz, H=64, L=3, bf16=False):
    """Gradient of the loss with respect to the flat parameter vector."""
    p = unflatten(theta, H, L)
    cons, var, sgn = edges(inst)
    n, m = inst.n, len(inst.lit_off) - 1
    k, deg = cache["k"], cache["deg"]
    g = {name: np.zeros(shp) for name, shp in param_shapes(H, L)}
    hv = cache["hv_out"]
    g["w"] = hv.T @ dz
    g["b"] = np.array([dz.sum()])
    dhv = np.outer(dz, p["w"])
    dhc = np.zeros((m, H))
    for l in reversed(range(L)):
        c = cache["layers"][l]
        dpre = dhv * (c["hv"] > 0)
        g[f"Wv{l}"] = _mm(dpre.T, c["Xv"], bf16)
        g[f"bv{l}"] = dpre.sum(axis=0)
        dXv = _mm(dpre, p[f"Wv{l}"], bf16)
        dhv_in = dXv[:, :H]
        dqv = dXv[:, H:] / np.maximum(deg, 1.0)[:, None]
        dQ = np.zeros((m, H))
        np.add.at(dQ, cons, sgn[:, None] * dqv[var])
        g[f"V{l}"] = _mm(dQ.T, c["hc"], bf16)
        dhc = dhc + _mm(dQ, p[f"V{l}"], bf16)
        dpre = dhc * (c["hc"] > 0)
        g[f"Wc{l}"] = _mm(dpre.T, c["Xc"], bf16)
        g[f"bc{l}"] = dpre.sum(axis=0)
        dXc = _mm(dpre, p[f"Wc{l}"], bf16)
        dhc = dXc[:, :H]
        dmc = dXc[:, H:] / np.maximum(k, 1.0)[:, None]
        dP = np.zeros((n, H))
        np.add.at(dP, var, sgn[:, None] * dmc[cons])
        g[f"U{l}"] = _mm(dP.T, c["hv_in"], bf16)
        dhv = dhv_in + _mm(dP, p[f"U{l}"], bf16)
    dpre = dhv * (cache["hv0"] > 0)
    g["Av"] = _mm(dpre.T, cache["fv"], bf16)
    g["av"] = dpre.sum(axis=0)
    dpre = dhc * (cache["hc0"] > 0)
    g["Ac"] = _mm(dpre.T, cache["fc"], bf16)
    g["ac"] = dpre.sum(axis=0)
    return np.concatenate([g[name].ravel() for name, _ in param_shapes(H, L)])


def loss_and_grad(inst, theta, y, wmask, H=64, L=3, bf16=False):
    mu, cache = forward(inst, theta, H, L, bf16)
    loss, dz = loss_and_dz(cache["z"], y, wmask)
    return loss, backward(inst, theta, cache, dz, H, L, bf16), mu


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma & Ba, 2015) with bias correction; t counts from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
