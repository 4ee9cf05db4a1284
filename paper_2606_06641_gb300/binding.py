"""Thin Python binding of the C ABI in include/afsat.h (argument marshalling only).

Every computation runs in libafsat's CUDA kernels; this module converts
instances to ``afs_cons`` records, passes torch tensors' device pointers and
the current CUDA stream, and turns status codes into exceptions. There is no
CPU fallback: if the library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from .synth import Instance

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libafsat.so")

AFS_OK = 0
ERRORS = {-1: "AFS_E_ARG", -2: "AFS_E_VAR_RANGE", -3: "AFS_E_LEN", -4: "AFS_E_TYPE", -5: "AFS_E_CUDA",
          -6: "AFS_E_TIMEOUT", -7: "AFS_E_VERIFY", -8: "AFS_E_STATE"}
BASIS_PGF, BASIS_ESP = 0, 1
X_F32, X_BF16 = 0, 1
MAX_LEN = 512

CONS_DTYPE = np.dtype([("type", "u1"), ("op", "u1"), ("parity", "u1"), ("reserved", "u1"),
                       ("param", "<i4"), ("lit_offset", "<i4"), ("len", "<i4")])

# Every symbol declared in include/afsat.h, with (restype, argtypes).
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
SIGNATURES = {
    "afs_default_params": (None, [_P]),
    "afs_load_instance": (_I32, [_P, _I32, _P, _I64, _I32, _P, _P, _P]),
    "afs_load_batch": (_I32, [_P, _P, _P, _P, _I64, _P, _I32, _P, _P, _P]),
    "afs_free": (None, [_P]),
    "afs_init_restarts": (_I32, [_P, _I32, ctypes.c_uint64, _P, _P]),
    "afs_step": (_I32, [_P, _I32, _P]),
    "afs_round_and_verify": (_I32, [_P, _P, _P, _P, _P, _P]),
    "afs_get_x": (_I32, [_P, _P, _P]),
    "afs_set_x": (_I32, [_P, _P, _P]),
    "afs_get_verify": (_I32, [_P, _P, _P, _P]),
    "afs_eval_fe_grad": (_I32, [_P, _P, _I32, _I32, _P, _P, _P]),
    "afs_eval_fe_grad_noalloc": (_I32, [_P, _P, _I32, _P, _P, _P]),
    "afs_step_host": (_I32, [_P, _P, _P, _P, _P]),
    "afs_mpnn_create": (_I32, [_I32, _I32, ctypes.c_uint64, _P]),
    "afs_mpnn_free": (None, [_P]),
    "afs_mpnn_num_params": (_I32, [_P, _P]),
    "afs_mpnn_get_params": (_I32, [_P, _P, _P]),
    "afs_mpnn_set_params": (_I32, [_P, _P, _P]),
    "afs_mpnn_forward": (_I32, [_P, _P, _P, _P]),
    "afs_mpnn_loss_grad": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "afs_mpnn_adam_step": (_I32, [_P, ctypes.c_float, _P]),
    "afs_mpnn_nudge_restarts": (_I32, [_P, _P, ctypes.c_float, ctypes.c_float, _P]),
    "afs_mpnn_init_restarts": (_I32, [_P, _P, _I32, ctypes.c_uint64, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, _P]),
    "afs_device_error": (_I32, [_P, _P, _P]),
    "afs_debug_wait_timeout": (_I32, [_P, _I32]),
    "afs_info": (_I32, [_P, _P]),
    "afs_work_per_restart": (_I32, [_P, _P]),
    "afs_set_kernel_timing": (_I32, [_P, _I32]),
    "afs_kernel_timing": (_I32, [_P, _P, _P, _P, _P]),
    "afs_last_launch_count": (_I32, [_P, _P]),
    "afs_tuning": (_I32, [_P, _P, _P, _I32]),
    "afs_tiles": (_I32, [_P, _P, _P, _P, _I32]),
    "afs_get_step_check": (_I32, [_P, _P, _P, _P]),
    "afs_set_fixed": (_I32, [_P, _P, _I32, _P]),
    "afs_step_ls": (_I32, [_P, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I32, _P, _P]),
    "afs_set_tiles": (_I32, [_P, _I32, _P, _P, _I32]),
    "afs_long_tiles": (_I32, [_P, _P, _P, _P, _I32, _P]),
    "afs_group_times": (_I32, [_P, _I32, _P, _P, _P, _P, _I32, _P, _P]),
    "afs_step_mode": (_I32, [_P, _P, _P]),
    "afs_set_long_tiles": (_I32, [_P, _P, _P, _I32]),
    "afs_coef_table": (_I32, [_I32, _I32, _I32, _I32, _I32, _I32, _I32, _P, _I32, _P]),
    "afs_esp_coefficients": (_I32, [_I32, _I32, _I32, _I32, _I32, _P]),
    "afs_last_error": (ctypes.c_char_p, []),
    "afs_version": (ctypes.c_char_p, []),
}


class AfsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_float), ("basis", _I32), ("x_storage", _I32), ("verify_every", _I32),
                ("chunk", _I32), ("autotune", _I32), ("use_graph", _I32), ("persistent", _I32)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libafsat.so from the package tree (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libafsat.so is not built ({LIB_PATH}); run the package build first")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(l, name)
            fn.restype = res
            fn.argtypes = args
        _lib = l
    return _lib


def _check(rc: int) -> None:
    if rc != AFS_OK:
        raise AfsError(rc, lib().afs_last_error().decode())


def default_params(**kw) -> Params:
    p = Params()
    lib().afs_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _stream(stream=None) -> int:
    if isinstance(stream, int):
        return stream
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def cons_records(inst: Instance) -> np.ndarray:
    rec = np.zeros(inst.m, dtype=CONS_DTYPE)
    rec["type"] = inst.ctype
    rec["op"] = inst.op
    rec["parity"] = inst.parity
    rec["param"] = inst.param
    rec["lit_offset"] = inst.lit_off[:-1]
    rec["len"] = np.diff(inst.lit_off)
    return rec


class Handle:
    """One loaded instance (or batch) with its device state."""

    def __init__(self, ptr: int, n: int, m: int, n_inst: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.n, self.m, self.n_inst = n, m, n_inst
        self.B = 0

    def __del__(self):
        try:
            if self.ptr:
                lib().afs_free(self.ptr)
                self.ptr = ctypes.c_void_p(0)
        except Exception:
            pass

    def free(self) -> None:
        if self.ptr:
            lib().afs_free(self.ptr)
            self.ptr = ctypes.c_void_p(0)


def load_instance(inst: Instance, params: Optional[Params] = None, stream=None) -> Handle:
    rec = cons_records(inst)
    lits = np.ascontiguousarray(inst.lits, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(lib().afs_load_instance(rec.ctypes.data, inst.m, lits.ctypes.data, lits.shape[0], inst.n,
                                   ctypes.byref(params) if params is not None else None, _stream(stream),
                                   ctypes.byref(out)))
    return Handle(out.value, inst.n, inst.m, 1)


def load_batch(insts: Sequence[Instance], params: Optional[Params] = None, stream=None) -> Handle:
    count = np.fromiter((i.m for i in insts), np.int32, len(insts))
    nv = np.fromiter((i.n for i in insts), np.int32, len(insts))
    nl = np.fromiter((i.n_lits for i in insts), np.int64, len(insts))
    begin = np.zeros(len(insts), np.int32)
    np.cumsum(count[:-1], out=begin[1:])
    lit_base = np.zeros(len(insts), np.int64)
    np.cumsum(nl[:-1], out=lit_base[1:])
    m = int(count.sum())
    rec = np.zeros(m, dtype=CONS_DTYPE)
    if m:
        rec["type"] = np.concatenate([i.ctype for i in insts])
        rec["op"] = np.concatenate([i.op for i in insts])
        rec["parity"] = np.concatenate([i.parity for i in insts])
        rec["param"] = np.concatenate([i.param for i in insts])
        offs = np.concatenate([i.lit_off for i in insts])      # m + n_inst entries (each instance's m + 1)
        last = np.cumsum(count + 1) - 1                          # the closing offset of each instance
        keep = np.ones(offs.shape[0], bool)
        keep[last] = False
        rec["lit_offset"] = offs[keep] + np.repeat(lit_base, count)
        rec["len"] = offs[1:][keep[:-1]] - offs[:-1][keep[:-1]]
    lit = np.ascontiguousarray(np.concatenate([i.lits for i in insts]).astype(np.int32, copy=False)) \
        if len(insts) else np.zeros(0, np.int32)
    out = ctypes.c_void_p()
    _check(lib().afs_load_batch(rec.ctypes.data, begin.ctypes.data, count.ctypes.data, lit.ctypes.data,
                                lit.shape[0], nv.ctypes.data, len(insts),
                                ctypes.byref(params) if params is not None else None, _stream(stream),
                                ctypes.byref(out)))
    return Handle(out.value, int(nv.sum()), m, len(insts))


def init_restarts(h: Handle, B: int, seed: int = 0, x0=None, stream=None) -> None:
    if x0 is not None:
        assert x0.is_cuda and x0.dtype.itemsize == 4 and x0.is_contiguous() and tuple(x0.shape) == (h.n, B)
    _check(lib().afs_init_restarts(h.ptr, B, seed, _ptr(x0), _stream(stream)))
    h.B = B


def step(h: Handle, nsteps: int, stream=None) -> None:
    _check(lib().afs_step(h.ptr, nsteps, _stream(stream)))


def round_and_verify(h: Handle, stream=None):
    """Returns (unsat[n_inst, B], best[n_inst], assignment[n] (+1/-1), solved[n_inst])."""
    un = np.zeros((h.n_inst, h.B), np.int32)
    best = np.zeros(h.n_inst, np.int32)
    asg = np.zeros(h.n, np.int8)
    sol = np.zeros(h.n_inst, np.int32)
    _check(lib().afs_round_and_verify(h.ptr, un.ctypes.data, best.ctypes.data, asg.ctypes.data, sol.ctypes.data,
                                      _stream(stream)))
    return un, best, asg, sol


def get_x(h: Handle, stream=None):
    import torch
    out = torch.empty((h.n, h.B), dtype=torch.float32, device="cuda")
    _check(lib().afs_get_x(h.ptr, _ptr(out), _stream(stream)))
    return out


def set_x(h: Handle, x, stream=None) -> None:
    assert x.is_cuda and x.dtype.itemsize == 4 and x.is_contiguous() and tuple(x.shape) == (h.n, h.B)
    _check(lib().afs_set_x(h.ptr, _ptr(x), _stream(stream)))


def get_verify(h: Handle, stream=None):
    import torch
    un = torch.empty((h.n_inst, h.B), dtype=torch.int32, device="cuda")
    sol = torch.empty(h.n_inst, dtype=torch.int32, device="cuda")
    _check(lib().afs_get_verify(h.ptr, _ptr(un), _ptr(sol), _stream(stream)))
    return un, sol


def step_ls(h: Handle, nsteps: int, s: float = 1.0, beta: float = 0.5, c: float = 1e-4, trials: int = 6,
            stream=None):
    """nsteps iterations with Armijo backtracking per restart; returns the trial
    each restart took in the last iteration (-1 = none accepted) [n_inst, B]."""
    import torch
    chosen = torch.empty((h.n_inst, h.B), dtype=torch.int32, device="cuda")
    _check(lib().afs_step_ls(h.ptr, int(nsteps), float(s), float(beta), float(c), int(trials), _ptr(chosen),
                             _stream(stream)))
    return chosen


def set_fixed(h: Handle, values=None, stream=None) -> None:
    """Partial assignments: values [n] or [groups, n] int8 (+1 True, -1 False,
    0 free; restart b uses row b * groups // B), or a {variable (1-based): bool}
    dict such as a reader's units; None clears them."""
    if values is None:
        _check(lib().afs_set_fixed(h.ptr, None, 0, _stream(stream)))
        return
    if isinstance(values, dict):
        arr = np.zeros(h.n, np.int8)
        for v, val in values.items():
            arr[int(v) - 1] = 1 if val else -1
        values = arr
    arr = np.ascontiguousarray(np.asarray(values, dtype=np.int8))
    if arr.ndim == 1:
        arr = arr[None, :]
    assert arr.shape[1] == h.n
    _check(lib().afs_set_fixed(h.ptr, arr.ctypes.data, arr.shape[0], _stream(stream)))


def get_step_check(h: Handle, stream=None):
    """Per instance and restart: True where the last step's exact check found
    every constraint satisfied (bool tensor [n_inst, B] on the device)."""
    import torch
    W = ctypes.c_int32()
    _check(lib().afs_get_step_check(h.ptr, None, ctypes.byref(W), _stream(stream)))
    words = torch.empty((h.n_inst, W.value), dtype=torch.int32, device="cuda")
    _check(lib().afs_get_step_check(h.ptr, _ptr(words), None, _stream(stream)))
    shifts = torch.arange(32, device="cuda", dtype=torch.int32)
    bits = (words.unsqueeze(-1) >> shifts) & 1
    return bits.reshape(h.n_inst, -1)[:, :h.B] != 0


def eval_fe_grad(h: Handle, x, want_fe: bool = True, want_grad: bool = True, stream=None):
    """FE per constraint [m, B] and objective gradient [n, B] at x [n, B] (float32 or bfloat16)."""
    import torch
    assert x.is_cuda and x.is_contiguous() and x.shape[0] == h.n
    dt = X_BF16 if x.dtype == torch.bfloat16 else X_F32
    assert dt == X_BF16 or x.dtype == torch.float32
    B = x.shape[1]
    fe = torch.empty((h.m, B), dtype=torch.float32, device=x.device) if want_fe else None
    g = torch.empty((h.n, B), dtype=torch.float32, device=x.device) if want_grad else None
    _check(lib().afs_eval_fe_grad(h.ptr, _ptr(x), dt, B, _ptr(fe), _ptr(g), _stream(stream)))
    return fe, g


def eval_fe_grad_noalloc(h: Handle, x, fe=None, grad=None, stream=None):
    """FE [m, B] and gradient [n, B] at FP32 x [n, B] through the entry point
    that allocates no device memory (its scratch is a fixed array inside the
    library). The caller passes the output buffers (either may be None)."""
    assert x.is_cuda and x.is_contiguous() and x.shape[0] == h.n
    B = x.shape[1]
    for out, rows in ((fe, h.m), (grad, h.n)):
        if out is not None:
            assert out.is_cuda and out.is_contiguous() and tuple(out.shape) == (rows, B)
    _check(lib().afs_eval_fe_grad_noalloc(h.ptr, _ptr(x), B, _ptr(fe), _ptr(grad), _stream(stream)))
    return fe, grad


def step_host(h: Handle, x_host, x_out_host=None, stream=None):
    """One whole step through host memory; returns unsat counts [n_inst, B] (host)."""
    import torch
    assert not x_host.is_cuda and x_host.dtype == torch.float32 and tuple(x_host.shape) == (h.n, h.B)
    un = torch.empty((h.n_inst, h.B), dtype=torch.int32).pin_memory() if not hasattr(h, "_un_pinned") else h._un_pinned
    h._un_pinned = un
    _check(lib().afs_step_host(h.ptr, _ptr(x_host), _ptr(x_out_host), _ptr(un), _stream(stream)))
    return un


class Mpnn:
    """The learned initialiser's network (parameters live on the device)."""

    def __init__(self, layers: int = 3, seed: int = 0, hidden: int = 64):
        out = ctypes.c_void_p()
        _check(lib().afs_mpnn_create(hidden, layers, seed, ctypes.byref(out)))
        self.ptr = out
        n = ctypes.c_int64()
        _check(lib().afs_mpnn_num_params(self.ptr, ctypes.byref(n)))
        self.n_params = n.value
        self.layers = layers

    def __del__(self):
        try:
            if self.ptr:
                lib().afs_mpnn_free(self.ptr)
                self.ptr = ctypes.c_void_p(0)
        except Exception:
            pass

    def get_params(self, stream=None):
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(lib().afs_mpnn_get_params(self.ptr, _ptr(out), _stream(stream)))
        return out

    def set_params(self, theta, stream=None) -> None:
        assert theta.is_cuda and theta.dtype.itemsize == 4 and theta.numel() == self.n_params
        _check(lib().afs_mpnn_set_params(self.ptr, _ptr(theta.contiguous()), _stream(stream)))

    def forward(self, h: Handle, stream=None):
        import torch
        mu = torch.empty(h.n, dtype=torch.float32, device="cuda")
        _check(lib().afs_mpnn_forward(self.ptr, h.ptr, _ptr(mu), _stream(stream)))
        return mu

    def loss_grad(self, h: Handle, y, w=None, want_grad: bool = False, stream=None):
        """Returns (loss, gradient tensor or None); y and w are device tensors [n]."""
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda") if want_grad else None
        loss = ctypes.c_float()
        _check(lib().afs_mpnn_loss_grad(self.ptr, h.ptr, _ptr(y), _ptr(w), _ptr(g), ctypes.byref(loss),
                                        _stream(stream)))
        return loss.value, g

    def adam_step(self, lr: float, stream=None) -> None:
        _check(lib().afs_mpnn_adam_step(self.ptr, lr, _stream(stream)))

    def init_restarts(self, h: Handle, B: int, seed: int = 0, uniform_frac: float = 0.5,
                      sigma_min: float = 0.3, sigma_max: float = 1.5, stream=None) -> None:
        _check(lib().afs_mpnn_init_restarts(self.ptr, h.ptr, B, seed, uniform_frac, sigma_min, sigma_max,
                                            _stream(stream)))

    def nudge_restarts(self, h: Handle, alpha_min: float = 0.0, alpha_max: float = 1.0, stream=None):
        """x = clamp(x + alpha_b mu, -1, 1) on the current state, alpha ramped over the restarts."""
        _check(lib().afs_mpnn_nudge_restarts(self.ptr, h.ptr, alpha_min, alpha_max, _stream(stream)))


def device_error(h: Handle, stream=None) -> int:
    """AFS_OK or AFS_E_TIMEOUT from the handle's device status word (cleared)."""
    code = ctypes.c_int32()
    _check(lib().afs_device_error(h.ptr, ctypes.byref(code), _stream(stream)))
    return code.value


def debug_wait_timeout(h: Handle, enable: bool) -> None:
    _check(lib().afs_debug_wait_timeout(h.ptr, 1 if enable else 0))


def info(h: Handle) -> List[int]:
    out = (ctypes.c_int64 * 6)()
    _check(lib().afs_info(h.ptr, out))
    return list(out)


def work_per_restart(h: Handle) -> float:
    v = ctypes.c_double()
    _check(lib().afs_work_per_restart(h.ptr, ctypes.byref(v)))
    return v.value


def set_kernel_timing(h: Handle, enable: bool) -> None:
    _check(lib().afs_set_kernel_timing(h.ptr, 1 if enable else 0))


def kernel_timing(h: Handle):
    fe, csr = ctypes.c_double(), ctypes.c_double()
    nf, nc = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().afs_kernel_timing(h.ptr, ctypes.byref(fe), ctypes.byref(nf), ctypes.byref(csr), ctypes.byref(nc)))
    return fe.value, nf.value, csr.value, nc.value


def last_launch_count(h: Handle) -> int:
    v = ctypes.c_int64()
    _check(lib().afs_last_launch_count(h.ptr, ctypes.byref(v)))
    return v.value


def tuning(h: Handle):
    chunk = ctypes.c_int32()
    rpl = (ctypes.c_int32 * 33)()
    _check(lib().afs_tuning(h.ptr, ctypes.byref(chunk), rpl, 33))
    return chunk.value, {k: rpl[k] for k in range(33) if rpl[k]}


def tiles(h: Handle):
    """(chunk, {k: (restarts per lane, constraints per warp)}) of the short buckets."""
    chunk = ctypes.c_int32()
    rpl = (ctypes.c_int32 * 33)()
    cpw = (ctypes.c_int32 * 33)()
    _check(lib().afs_tiles(h.ptr, ctypes.byref(chunk), rpl, cpw, 33))
    return chunk.value, {k: (rpl[k], cpw[k]) for k in range(33) if rpl[k]}


def set_tiles(h: Handle, chunk: int = 0, tiles=None):
    """Fix the chunk and per-length (rpl, cpw) tile shapes; 0 keeps a value."""
    rpl = (ctypes.c_int32 * 33)()
    cpw = (ctypes.c_int32 * 33)()
    for k, (r, c) in (tiles or {}).items():
        if not 0 <= int(k) < 33:
            raise ValueError(f"no short bucket for length {k}")
        rpl[int(k)] = int(r)
        cpw[int(k)] = int(c)
    _check(lib().afs_set_tiles(h.ptr, int(chunk), rpl, cpw, 33))


def step_mode(h: Handle):
    """(persistent, blocks): whether afs_step runs as one persistent launch, and its grid."""
    p = ctypes.c_int32()
    bl = ctypes.c_int32()
    _check(lib().afs_step_mode(h.ptr, ctypes.byref(p), ctypes.byref(bl)))
    return bool(p.value), bl.value


def group_times(h: Handle, reps: int = 3, stream=None):
    """[(kind, kmax, ms per launch, algorithmic FP32 instructions per launch)]
    of every FE launch group (kind 0 short, 1 long, 2 fused 3-literal pass)."""
    n = ctypes.c_int32()
    _check(lib().afs_group_times(h.ptr, 1, None, None, None, None, 0, ctypes.byref(n), _stream(stream)))
    cnt = max(1, n.value)
    ms = (ctypes.c_double * cnt)()
    kind = (ctypes.c_int32 * cnt)()
    km = (ctypes.c_int32 * cnt)()
    work = (ctypes.c_double * cnt)()
    _check(lib().afs_group_times(h.ptr, int(reps), ms, kind, km, work, n.value, ctypes.byref(n), _stream(stream)))
    return [(kind[i], km[i], ms[i], work[i]) for i in range(n.value)]


def long_tiles(h: Handle):
    """[(lanes per restart, warps per CTA, longest k)] of the long groups, longest first."""
    n = ctypes.c_int32()
    _check(lib().afs_long_tiles(h.ptr, None, None, None, 0, ctypes.byref(n)))
    lw = (ctypes.c_int32 * max(1, n.value))()
    nw = (ctypes.c_int32 * max(1, n.value))()
    km = (ctypes.c_int32 * max(1, n.value))()
    _check(lib().afs_long_tiles(h.ptr, lw, nw, km, n.value, ctypes.byref(n)))
    return [(lw[i], nw[i], km[i]) for i in range(n.value)]


def set_long_tiles(h: Handle, tiles):
    """Fix the long groups' (lanes, warps) tiles, in long_tiles order; (0, 0) keeps one."""
    n = len(tiles)
    lw = (ctypes.c_int32 * max(1, n))(*[int(t[0]) for t in tiles])
    nw = (ctypes.c_int32 * max(1, n))(*[int(t[1]) for t in tiles])
    _check(lib().afs_set_long_tiles(h.ptr, lw, nw, n))


def parse_tiles(spec: str):
    """'1024:3=4x2,20=1x1' -> (1024, {3: (4, 2), 20: (1, 1)})."""
    chunk_s, _, rest = spec.partition(":")
    tiles = {}
    for item in filter(None, rest.split(",")):
        k, _, shape = item.partition("=")
        r, _, c = shape.partition("x")
        tiles[int(k)] = (int(r), int(c or 0))
    return int(chunk_s or 0), tiles


def format_tiles(chunk: int, tiles) -> str:
    return f"{chunk}:" + ",".join(f"{k}={r}x{c}" for k, (r, c) in sorted(tiles.items()))


def coef_table(ctype: int, k: int, op: int = 0, param: int = 0, parity: int = 1, basis: int = BASIS_PGF,
               form: int = 0) -> np.ndarray:
    n = ctypes.c_int32()
    _check(lib().afs_coef_table(ctype, k, op, param, parity, basis, form, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, np.float32)
    _check(lib().afs_coef_table(ctype, k, op, param, parity, basis, form, out.ctypes.data, n.value, ctypes.byref(n)))
    return out


def esp_coefficients(ctype: int, k: int, op: int = 0, param: int = 0, parity: int = 1) -> np.ndarray:
    out = np.zeros(k + 1, np.float64)
    _check(lib().afs_esp_coefficients(ctype, k, op, param, parity, out.ctypes.data))
    return out


def version() -> str:
    return lib().afs_version().decode()
