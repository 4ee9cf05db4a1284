"""Benchmark of the Fourier-expansion CLS hot path on GB300.

Headline workload (``--workload long``, the default): the long-constraint
instance (n=10000 variables; 30000 random 3-clauses + 500 CARD >= r / EK = r
constraints of length uniform in [64, 512], r uniform in [k/4, 3k/4]),
B=4096 restarts per GPU, FP32 state: the largest single-GPU configuration. A
step is one pass of the whole hot path for all restarts: FE and analytic
gradient of every constraint, the per-step exact check of the state read, the
CSR gather and projected step. Metric: literal-evals/s = literal occurrences x
restarts x steps / s.

The same JSON line carries the other two throughput workloads under
``workloads``: ``hybrid`` (n=2000; 8000 3-clauses, 400 XOR(5), 200 CARD(20)
>= 10, 100 NAE(4); B=1024) and ``batch`` (256 instances, n log-uniform in
[100, 20000], B=64 each, one handle), each with its own timing, roofline,
end-to-end figure and CPU baseline, plus ``time_to_solve`` (random 3-SAT
n=50: plain CLS against the batched form at an equal solve rate).

Timing: W untimed warm-up steps; K timed steps as K/S replays of an S-step
CUDA graph (S = --steps-per-graph), each replay bracketed by CUDA events on
the launching stream, with L2 flushed (a 512 MB write) between replays; a
``sustained`` figure repeats replays until at least --sustained-s seconds of
device time. Under torchrun every rank runs its own restarts (weak scaling,
no collective on the data path); the timed region is bracketed by a barrier
and device syncs and the max over ranks is reported.

Roofline: the dominant kernel of each workload (the kernel with the largest
share of FE+gradient time) is timed per launch with CUDA events on the
launching stream (afs_group_times) and rated at its algorithmic FP32
instructions (16 per (literal, root) plus 2 per root, R(k) = floor((k+1)/2);
3 per occurrence for the fused 3-literal pass) against SMs x 128 FP32 lanes x
the maximum SM clock.

--impl reference times the CPU oracle (FP64 numpy, Poisson-binomial
recurrence) on a bounded sample of the same workload, on all host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import tempfile
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "hybrid": ("hybrid mixed-type instance n=2000: 8000 3-OR, 400 XOR(5, fair parity), 200 CARD(20)>=10, "
               "100 NAE(4); B=1024 restarts per GPU", 1024),
    "long": ("long-constraint instance n=10000: 30000 3-OR + 500 CARD>=r / EK=r of length U[64,512], "
             "r U[k/4,3k/4]; B=4096 restarts per GPU", 4096),
    "batch": ("uneven batch: 256 instances, n log-U[100,20000], m/n U[4.0,4.3], 90% 3-OR, 5% XOR(3..8), "
              "5% CARD(10..100); B=64 restarts each, one handle", 64),
}
METRIC = "FE+grad literal-evals/s"
LINE_SEARCH = (1.0, 0.5, 1e-4, 6)   # first step, backtracking factor, sufficient-decrease constant, trials
UNIT = "literal-evals/s"
# the sources each dominant kernel is built from (its counters are valid while
# their hash is unchanged)
_CS = "paper_2606_06641_gb300/csrc/"
KERNEL_SOURCES = {
    "fe_grad_short_kernel": [_CS + "fe_short.cuh", _CS + "short_dispatch.cuh", _CS + "coef.cpp", _CS + "coef.h",
                             _CS + "afsat_internal.h"],
    "fe_grad_long_pgf_kernel": [_CS + "long_pgf.cu", _CS + "bulk_copy.cuh", _CS + "coef.cpp", _CS + "coef.h",
                                _CS + "afsat_internal.h"],
    "fused_grad_kernel": [_CS + "kernels.cu", _CS + "step_units.cuh", _CS + "fe_short.cuh",
                          _CS + "afsat_internal.h"],
}


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"afsat_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id_for(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else f"GPU-{u}"
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else str(dev)


def make_workload(name: str):
    from paper_2606_06641_gb300 import synth
    if name == "hybrid":
        return [synth.hybrid_n2000(0)]
    if name == "long":
        return [synth.long_card_n10000(0)]
    if name == "batch":
        return synth.instance_batch(256)
    raise ValueError(name)


def _single_thread():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"


def _oracle_worker(task):
    """One host core: the oracle's full step (FE, gradient, projected step,
    exact check) on B_w restarts of one instance, repeated until budget_s."""
    inst, B_w, budget_s, seed = task
    import numpy as np

    from oracle import fe_oracle as O
    from paper_2606_06641_gb300 import synth
    x = synth.uniform_x0(inst.n, B_w, seed).astype(np.float64)
    reps = 0
    t0 = time.perf_counter()
    while True:
        x = O.pgd_step(inst, x, 0.1)
        O.unsat_count(inst, x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return inst.n_lits * B_w * reps, el, reps


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_oracle_sample(insts, B_sample: int, budget_s: float, cores: int = 0, seed: int = 0):
    """The oracle's step on every host core at once (a spawned process per
    core, one numpy thread each): core w runs B_sample restarts of instance
    w mod len(insts) for about budget_s seconds. Returns the summed rate in
    literal-evals/s, the cores used and a description of the sample."""
    import multiprocessing as mp
    cores = cores or host_cores()
    tasks = [(insts[w % len(insts)], B_sample, budget_s, seed + w) for w in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_single_thread) as pool:
        res = pool.map(_oracle_worker, tasks)
    rate = sum(evals / el for evals, el, _ in res)
    steps = sum(r for _, _, r in res)
    n_inst = min(cores, len(insts))
    sample = (f"FP64 oracle step (FE, gradient, projected step, exact check) on {B_sample} restarts per core of "
              f"{n_inst} instance(s), {cores} cores in parallel for {budget_s:.0f} s ({steps} steps in total)")
    return rate, cores, sample


def run_reference(args):
    """The oracle as it stands, on all host cores: each of the K timed steps is
    a bounded sample of the workload (every core runs the oracle's step on its
    own restarts for --ref-step-s seconds); value = summed literal-evals/s."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    insts = make_workload(args.workload)
    desc, B_full = WORKLOADS[args.workload]
    B_sample = 8 if args.workload == "hybrid" else 2
    cores = host_cores()
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_sample(insts, B_sample, 0.0, cores)
    rates = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        r, cores, sample = cpu_oracle_sample(insts, B_sample, args.ref_step_s, cores)
        rates.append(r)
    el = time.perf_counter() - t_all
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "sample": f"{B_sample} of {B_full} restarts per core per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                         "sample": sample + f"; {args.steps} such steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_time_to_solve(n_inst: int, B: int, eta: float, max_steps: int, seed: int = 17):
    """Plain CLS vs the batched form on random 3-SAT instances (n=50, m=213),
    both from the same Philox starting points."""
    import numpy as np
    import torch

    from paper_2606_06641_gb300 import binding as bd
    from paper_2606_06641_gb300 import solver
    from paper_2606_06641_gb300 import synth
    insts = [synth.learned_split(i, "test") for i in range(n_inst)]
    hb = bd.load_batch(insts, bd.default_params(eta=eta, autotune=0))
    bd.init_restarts(hb, B, seed=seed)
    x_all = bd.get_x(hb)
    hb.free()
    x0s, v0 = [], 0
    for inst in insts:
        x0s.append(x_all[v0:v0 + inst.n].contiguous())
        v0 += inst.n
    torch.cuda.synchronize()
    solver.solve_batched(insts[:2], B, eta, 5, seed=seed)       # warm the library and allocator
    plain = solver.solve_plain(insts, B, eta, max_steps, x0s=x0s)
    batched = solver.solve_batched(insts, B, eta, max_steps, x0=x_all, steps_per_poll=10)
    ls = LINE_SEARCH
    batched_ls = solver.solve_batched(insts, B, eta, max_steps, x0=x_all, line_search=ls)
    forms = {"plain": (plain.solved, plain.seconds, plain.steps, plain.total_seconds),
             "batched": (batched.solved, batched.seconds, batched.steps, batched.total_seconds),
             "batched_line_search": (batched_ls.solved, batched_ls.seconds, batched_ls.steps,
                                     batched_ls.total_seconds)}
    out = tts_summary(forms)
    out.update({"instances": n_inst, "n": 50, "m": 213, "restarts": B, "eta": eta, "max_steps": max_steps,
                "line_search": {"s": ls[0], "beta": ls[1], "c": ls[2], "trials": ls[3],
                                "note": "Armijo backtracking per restart, checked every iteration"},
                "same_solved_set": bool(np.array_equal(plain.solved, batched.solved)),
                "start_points": "identical (Philox, batch convention) for both forms"})
    return out


def tts_summary(forms):
    """Time-to-solve at an equal solve rate: with k = half the smallest number
    of instances any form solved, each form's k-th fastest completion time
    (from the start of its run) is its median time-to-solve over that common
    solved fraction. Also the solve rate, median steps over solved instances
    and total wall time."""
    import numpy as np
    kmin = min(int(v[0].sum()) for v in forms.values())
    k = max(1, kmin // 2)
    res = {"equal_rate_rank": k}
    for name, (solved, secs, steps, wall) in forms.items():
        t = np.sort(np.where(solved, secs, np.inf))
        res[name] = {"solved": int(solved.sum()), "solve_rate": float(solved.mean()),
                     "median_tts_s": float(t[k - 1]) if kmin > 0 else None,
                     "median_steps_solved": float(np.median(steps[solved])) if solved.any() else None,
                     "wall_s": float(wall)}
    if "plain" in res and kmin > 0:
        for name in forms:
            if name != "plain" and res[name]["median_tts_s"]:
                res[f"{name}_vs_plain_speedup"] = res["plain"]["median_tts_s"] / res[name]["median_tts_s"]
    return res


def paired_bootstrap(d, reps: int = 2000, seed: int = 0):
    """Median of the paired differences d and its 95% bootstrap interval."""
    import numpy as np
    if d.size == 0:
        return None
    rng = np.random.default_rng(seed)
    meds = np.median(d[rng.integers(0, d.size, (reps, d.size))], axis=1)
    return {"median": float(np.median(d)), "ci95": [float(np.percentile(meds, 2.5)), float(np.percentile(meds, 97.5))],
            "pairs": int(d.size)}


def measure_learned(args):
    """Learned initialiser: train the message-passing network on the descent's
    own solutions of training instances, then solve the held-out instances in
    one batched handle from uniform starts and from the same starts nudged
    toward the network's proposal, and (the first ones) with plain CLS; times
    to solve are wall times from the start of each run (instance upload and,
    for the learned form, the network's inference included)."""
    import numpy as np
    import torch

    from paper_2606_06641_gb300 import binding as bd
    from paper_2606_06641_gb300 import learned, solver, synth
    eta, steps, B = 0.1, 500, 256
    t0 = time.perf_counter()
    train = [synth.learned_split(i, "train") for i in range(args.learned_train)]
    test = [synth.learned_split(i, "test") for i in range(args.learned_test)]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    labels = learned.harvest(train, 64, eta, steps, seed=1)
    t_harvest = time.perf_counter() - t0
    batches = learned.make_batches(labels, 64)
    net = bd.Mpnn(layers=3, seed=7)
    t0 = time.perf_counter()
    hist = learned.train(net, batches, args.learned_epochs, 3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    start = learned.DEFAULT_START
    for _ in range(2):  # warm-up of both forms (library caches, the network's workspace)
        learned.evaluate(None, test, B, eta, steps, seed=3)
        learned.evaluate(net, test, B, eta, steps, seed=3, start=start)
    res_u = learned.evaluate(None, test, B, eta, steps, seed=3)
    res_l = learned.evaluate(net, test, B, eta, steps, seed=3, start=start)
    n_plain = min(len(test), args.learned_plain)
    # plain CLS from the uniform form's own starting points (same trajectories)
    hs = bd.load_batch(test[:n_plain], bd.default_params(eta=eta, autotune=0))
    bd.init_restarts(hs, B, seed=3)
    x_all = bd.get_x(hs)
    hs.free()
    x0s, v0 = [], 0
    for inst in test[:n_plain]:
        x0s.append(x_all[v0:v0 + inst.n].contiguous())
        v0 += inst.n
    plain = solver.solve_plain(test[:n_plain], B, eta, steps, x0s=x0s)
    forms = {"uniform_batched": res_u, "learned_batched": res_l}
    summ_all = tts_summary({k: (v[0], v[2], v[1], v[3]) for k, v in forms.items()})
    summ_plain = tts_summary({k: (v[0][:n_plain], v[2][:n_plain], v[1][:n_plain], v[3]) for k, v in forms.items()} |
                             {"plain": (plain.solved, plain.seconds, plain.steps, plain.total_seconds)})
    both = res_u[0] & res_l[0]
    return {
        "metric": "median time-to-solve at equal solve rate (learned vs uniform starts, batched; plain CLS)",
        "unit": "s", "higher_is_better": False,
        "config": {"workload": f"random 3-SAT n=50 m=213; {args.learned_train} training instances, {len(test)} "
                               f"held-out, B={B}, {steps} steps, eta={eta}",
                   "network": "3 rounds, hidden 64, BF16 tensor-core GEMMs, FP32 accumulation",
                   "learned_starts": f"uniform starts nudged toward mu: x = clamp(u + alpha_b mu), alpha ramped "
                                     f"{start[1]}..{start[2]} over the restarts",
                   "timing": "wall time from the start of each run (instance upload, starting points, network "
                             "inference for the learned form, steps polled every 10); both forms warmed up"},
        "labels": {"labelled_instances": len(labels.insts), "mean_solutions": float(labels.n_solutions.mean())
                   if len(labels.insts) else 0.0},
        "train": {"epochs": args.learned_epochs, "loss_first": hist[0] if hist else None,
                  "loss_last": hist[-1] if hist else None, "train_s": t_train, "harvest_s": t_harvest,
                  "generate_s": t_gen},
        "held_out": {
            "uniform": {"solve_rate": float(res_u[0].mean()), "median_steps": float(np.median(res_u[1][res_u[0]]))
                        if res_u[0].any() else None, "wall_s": res_u[3]},
            "learned": {"solve_rate": float(res_l[0].mean()), "median_steps": float(np.median(res_l[1][res_l[0]]))
                        if res_l[0].any() else None, "wall_s": res_l[3]},
            "solved_only_by_learned": int((res_l[0] & ~res_u[0]).sum()),
            "solved_only_by_uniform": int((res_u[0] & ~res_l[0]).sum()),
            "paired_steps_uniform_minus_learned": paired_bootstrap(res_u[1][both] - res_l[1][both]),
            "paired_tts_s_uniform_minus_learned": paired_bootstrap(res_u[2][both] - res_l[2][both]),
        },
        "time_to_solve": summ_all,
        "time_to_solve_with_plain": summ_plain | {"instances": n_plain},
    }


def run_learned(args):
    from paper_2606_06641_gb300 import build as _b
    _b.build()
    print(json.dumps(measure_learned(args)), flush=True)
    return 0


def precision_report(inst, n_restarts: int = 4):
    """Max errors of the FE values and gradient against the FP64 oracle for the
    FP32 PGF basis, the paper's ESP basis with scaled products, and BF16 state
    (at the original FP32 point), on sampled restarts."""
    import numpy as np
    import torch

    from oracle import fe_oracle as O
    from paper_2606_06641_gb300 import binding as bd
    from paper_2606_06641_gb300 import synth
    x = synth.uniform_x0(inst.n, n_restarts, 5)
    fe_ref, _, g_ref = O.evaluate(inst, x.astype(np.float64))
    xd = torch.from_numpy(x).cuda()
    out = {}
    for name, params, xin in (("pgf_f32", bd.default_params(), xd),
                              ("esp_scaled_f32", bd.default_params(basis=bd.BASIS_ESP), xd),
                              ("pgf_bf16_state", bd.default_params(), xd.to(torch.bfloat16))):
        h = bd.load_instance(inst, params)
        fe, g = bd.eval_fe_grad(h, xin)
        fe = fe.cpu().numpy()
        g = g.cpu().numpy()
        k = np.diff(inst.lit_off)
        long_rows = k > 32
        d_fe = np.abs(fe - fe_ref)
        d_g = np.abs(g - g_ref)
        out[name] = {"fe_max_err": float(np.nanmax(np.where(np.isfinite(d_fe), d_fe, np.inf))),
                     "fe_max_err_long": float(np.nanmax(np.where(np.isfinite(d_fe[long_rows]), d_fe[long_rows], np.inf))),
                     "grad_max_err": float(np.nanmax(np.where(np.isfinite(d_g), d_g, np.inf)))}
        h.free()
    return {"restarts": n_restarts, **out}


STEP_MODES = {"auto": 0, "persistent": 1, "graph": -1}   # afs_params.persistent
KIND_NAMES = {0: "fe_grad_short_kernel", 1: "fe_grad_long_pgf_kernel", 2: "fused_grad_kernel"}
COUNTERS_FILE = os.path.join(ROOT, "profiles", "kernel_counters.json")


def load_counters(workload: str):
    """ncu counters recorded for this workload, per kernel (executed warp
    instructions and DRAM bytes per restart per step): those taken on the
    kernel's current sources."""
    if not os.path.exists(COUNTERS_FILE):
        return {}
    with open(COUNTERS_FILE) as fh:
        per_kernel = json.load(fh).get("workloads", {}).get(workload, {})
    return {k: c for k, c in per_kernel.items()
            if k in KERNEL_SOURCES and c.get("kernel_source_hash") == kernel_source_hash(k)}


def long_kernel_form_ops(insts, tiles) -> float:
    """FP32 operations per restart and step of the long kernel's own forms,
    summed over the long constraints (k > 32) from each table's head and the
    lanes per restart W of the constraint's length group: per root the
    forward walk (W >= 16: twelve per octet, three per literal past the last
    octet; W = 8: three per literal, four in form B), four per segment for
    s^16 and six for T and the value; per exactly treated root and literal
    3.25 (four-root fractions, W >= 16 and k > 4 W) or 4 (one term a root);
    per expanded root 2 nc (its sums), plus 3 nc per literal for the
    Chebyshev sum; 4 per literal for the real root's scan."""
    import numpy as np

    from paper_2606_06641_gb300 import binding as bd
    groups = sorted((km, lw) for lw, _, km in tiles)  # shortest first
    cache = {}
    total = 0.0
    for inst in insts:
        ks = inst.lengths
        for c in np.nonzero(ks > 32)[0]:
            k = int(ks[c])
            key = (int(inst.ctype[c]), k, int(inst.op[c]), int(inst.param[c]), int(inst.parity[c]))
            if key not in cache:
                t = bd.coef_table(*key, basis=bd.BASIS_PGF, form=1).astype(np.float64).reshape(-1, 4)
                cache[key] = (int(t[0, 1]), t[0, 3] > 0.5, int(t[1, 0]), int(t[1, 1]), int(t[1, 2]))
            nr, has_real, fb, nx, nc = cache[key]
            W = next((lw for km, lw in groups if km >= k), 32)
            nseg = (k + 15) // 16
            fwd = (12 * (k // 8) + 3 * (k % 8) if W >= 16 else 3 * k) + 4 * (nseg - 1) + 6
            nx = nx // W * W if nc <= 2 * W else 0
            d_exact = (3.25 if W >= 16 and k > 4 * W else 4.0) * k
            ops = nr * fwd + (nr - nx) * d_exact + nx * 2 * nc + (3 * nc * k if nx else 0)
            if W < 16:
                ops += max(0, nr - fb) * k
            if has_real:
                ops += 4 * k
            total += ops
    return total


def dominant_kernel(groups, B: int, chunk: int, peak_tinst: float, peak_src: str, sm_max: float, sms: int,
                    counters, long_form_ops: float = 0.0):
    """Roofline object of the kernel with the largest FE+gradient time per
    step: achieved = its algorithmic instructions per launch / its event-timed
    duration per launch (launches over the same chunk of restarts)."""
    launches_per_step = (B + chunk - 1) // chunk
    per_kind = {}
    for kind, kmax, ms, work in groups:
        d = per_kind.setdefault(kind, {"ms": 0.0, "work": 0.0, "launches": 0, "kmax": []})
        d["ms"] += ms
        d["work"] += work
        d["launches"] += 1
        d["kmax"].append(kmax)
    kind = max(per_kind, key=lambda k: per_kind[k]["ms"])
    d = per_kind[kind]
    total_ms = sum(v["ms"] for v in per_kind.values())
    achieved = d["work"] / (d["ms"] * 1e-3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak_tinst, "unit": "Tinst/s",
           "frac": achieved / peak_tinst, "traffic": None,
           "kernel": KIND_NAMES[kind],
           "launches_per_step": d["launches"] * launches_per_step,
           "ms_per_step": d["ms"] * launches_per_step,
           "share_of_fe_time": d["ms"] / total_ms if total_ms else None,
           "group_lengths": d["kmax"],
           "work_instr_per_step": d["work"] * launches_per_step,
           "accounting": "algorithmic FP32 lane instructions: 16 per (literal, root) + 2 per root, "
                         "R(k) = floor((k+1)/2); fused 3-literal pass: 3 per occurrence",
           "timing": "CUDA events on the launching stream around each launch group of the step "
                     "(afs_group_times, 5 launches per group over one restart chunk, current state)",
           "peak_basis": f"{sms} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (max SM clock, {peak_src})"}
    if kind == 1 and long_form_ops > 0:
        # the long kernel's own forms (octet walk, gradient by division in
        # four-root fractions, Chebyshev-expanded roots): their FP32
        # operations per step over the same event-timed launches
        ops = long_form_ops * B
        out["kernel_form"] = {"ops_per_step": ops,
                              "achieved": ops / (out["ms_per_step"] * 1e-3) / 1e12,
                              "frac": ops / (out["ms_per_step"] * 1e-3) / 1e12 / peak_tinst,
                              "note": "the frac above counts 16 per (literal, root), the prefix/suffix work "
                                      "model; this one the FP32 operations the kernel's forms take "
                                      "(long_kernel_form_ops)"}
    elif kind == 0 and max(d["kmax"]) <= 24:
        # the short kernel's own algorithm (gradient by division): per
        # (literal, root) 3 FP32 instructions for the forward product and,
        # for the derivative, w = l / gamma, numerator, denominator,
        # reciprocal and sum
        own = 8
        out["division_form"] = {"instr_per_literal_root": own,
                                "frac": achieved / peak_tinst * own / 16.0,
                                "note": "the frac above counts 16 per (literal, root), the prefix/suffix work model"}
    counters = counters.get(KIND_NAMES[kind]) if counters else None
    if counters:
        wi = counters["warp_inst_per_restart_step"] * B
        out["executed_lane_instr_per_step"] = 32.0 * wi
        out["issue_frac"] = 32.0 * wi / (out["ms_per_step"] * 1e-3) / 1e12 / peak_tinst
        out["traffic"] = counters.get("dram_bytes_per_restart_step", 0.0) * B / out["launches_per_step"]
        out["counters_source"] = counters.get("source")
    return out


def measure_workload(name: str, args, rank: int, world: int, stream, want_cpu: bool, want_e2e: bool,
                     sample_clocks: bool, dev: int):
    """Time one workload: K steps as graph replays (the contract's figure), a
    sustained figure over >= --sustained-s of replays, the dominant kernel's
    roofline, the end-to-end figure through host buffers, the CPU oracle."""
    import torch

    from paper_2606_06641_gb300 import binding as bd
    desc, B_default = WORKLOADS[name]
    B = (args.restarts if name == args.workload else 0) or B_default
    insts = make_workload(name)
    params = bd.default_params(eta=0.1, verify_every=1, chunk=args.chunk, autotune=0 if args.tiles else 1,
                               persistent=STEP_MODES[args.step_mode])
    h = bd.load_instance(insts[0], params) if len(insts) == 1 else bd.load_batch(insts, params)
    bd.init_restarts(h, B, seed=1000 + rank)
    if args.tiles and name == args.workload:
        bd.set_tiles(h, *bd.parse_tiles(args.tiles))
    if args.long_tiles and name == args.workload:
        bd.set_long_tiles(h, [tuple(int(v) for v in t.split("x")) for t in args.long_tiles.split(",")])
    S = max(1, min(args.steps_per_graph, args.steps))
    R = max(1, args.steps // S)
    K = R * S
    L = sum(i.n_lits for i in insts)
    n_total = sum(i.n for i in insts)

    # warm-up: W single steps, then one untimed replay of the timed graph
    for _ in range(max(args.warmup, 3)):
        bd.step(h, 1)
    bd.step(h, S)
    torch.cuda.synchronize()

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sampler = ClockSampler(gpu_id_for(dev)) if (rank == 0 and sample_clocks) else None
    if sampler:
        sampler.start()
        time.sleep(0.4)

    def replays(count):
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(count)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(count)]
        n_launch = 0
        for r in range(count):
            flush.fill_(float(r))
            e0[r].record(stream)
            bd.step(h, S)
            # each replay ends, as a solver's poll does, with the exact count of
            # the state it left (two kernels: the counting check and the fold)
            bd.get_verify(h)
            e1[r].record(stream)
            n_launch += bd.last_launch_count(h) + 2
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(e0, e1)), n_launch

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # (the timed replays are the profiler's capture range: ncu --profile-from-start off)
    torch.cuda.profiler.start()
    dev_ms, launches = replays(R)
    torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    # sustained: replays until at least --sustained-s of device time
    sus_ms, sus_steps = dev_ms, K
    while sus_ms < 1e3 * args.sustained_s:
        more = max(1, int((1e3 * args.sustained_s - sus_ms) / max(sus_ms / (sus_steps / S), 1e-3)) + 1)
        m_ms, _ = replays(min(more, 5000))
        sus_ms += m_ms
        sus_steps += min(more, 5000) * S
    clocks = sampler.stop() if sampler else None
    t = torch.tensor([dev_ms, sus_ms / sus_steps * K], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    dev_ms, sus_equiv = float(t[0].item()), float(t[1].item())

    # phase breakdown from an instrumented replay of the same length: event
    # nodes inside the graph around the FE phase and the CSR pass of every
    # step (they serialise the graph, so they stay out of the timed replays)
    bd.set_kernel_timing(h, True)
    bd.step(h, S)
    torch.cuda.synchronize()
    bd.set_kernel_timing(h, True)  # reset the sums, keep the instrumented graph
    for r in range(R):
        flush.fill_(float(r))
        bd.step(h, S)
    torch.cuda.synchronize()
    fe_ms, fe_n, csr_ms, csr_n = bd.kernel_timing(h)
    bd.set_kernel_timing(h, False)

    # per launch group: event-timed launches on this stream, algorithmic work
    groups = bd.group_times(h, reps=5, stream=stream)
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = props.multi_processor_count
    peak_tinst = sms * 128 * sm_max * 1e6 / 1e12
    chunk, rpl = bd.tuning(h)
    roof = dominant_kernel(groups, B, chunk, peak_tinst, peak_src, sm_max, sms, load_counters(name),
                           long_kernel_form_ops(insts, bd.long_tiles(h)))
    step_work = sum(w for _, _, _, w in groups) * ((B + chunk - 1) // chunk)
    roof["step_work_instr"] = step_work
    roof["step_frac"] = step_work / (dev_ms / K * 1e-3) / 1e12 / peak_tinst
    roof["fe_ms_per_step"] = fe_ms / K
    roof["csr_ms_per_step"] = csr_ms / K
    roof["phases_measured"] = ("FE phase (length buckets, fused pass, per-step check; concurrent) and CSR pass "
                               "from an instrumented replay of the same steps (event nodes in the graph)")

    # end to end through the public API: pinned host x in, one step, x and unsat counts out
    e2e = None
    if want_e2e:
        x_host = bd.get_x(h).cpu().pin_memory()
        for _ in range(2):
            bd.step_host(h, x_host, x_host)
        E = max(3, min(args.steps, 30))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(E):
            bd.step_host(h, x_host, x_host)
        el = time.perf_counter() - t0
        e2e = {"value": L * B * E * world / el, "unit": UNIT, "h2d_bytes_per_step": n_total * B * 4,
               "d2h_bytes_per_step": n_total * B * 4 + len(insts) * B * 4, "steps": E}
    tiles = bd.format_tiles(*bd.tiles(h))
    long_tiles = [f"k<={km}:{lw}x{nw}" for lw, nw, km in bd.long_tiles(h)]
    pmode, pblocks = bd.step_mode(h)
    h.free()
    del flush
    torch.cuda.empty_cache()

    cpu = None
    if want_cpu:
        Bs = 8 if name == "hybrid" else 2
        v, cores, sample = cpu_oracle_sample(insts, Bs, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle", "sample": sample}

    return {
        "value": L * B * K * world / (dev_ms * 1e-3), "ms_per_step": dev_ms / K, "steps": K,
        "sustained": {"value": L * B * K * world / (sus_equiv * 1e-3), "ms_per_step": sus_equiv / K,
                      "steps": sus_steps, "device_s": sus_ms / 1e3},
        "config": {"workload": desc, "restarts": B, "literals": L, "instances": len(insts),
                   "l2": f"flushed (512 MB write) between timed replays of {S} steps",
                   "step_mode": (f"persistent ({pblocks} cooperative blocks, one launch per replay)" if pmode
                                 else "CUDA-graph replay of the per-step launches"),
                   "chunk_restarts": chunk, "restarts_per_lane": rpl, "tiles": tiles, "long_tiles": long_tiles,
                   "tiles_source": "given" if (args.tiles and name == args.workload) else "autotuned",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
    }


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()

    from paper_2606_06641_gb300 import build as _b
    if rank == 0 or world == 1:
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    solo = rank == 0 and world == 1
    head = measure_workload(args.workload, args, rank, world, stream, solo and not args.no_cpu,
                            not args.no_e2e, True, dev)
    extras = {}
    for name in [w for w in args.extras.split(",") if w and w != args.workload]:
        extras[name] = measure_workload(name, args, rank, world, stream, solo and not args.no_cpu,
                                        not args.no_e2e, True, dev)
    tts = None
    if rank == 0 and not args.no_tts:
        tts = measure_time_to_solve(args.tts_instances, 32, args.tts_eta, 500)
    learned_res = None
    if rank == 0 and not args.no_learned:
        learned_res = measure_learned(args)
    precision = None
    if rank == 0 and args.workload == "long" and not args.no_cpu:
        precision = precision_report(make_workload("long")[0])

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": head["steps"],
            "warmup": max(args.warmup, 3), "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": head["config"], "roofline": head["roofline"], "cpu_baseline": head["cpu_baseline"],
            "e2e": head["e2e"], "clocks": head["clocks"], "gpu_launches": head["gpu_launches"],
            "sustained": head["sustained"],
        }
        if extras:
            line["workloads"] = {k: {kk: vv for kk, vv in v.items() if kk != "steps"} for k, v in extras.items()}
        if tts is not None:
            line["time_to_solve"] = tts
        if learned_res is not None:
            line["learned"] = learned_res
        if precision is not None:
            line["precision"] = precision
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch_sweep(args):
    """Throughput against the restart count B for one workload (where the
    autotuned chunk and the L2 make the rate peak). One line per run:
    B, chunk, tiles, literal-evals/s, ms per step; same timing rules as the
    main measurement (graph replays of 10 steps, L2 flushed between)."""
    import torch
    from paper_2606_06641_gb300 import binding as bd
    from paper_2606_06641_gb300 import build as _b
    _b.build()
    insts = make_workload(args.workload)
    L = sum(i.n_lits for i in insts)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # half a second of device work first, so that the first point does not
    # run at the idle clocks
    t_end = time.time() + 0.5
    while time.time() < t_end:
        flush.fill_(1.0)
        torch.cuda.synchronize()
    rows = []
    for B in [int(b) for b in args.sweep_b.split(",")]:
        params = bd.default_params(eta=0.1, verify_every=1)
        h = bd.load_instance(insts[0], params) if len(insts) == 1 else bd.load_batch(insts, params)
        bd.init_restarts(h, B, seed=1000)
        S, R = 10, max(1, args.steps // 10)
        for _ in range(3):
            bd.step(h, 1)
        bd.step(h, S)
        torch.cuda.synchronize()
        ms = 0.0
        for r in range(R):
            flush.fill_(float(r))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bd.step(h, S)
            bd.get_verify(h)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        chunk, tiles = bd.tiles(h)
        rows.append({"B": B, "value": L * B * R * S / (ms * 1e-3), "ms_per_step": ms / (R * S), "chunk": chunk,
                     "tiles": bd.format_tiles(chunk, tiles)})
        h.free()
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"metric": METRIC, "unit": UNIT, "workload": WORKLOADS[args.workload][0],
                      "batch_sweep": rows}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="long", choices=sorted(WORKLOADS) + ["learned"])
    ap.add_argument("--extras", default="hybrid,batch",
                    help="comma-separated further workloads measured into the same line ('' for none)")
    ap.add_argument("--sustained-s", type=float, default=1.0, help="device seconds of the sustained figure")
    ap.add_argument("--ref-step-s", type=float, default=4.0, help="reference arm: seconds per sampled step")
    ap.add_argument("--learned-train", type=int, default=10000)
    ap.add_argument("--learned-test", type=int, default=512)
    ap.add_argument("--learned-epochs", type=int, default=30)
    ap.add_argument("--learned-plain", type=int, default=128, help="held-out instances also run by plain CLS")
    ap.add_argument("--restarts", type=int, default=0, help="restarts per GPU (0 = the workload's)")
    ap.add_argument("--steps-per-graph", type=int, default=10)
    ap.add_argument("--chunk", type=int, default=0, help="restarts per chunk (0 = autotuned)")
    ap.add_argument("--tiles", default="", help="fixed chunk and tiles, 'chunk:k=RPLxCPW,...' (no autotuning)")
    ap.add_argument("--long-tiles", default="", help="fixed long-group tiles, 'LANESxWARPS,...' longest group first")
    ap.add_argument("--sweep-b", default="", help="comma-separated restart counts: throughput against B")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--tts-instances", type=int, default=128)
    ap.add_argument("--tts-eta", type=float, default=0.1)
    ap.add_argument("--step-mode", default="auto", choices=sorted(STEP_MODES),
                    help="steps as graph-replayed per-step launches, one persistent launch, or the faster (autotuned)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tts", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload == "learned":
            args.workload = "long"
        return run_reference(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.sweep_b:
        return run_batch_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
