#!/usr/bin/env python
"""Throughput of the TSFCDE time march on GB300: grid-point updates per second (n * M / s).

A step is one whole time march of the workload (all M levels: history sum, FFT Toeplitz
products, circulant-preconditioned CGS per level) from u^0, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--workload large|small|mixed|batch|history] [--precond tchan|strang|none]
                    [--precision fp64|mixed] [--algorithm ids|ids-const] [--instances K]
                    [--no-autotune] [--no-cpu-baseline] [--co]

Default workload: n = 2^16-1 interior points, M = 1024 levels, alpha = 0.3, beta = 1.9,
gamma = 0.5, d+ = 1+t, d- = 1-t/2, u = (t^2+1) x^2 (1-x)^2, T. Chan preconditioner, tol 1e-12,
FP64.  Other workloads: small (n = 127, M = 64, Strang), mixed (n = 2^20-1, M = 512, mixed
precision by default), batch (4096 constant-coefficient instances, M = 256; --algorithm
ids-const applies A^{-1} by the Gohberg-Semencul formula for j >= 1), history (n = 2^18-1,
M = 8192, mixed precision with FP64 history; --co adds the convergence order in tau).

Multi-GPU (torchrun): one instance runs as independent replicas, one per rank (the march is
sequential in time and a single instance does not shard; weak scaling); the batch and history
workloads shard their instances over the ranks by estimated cost (strong scaling).  The step
time is the slowest rank's.

--impl reference times the FP64 CPU oracle (dense Gaussian elimination per level) on the host
cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import tsfcde_workloads as W  # noqa: E402

_ARGS = None
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12     # SMs x FP64 FMA/clk x 2 flop x max clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 FMA/clk x 2 flop x max clock


def hbm_peak():
    """Measured copy bandwidth (MEASURED_PEAKS.json) or the profiling recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (profiling recipe)"


def roofline(kernel, flops, kernel_ms, precision, outer_steps=0):
    """Roofline entry of the dominant kernel: the algorithmic flops of the FP64 method (the FFT
    Toeplitz products, the history sum and the vector work, counted as if every operation were
    FP64) per second, against the FP64 pipe's peak derived from unit counts and clocks.  The FP64
    path is bound by that pipe.  The mixed path does the same algorithmic work with its inner
    solves on the FP32 pipe (FP32 or float-float, 1 to ~20 FP32 instructions per flop), so its
    fraction reads as the FP64-equivalent rate it reaches: above 1 would mean it beats a perfect
    FP64 kernel."""
    achieved = flops / (kernel_ms / 1e3) / 1e12
    peak = FP64_PEAK_TFLOPS
    src = "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (recipe nominal FP64 1.25 TFLOP/s)"
    out = {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": None, "peak_source": src}
    if precision != "fp64":
        out["note"] = ("mixed precision: FP64-equivalent rate of the method's algorithmic flops; "
                       "the inner solves run on the FP32 pipe and are latency/issue bound (ncu "
                       "summary in profiles/)")
    return out


class Ranks:
    """One process per GPU (torchrun env): world, rank, local device, the process group."""

    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None

    def init(self):
        import torch
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            self.dist = dist
        torch.cuda.set_device(self.local)
        return self

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x):
        from paper_1603_00279_gb300.multirank import max_over_ranks
        return max_over_ranks(x, self.dist, device="cuda")


def shard_instances(probs, ranks):
    """This rank's instances: cost-balanced shards of the whole set (strong scaling)."""
    from paper_1603_00279_gb300.multirank import instance_cost, shard
    if len(probs) < ranks.world:
        raise SystemExit(f"{len(probs)} instances cannot be shared by {ranks.world} ranks "
                         "(use --instances >= the number of GPUs)")
    costs = [instance_cost(q.n, q.M) for q in probs]
    return [probs[i] for i in shard(costs, ranks.world, ranks.rank)]


def workload(name: str, precond):
    if name == "large":
        p = W.config_large()
    elif name == "small":
        p = W.config_small()
    elif name in ("mixed", "precision"):
        p = W.config_mixed()
        p.name = name
    elif name == "batch":
        return W.config_batch(count=_ARGS.instances or 4096)
    elif name == "history":
        return W.config_history()[:(_ARGS.instances or 1)]
    else:
        raise SystemExit(f"unknown workload {name}")
    if precond:
        p.preconditioner = precond
    return p


def describe(p) -> dict:
    name = "history" if p.name.startswith("history") else p.name
    if name == "mixed":
        name = "precision"
    return {"workload": f"tsfcde_{name}", "n": p.n, "M": p.M, "alpha": p.alpha, "beta": p.beta,
            "preconditioner": p.preconditioner, "tol": p.tol, "source": "separable(4)",
            "updates_per_step": p.n * p.M}


# ---------------------------------------------------------------------------------------------
# algorithmic work of one march (FFT flops by the 5 N log2 N convention for a complex FFT of
# length N; a real-input transform of length L counts 2.5 L log2 L)
# ---------------------------------------------------------------------------------------------
def algorithmic_flops(p, iters: np.ndarray, newsym_levels: int) -> float:
    return _alg_flops(p.n, p.M, p.preconditioner, iters, newsym_levels)


def _alg_flops(n, M, preconditioner, iters, newsym_levels):
    L = max(8, 1 << math.ceil(math.log2(2 * n)))
    lg = math.log2(L)
    conv = 5.0 * L * lg + 3.0 * L
    pc = preconditioner != "none"
    convs = M + (4 if pc else 2) * float(iters.sum())
    sym = (12.5 * L * lg + 24.0 * n) if pc else 0.0
    hist = 2.0 * n * (M * (M - 1) / 2.0)
    vec = 19.0 * n * float(iters.sum()) + 12.0 * n * M
    return conv * convs + sym * newsym_levels + hist + vec


def _fast_history_flops(n, M, B=128):
    """FP64 flops of the history sum as the fast history computes it (blocked FFT convolution in
    time, blocks of B levels), per march: per block start q >= 1 one 2B-point complex FFT per two
    points for the new block and one inverse per two points (5 B log2(2B) flops per point each),
    and q (B+1) complex multiply-adds (8 flops) per point; per level the endpoint term, the far
    part and the direct terms of its own block (2 flops each)."""
    lg = math.log2(2 * B)
    f = 0.0
    for q in range(1, (M - 1) // B + 1):
        f += 2 * 5.0 * B * lg + 8.0 * q * (B + 1)
    for j in range(1, M):
        f += 2.0 * (j % B) + 3.0 if j >= B else 2.0 * j
    return f * n


def _alg_flops_const(n, M, preconditioner, iters, applications):
    """Algorithm "... with constant coefficients": the CGS iterations of level 0 and of the two
    generator solves, one right-hand-side product per level, and per application of A^{-1}
    four triangular Toeplitz products plus the FP64 residual product; the generator refinement
    (2 x 5 products) and the factor spectra (8 forward transforms, once per march)."""
    L = max(8, 1 << math.ceil(math.log2(2 * n)))
    lg = math.log2(L)
    conv = 5.0 * L * lg + 3.0 * L
    pc = preconditioner != "none"
    convs = M + (4 if pc else 2) * float(iters.sum()) + 5.0 * applications + 10.0 + 4.0
    sym = (12.5 * L * lg + 24.0 * n) if pc else 0.0
    hist = 2.0 * n * (M * (M - 1) / 2.0)
    vec = 19.0 * n * float(iters.sum()) + 12.0 * n * M + 6.0 * n * applications
    return conv * convs + sym * 2 + hist + vec


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self) -> dict:
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample (the reference arm and the cpu_baseline)
# ---------------------------------------------------------------------------------------------
def oracle_sample(p, budget_s: float = 15.0):
    """Time the oracle (dense GE per level) on the workload's parameters at a reduced n, for as
    many levels as fit the budget; returns (updates/s, description, cores)."""
    import oracle as O
    n_s = min(p.n, 2047)
    if p.name.startswith("history"):
        q = W.config_history(n=n_s, M=p.M)[int(p.name[len("history"):])]
    else:
        cls = {"large": W.config_large, "small": W.config_small, "mixed": W.config_mixed,
               "precision": W.config_mixed}[p.name]
        q = cls(n=n_s, M=p.M)
    q.preconditioner = p.preconditioner
    t0 = time.perf_counter()
    levels = 1
    O.run(q, levels=1)
    dt = time.perf_counter() - t0
    if dt < budget_s / 4:
        levels = max(2, min(p.M, int(budget_s / max(dt, 1e-3))))
        t0 = time.perf_counter()
        O.run(q, levels=levels)
        dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    desc = (f"oracle (dense LU per level, numpy/LAPACK) on the workload's alpha, beta and "
            f"coefficients at n={n_s} (workload n={p.n}), levels 0..{levels - 1} of M={p.M}; "
            f"{dt:.1f} s; value scaled to the workload's n by the n^-2 law of dense LU "
            f"(x{(n_s / p.n) ** 2:.3g})")
    return n_s * levels / dt, desc, cores, dt, n_s, levels


def oracle_single_core(p):
    """One level of the oracle at the sample size on one core (BLAS limited to one thread in a
    child process), in updates/s, or None if the child fails."""
    n_s = min(p.n, 2047)
    code = (
        "import sys, time, json\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import oracle as O, tsfcde_workloads as W\n"
        f"name = {p.name!r}\n"
        f"n_s, M = {n_s}, {p.M}\n"
        "if name.startswith('history'):\n"
        "    q = W.config_history(n=n_s, M=M)[int(name[7:])]\n"
        "else:\n"
        "    q = {'large': W.config_large, 'small': W.config_small, 'mixed': W.config_mixed,\n"
        "         'precision': W.config_mixed}[name](n=n_s, M=M)\n"
        "t0 = time.perf_counter(); O.run(q, levels=1); dt = time.perf_counter() - t0\n"
        "print(json.dumps(n_s / dt))\n")
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=120)
        return {"value": float(r.stdout.strip().splitlines()[-1]), "unit": "updates/s", "cores": 1,
                "sample": f"one level at n={n_s}"}
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return None


def run_reference(args, p):
    """The reference arm: the FP64 CPU oracle timed on the host cores, each step a bounded sample
    of the workload (its parameters at n = 2047), reported at the workload's n by the dense-LU
    law like cpu_baseline; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals, descs = [], []
    for _ in range(min(args.warmup, 1)):
        oracle_sample(p, budget_s=2.0)
    t_all = 0.0
    n_s = levels = 0
    for _ in range(args.steps):
        v, d, cores, dt, n_s, levels = oracle_sample(p, budget_s=args.ref_budget)
        vals.append(v)
        t_all += dt
        descs.append(d)
    v_sample = float(np.mean(vals))
    v = v_sample * (n_s / p.n) ** 2
    line = {"metric": "grid-point updates/s", "value": v, "unit": "updates/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (manufactured solution)",
            "config": {**describe(p), "oracle_sample_n": n_s},
            "cpu_baseline": {"value": v, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": descs[-1], "extrapolated": p.n != n_s,
                             "measured_sample": {"n": n_s, "levels": levels, "value": v_sample}},
            "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_reference_batch(args, probs):
    import oracle as O
    if int(os.environ.get("RANK", "0")) != 0:
        return
    M = probs[0].M
    vals = []
    t_all = 0.0
    desc = ""
    for _ in range(args.steps):
        t0 = time.perf_counter()
        upd, k = 0, 0
        while time.perf_counter() - t0 < 20.0 and k < len(probs):
            O.run(probs[k], levels=min(M, 8))
            upd += probs[k].n * min(M, 8)
            k += 1
        dt = time.perf_counter() - t0
        t_all += dt
        vals.append(upd / dt)
        desc = f"oracle (dense LU per level) on the first {k} instances of the batch, levels 0..7 each"
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    v = float(np.mean(vals))
    ns = np.array([q.n for q in probs])
    print(json.dumps({"metric": "grid-point updates/s", "value": v, "unit": "updates/s",
                      "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f64", "data": "synthetic (seeded instances)",
                      "config": {"workload": "tsfcde_batch", "instances": len(probs), "M": M,
                                 "sum_n": int(ns.sum())},
                      "cpu_baseline": {"value": v, "unit": "updates/s", "cores": cores,
                                       "kind": "oracle", "sample": desc},
                      "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------------------------
def kernel_sources_sha() -> str:
    """sha256 over the CUDA sources (sorted by name): identifies the kernels an ncu capture saw."""
    import hashlib
    d = os.path.join(ROOT, "paper_1603_00279_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def captured_traffic(name: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel
    from the committed ncu summary profiles/<name>, if that capture saw the current kernel sources
    (its `kernel_sources_sha256` line); else (None, reason)."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None, f"no capture ({name})"
    kv = {}
    for l in lines:
        l = l.strip().lstrip("-* `")
        if ":" in l and l.startswith(("traffic_bytes_per_launch", "kernel_sources_sha256")):
            k, v = l.split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    try:
        traffic = float(kv["traffic_bytes_per_launch"])
        sha = kv["kernel_sources_sha256"]
    except (KeyError, ValueError):
        return None, f"capture {name} has no traffic line"
    if sha != kernel_sources_sha():
        return None, f"kernel sources changed since the capture in profiles/{name}"
    return traffic, f"ncu capture, profiles/{name}"


def estimate_total_s(march_s: float, setup_s: float, steps: int, warmup: int, cpu_budget: float,
                     mixed_march_s: float = 0.0) -> float:
    """Wall time of one default single-instance bench run: warm-up and timed marches, the e2e
    march, the mixed-precision leg (one march plus its setup), the CPU oracle leg (the timed
    sample plus one single-core level) and setup."""
    marches = warmup + steps + 1
    return setup_s * 2 + marches * march_s + 1.2 * mixed_march_s + 1.5 * cpu_budget + 30.0


def level_gap(s_ref, s_other, levels):
    """Relative L2 gap per level between two marches (levels rebuilt through tsfcde_get_level)."""
    out = {}
    for j in levels:
        a, _ = s_ref.get_level(j)
        b, _ = s_other.get_level(j)
        den = float(np.linalg.norm(a))
        out[int(j)] = float(np.linalg.norm(b - a) / (den if den > 0 else 1.0))
    return out


def run_native(args, p):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1603_00279_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    import paper_1603_00279_gb300 as P

    stream = torch.cuda.Stream()
    lpl = args.levels_per_launch
    t_setup = time.perf_counter()
    s = P.Solver.from_problem(p, source="separable", device=local, stream=stream.cuda_stream,
                              maxit=args.maxit, precision=args.precision,
                              autotune=not args.no_autotune, levels_per_launch=lpl)
    setup_ms = 1e3 * (time.perf_counter() - t_setup)
    plan = s.plan()
    n, M = p.n, p.M

    def one_step():
        s.reset()
        return s.step(M)

    for _ in range(args.warmup):
        one_step()
    # timed region: device-resident inputs, one whole march per step
    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(one_step())
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * n * M * args.steps / (ms_max / 1e3)
    it, res = s.history(M)
    launches = int(sum(st["device_launches"] for st in stats))
    launches_per_step = launches / max(1, len(stats))
    kernel_ms = float(np.mean([st["device_ms"] for st in stats]))   # per march, all its launches
    newsym = M if p.name != "batch" else 2
    flops = algorithmic_flops(p, it, newsym)
    if args.precision == "mixed":   # one FP64 residual product per refinement step
        L = max(8, 1 << math.ceil(math.log2(2 * n)))
        outer = sum(st["outer_iterations"] for st in stats) / max(1, len(stats))
        flops += outer * (5.0 * L * math.log2(L) + 3.0 * L)

    # the history phase alone at the last level (reads all M-1 committed increments)
    hist = None
    if M >= 2:
        jh = M - 1
        for _ in range(2):
            s.history_sum(jh, want=False)
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        h0.record(stream)
        for _ in range(reps):
            s.history_sum(jh, want=False)
        h1.record(stream)
        torch.cuda.synchronize()
        hms = h0.elapsed_time(h1) / reps
        hbytes = 8.0 * n * jh + 16.0 * n
        peak = hbm_peak()
        hist = {"kernel": "history phase (level M-1)", "bound": "hbm",
                "achieved": hbytes / (hms / 1e3) / 1e9, "peak": peak[0], "unit": "GB/s",
                "frac": hbytes / (hms / 1e3) / 1e9 / peak[0], "traffic": None,
                "ms": hms, "fp64_tflops": 2.0 * n * jh / (hms / 1e3) / 1e12,
                "peak_source": peak[1]}

    fp64_measured = P.measure_fp64(local)    # the FP64 unit's FMA throughput, measured now

    # end to end through the C ABI with pinned host buffers: H2D of u^0, the march, D2H of u^M;
    # u^0 is the library's own sample of phi on its mesh (level 0 read back after a reset)
    s.reset()
    u0 = torch.from_numpy(s.get_level(0)[0]).pin_memory()
    uM = torch.empty(n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.reset(u0_ptr=u0.data_ptr())
    s.solve(out_ptr=uM.data_ptr())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    e2e_val = world * n * M / float(tt.item())

    # accuracy of the march against the manufactured solution (a property at any size)
    u_end = uM.numpy()
    err = float(np.sqrt(p.h) * np.linalg.norm(u_end - p.exact(p.grid(), p.T)))

    # mixed-precision leg of the precision workload: one timed march, and its per-level gap to
    # the FP64 march above (both contexts hold every level through their increment rings)
    mixed = None
    if args.precision == "fp64" and args.mixed_leg and world == 1:
        ts = time.perf_counter()
        sm = P.Solver.from_problem(p, source="separable", device=local, stream=stream.cuda_stream,
                                   maxit=args.maxit, precision="mixed",
                                   autotune=not args.no_autotune, levels_per_launch=lpl)
        msetup = 1e3 * (time.perf_counter() - ts)
        torch.cuda.synchronize()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        mst = sm.step(M)
        m1.record(stream)
        torch.cuda.synchronize()
        mms = m0.elapsed_time(m1)
        levels = sorted(set(list(range(1, min(M, 8) + 1)) +
                        [j for j in (16, 32, 64, 128, 256, M // 2, 3 * M // 4, M - 1, M) if 1 <= j <= M]))
        gaps = level_gap(s, sm, levels)
        um = sm.get_level(M)[0]
        merr = float(np.sqrt(p.h) * np.linalg.norm(um - p.exact(p.grid(), p.T)))
        it_m, _ = sm.history(M)
        mflops = algorithmic_flops(p, it_m, M)
        L_ = max(8, 1 << math.ceil(math.log2(2 * n)))
        mflops += mst["outer_iterations"] * (5.0 * L_ * math.log2(L_) + 3.0 * L_)
        mixed = {"value": n * M / (mms / 1e3), "unit": "updates/s", "ms_per_march": mms,
                 "roofline": roofline("level_kernel (mixed)", mflops, mst["device_ms"], "mixed"),
                 "vs_fp64": (n * M / (mms / 1e3)) / value,
                 "rel_l2_gap_to_fp64_by_level": gaps,
                 "max_gap_levels_1_8": max(gaps[j] for j in levels if j <= 8),
                 "max_gap": max(gaps.values()),
                 "l2_error_vs_exact_at_T": merr,
                 "refinement_steps": int(mst["outer_iterations"]),
                 "escalated_levels": int(mst["escalated_levels"]),
                 "floor_levels": int(mst["floor_levels"]),
                 "cgs_iterations": int(mst["total_iterations"]),
                 "setup_ms": msetup,
                 "dtype": "f32 / float-float inner, f64 refinement, history and weights"}
        sm.close()
    s.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    clocks = clk.summary()
    traffic, tsrc = captured_traffic(args.traffic_profile) if lpl == 64 else (None, "launch shape differs from the capture")
    rl = roofline("level_kernel", flops / launches_per_step, kernel_ms / launches_per_step, args.precision)
    rl["fp64_fma_measured_tflops"] = fp64_measured
    rl["traffic"] = traffic
    rl["traffic_source"] = tsrc
    rl["per"] = f"launch ({lpl or M} levels; {launches_per_step:.0f} launches per march)"
    line = {
        "metric": "grid-point updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32 inner / f64 refinement",
        "data": "synthetic (manufactured solution u=(t^2+1)x^2(1-x)^2, analytic source)",
        "config": {**describe(p), "parallelism": f"replicas{world}", "fft_plan": plan,
                   "levels_per_launch": lpl,
                   "l2": "inputs larger than L2 (history ring %.0f MB, work arrays %.0f MB)"
                         % (M * n * 8 / 1e6, 24 * n * 8 / 1e6)},
        "e2e": {"value": e2e_val, "unit": "updates/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n, "marches": 1},
        "gpu_launches": launches,
        "setup_ms": setup_ms,
        "roofline": rl,
        "history_roofline": hist,
        "cgs_iterations": {"mean": float(it.mean()), "min": int(it.min()), "max": int(it.max()),
                           "levels_at_maxit": int((it >= args.maxit).sum())},
        "max_level_residual": float(res.max()),
        "refinement": ({"outer_steps": int(sum(st["outer_iterations"] for st in stats)) // max(1, args.steps),
                        "escalated_levels": int(sum(st["escalated_levels"] for st in stats)) // max(1, args.steps)}
                       if args.precision == "mixed" else None),
        "l2_error_vs_exact_at_T": err,
        "mixed": mixed,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_line(p, args.cpu_budget)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline_line(p, budget_s):
    """The oracle timed on a bounded sample (the workload's parameters at n = 2047), reported at
    the workload's n by the dense-LU law: elimination costs 2/3 n^3 flops per level, so updates/s
    scale as n^-2.  The measured sample is kept beside it."""
    v, d, cores, dt, n_s, levels = oracle_sample(p, budget_s=budget_s)
    scale = (n_s / p.n) ** 2
    return {"value": v * scale, "unit": "updates/s", "cores": cores, "kind": "oracle",
            "sample": d, "extrapolated": p.n != n_s,
            "law": "dense LU per level: 2/3 n^3 flop, so updates/s ~ n^-2",
            "measured_sample": {"n": n_s, "levels": levels, "seconds": dt, "value": v},
            "single_core": oracle_single_core(p)}


def run_native_batch(args, probs_all):
    """Batched workload: every instance marched through all M levels per step.  With several
    ranks each marches a cost-balanced shard of the instances (no collective on the data path);
    the step time is the slowest rank's."""
    import torch
    ranks = Ranks().init()
    from paper_1603_00279_gb300 import build
    if ranks.rank == 0 or ranks.world == 1:
        build.build()
    ranks.barrier()
    import paper_1603_00279_gb300 as P
    probs = shard_instances(probs_all, ranks)
    ntot_all = sum(p.n for p in probs_all)
    M = probs[0].M
    precond = args.precond or "strang"
    stream = torch.cuda.Stream()
    const = args.algorithm == "ids-const"
    t_setup = time.perf_counter()
    b = P.Batch(probs, M, preconditioner=precond, precision=args.precision,
                maxit=args.maxit, stream=stream.cuda_stream, algorithm=args.algorithm,
                autotune=not args.no_autotune)
    setup_ms = 1e3 * (time.perf_counter() - t_setup)
    batch_plan = b.plan()
    ntot = sum(p.n for p in probs)

    def one_step():
        b.reset()
        return b.step(M)

    for _ in range(args.warmup):
        one_step()
    stats = []
    ranks.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(ranks.local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(one_step())
        e1.record(stream)
        torch.cuda.synchronize()
    ranks.barrier()
    ms = ranks.max(e0.elapsed_time(e1))
    value = ntot_all * M * args.steps / (ms / 1e3)
    kernel_ms = float(np.mean([st["device_ms"] for st in stats]))
    flops = 0.0
    its_all = []
    apps_per_level = (stats[-1]["outer_iterations"] / max(1, stats[-1]["gsf_levels"])) if const else 0.0
    for i, p in enumerate(probs):
        it, _ = b.history(i, M)
        its_all.append(it)
        if const:
            flops += _alg_flops_const(p.n, M, precond, it, apps_per_level * (M - 1))
        else:
            flops += _alg_flops(p.n, M, precond, it, 2)
    its_all = np.concatenate(its_all)
    # end to end: H2D of every u^0, march, D2H of every u^M through the C ABI
    b.reset()
    u0 = torch.from_numpy(np.concatenate([b.get_level(i, 0)[0] for i in range(len(probs))])).pin_memory()
    uM = torch.empty(ntot, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.set_initial(u0.data_ptr())
    b.step(M)
    b.get_all(uM.data_ptr())
    e2e_s = ranks.max(time.perf_counter() - t0)
    b.close()
    single = None
    if ranks.world == 1 and args.single_sample > 0:
        # the plain alternative to batching: the first instances (an i.i.d. sample of the
        # workload) marched one at a time through the single-instance ABI, same precision and
        # algorithm, device time of the marches
        sample = probs[:args.single_sample]
        ms_one = 0.0
        for q in sample:
            with P.Solver.from_problem(q, source="callback", preconditioner=precond,
                                       precision=args.precision, maxit=args.maxit,
                                       algorithm=args.algorithm, stream=stream.cuda_stream,
                                       autotune=not args.no_autotune) as s1:
                ms_one += s1.step(M)["device_ms"]
        one = sum(q.n for q in sample) * M / (ms_one / 1e3)
        single = {"instances": len(sample), "one_at_a_time_updates_per_s": one,
                  "batched_over_one_at_a_time": ntot_all * M * args.steps / (ms / 1e3) / one}
    if ranks.rank != 0:
        return
    ns = np.array([p.n for p in probs_all])
    line = {
        "metric": "grid-point updates/s", "value": value, "unit": "updates/s", "n_gpus": ranks.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "strong" if ranks.world > 1 else "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32 inner / f64 refinement",
        "data": "synthetic (seeded instances, sine-mode initial values, f = 0)",
        "config": {"workload": "tsfcde_batch", "instances": len(probs_all), "M": M,
                   "n_min": int(ns.min()), "n_max": int(ns.max()), "sum_n": int(ntot_all),
                   "preconditioner": precond, "tol": 1e-12,
                   "parallelism": (f"instance shards over {ranks.world} ranks (cost-balanced)"
                                   if ranks.world > 1 else "replicas1"),
                   "algorithm": ("IDS with constant coefficients (Gohberg-Semencul, levels >= 1)"
                                 if const else "IDS (PCGS every level)"),
                   "launch_plan": batch_plan,
                   "updates_per_step": int(ntot_all * M),
                   "l2": "inputs larger than L2 (history %.1f GB)" % (ntot_all * M * 8 / 1e9)},
        "e2e": {"value": ntot_all * M / e2e_s, "unit": "updates/s",
                "h2d_bytes_per_step": 8 * int(ntot_all), "d2h_bytes_per_step": 8 * int(ntot_all)},
        "gpu_launches": int(sum(st["device_launches"] for st in stats)),
        "setup_ms": setup_ms,
        "roofline": roofline("batch_level_kernel", flops, kernel_ms, args.precision),
        "cgs_iterations": {"mean": float(its_all.mean()), "min": int(its_all.min()),
                           "max": int(its_all.max()),
                           "levels_at_maxit": int((its_all >= args.maxit).sum())},
        "max_level_residual": float(max(st["max_residual"] for st in stats)),
        "refinement": ({"outer_steps": int(stats[-1]["outer_iterations"]),
                        "escalated_levels": int(stats[-1]["escalated_levels"])}
                       if args.precision == "mixed" and not const else None),
        "gohberg_semencul": ({"levels": int(stats[-1]["gsf_levels"]),
                              "applications_per_level": apps_per_level,
                              "note": "cgs_iterations include the two generator solves at level 1"}
                             if const else None),
        "single_instance_sample": single,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        import oracle as O
        t0 = time.perf_counter()
        upd = 0
        k = 0
        while time.perf_counter() - t0 < args.cpu_budget and k < len(probs):
            q = probs[k]
            lv = max(1, min(M, 8))
            O.run(q, levels=lv)
            upd += q.n * lv
            k += 1
        dt = time.perf_counter() - t0
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        line["cpu_baseline"] = {"value": upd / dt, "unit": "updates/s", "cores": cores, "kind": "oracle",
                                "sample": f"oracle (dense LU per level) on the first {k} instances "
                                          f"of the batch, levels 0..7 each, {dt:.1f} s"}
    print(json.dumps(line))


def run_native_history(args, probs):
    """History-dominated workload: instances of n = 2^18-1, M = 8192 (each holds a 17 GB FP64
    history ring, plus 34 GB of block spectra with fast history), FP64 history accumulation, the
    given precision for the solves.  The instances are set up in groups that fit the device's free
    memory; each group is warmed up and its timed marches are added to the step time (setup is
    outside the timed region).  One step marches every instance once."""
    import torch
    ranks = Ranks().init()
    from paper_1603_00279_gb300 import build
    if ranks.rank == 0 or ranks.world == 1:
        build.build()
    ranks.barrier()
    import paper_1603_00279_gb300 as P
    stream = torch.cuda.Stream()
    probs_all = probs
    probs = shard_instances(probs_all, ranks)
    ntot = sum(q.n * q.M for q in probs_all)
    fast = args.fast_history != "off"
    q0 = probs[0]
    stride = (q0.n + 31) // 32 * 32
    per_inst = 8 * stride * q0.M + 40 * 8 * 2 * stride
    if fast:
        per_inst += 16 * 129 * ((q0.M - 1) // 128) * stride + 8 * 128 * stride
    free = torch.cuda.mem_get_info()[0]
    G = max(1, min(len(probs), int(0.85 * free // per_inst)))
    groups = [list(range(i, min(len(probs), i + G))) for i in range(0, len(probs), G)]

    def make(q):
        return P.Solver.from_problem(q, source="separable", stream=stream.cuda_stream,
                                     precision=args.precision, maxit=args.maxit,
                                     fast_history=fast, autotune=not args.no_autotune)

    ms_total = 0.0
    stats = []           # per timed step: the stats of every instance
    errs = [None] * len(probs)
    launches = 0
    hist = e2e = None
    flops = 0.0
    kernel_ms = 0.0
    samples = []
    for gi, grp in enumerate(groups):
        ctxs = [make(probs[i]) for i in grp]
        for _ in range(args.warmup):
            for i, s in zip(grp, ctxs):
                s.reset()
                s.step(probs[i].M)
        ranks.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(ranks.local) as clk:
            e0.record(stream)
            gstats = []
            for _ in range(args.steps):
                row = []
                for i, s in zip(grp, ctxs):
                    s.reset()
                    row.append(s.step(probs[i].M))
                gstats.append(row)
            e1.record(stream)
            torch.cuda.synchronize()
        ms_total += e0.elapsed_time(e1)
        samples += clk.lines if hasattr(clk, "lines") else []
        stats.append(gstats)
        launches += int(sum(st["device_launches"] for row in gstats for st in row))
        for i, s in zip(grp, ctxs):
            q = probs[i]
            u, _ = s.get_level(q.M)
            errs[i] = float(np.sqrt(q.h) * np.linalg.norm(u - q.exact(q.grid(), q.T)))
            it_q, _ = s.history(q.M)
            flops += algorithmic_flops(q, it_q, 2)
            if fast:   # the history as the fast history computes it, not as the direct sum
                flops += _fast_history_flops(q.n, q.M) - 2.0 * q.n * (q.M * (q.M - 1) / 2.0)
        for row in gstats[-1:]:
            for i, st in zip(grp, row):
                kernel_ms += st["device_ms"]
                if args.precision == "mixed":
                    L = max(8, 1 << math.ceil(math.log2(2 * probs[i].n)))
                    flops += st["outer_iterations"] * (5.0 * L * math.log2(L) + 3.0 * L)
        if gi == 0:
            # history phase at the last level of the first instance (its method: fast or direct)
            s0 = ctxs[0]
            jh = q0.M - 1
            s0.history_sum(jh, want=False)
            h0 = torch.cuda.Event(enable_timing=True)
            h1 = torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            for _ in range(3):
                s0.history_sum(jh, want=False)
            h1.record(stream)
            torch.cuda.synchronize()
            hms = h0.elapsed_time(h1) / 3
            hd0 = torch.cuda.Event(enable_timing=True)
            hd1 = torch.cuda.Event(enable_timing=True)
            hd0.record(stream)
            s0.history_sum(jh, want=False, direct=True)
            hd1.record(stream)
            torch.cuda.synchronize()
            hdms = hd0.elapsed_time(hd1)
            hbytes = 8.0 * q0.n * jh + 16.0 * q0.n
            peak = hbm_peak()
            hist = {"kernel": "history phase (level M-1), direct sum", "bound": "hbm",
                    "achieved": hbytes / (hdms / 1e3) / 1e9, "peak": peak[0], "unit": "GB/s",
                    "frac": hbytes / (hdms / 1e3) / 1e9 / peak[0], "ms": hdms,
                    "fp64_tflops": 2.0 * q0.n * jh / (hdms / 1e3) / 1e12,
                    "fast_history_ms": hms if fast else None, "peak_source": peak[1]}
            # end to end through the C ABI for this group: H2D of u^0, march, D2H of u^M
            u0s = [torch.from_numpy(s.get_level(0)[0]).pin_memory() for s in ctxs]
            uMs = [torch.empty(probs[i].n, dtype=torch.float64).pin_memory() for i in grp]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s, a_, b_ in zip(ctxs, u0s, uMs):
                s.reset(u0_ptr=a_.data_ptr())
                s.solve(out_ptr=b_.data_ptr())
            torch.cuda.synchronize()
            e2e_s = time.perf_counter() - t0
            nsum = sum(probs[i].n * probs[i].M for i in grp)
            e2e = {"value": nsum / e2e_s, "unit": "updates/s",
                   "h2d_bytes_per_step": 8 * sum(probs[i].n for i in grp),
                   "d2h_bytes_per_step": 8 * sum(probs[i].n for i in grp),
                   "instances": len(grp), "note": "first memory group of instances"}
        for s in ctxs:
            s.close()
        del ctxs
    ms = ranks.max(ms_total)
    clk.lines = samples            # clocks over every group's timed region
    co = None
    if args.co:
        # the order of the scheme, from FP64 marches (tol 1e-12): the mixed march's FP64 residual
        # floor 64 u64 kappa_eff is within a factor of a few of the error at T on this workload
        def err_fp64(q):
            with P.Solver.from_problem(q, source="separable", stream=stream.cuda_stream,
                                       precision="fp64", maxit=args.maxit, fast_history=fast,
                                       autotune=not args.no_autotune) as sf:
                uq = sf.solve()
            return float(np.sqrt(q.h) * np.linalg.norm(uq - q.exact(q.grid(), q.T)))
        half, quarter = W.config_history()[0], W.config_history()[0]
        half.M, quarter.M = q0.M // 2, q0.M // 4
        e_full, e_half, e_q = err_fp64(W.config_history()[0]), err_fp64(half), err_fp64(quarter)
        co = {"E_M/4": e_q, "E_M/2": e_half, "E_M": e_full,
              "CO_tau_3level": math.log2((e_q - e_half) / (e_half - e_full)),
              "CO_tau": math.log2(e_half / e_full), "CO_tau_M4_M2": math.log2(e_q / e_half),
              "precision": "fp64",
              "note": "E = C tau^2 + E_inf; the three-level order cancels E_inf (h^2 term and FP64 "
                      "rounding, about a third of C tau^2 at M)"}
    if ranks.rank != 0:
        return
    its = [st["total_iterations"] / max(1, st["levels_advanced"])
           for g in stats for row in g for st in row]
    line = {"metric": "grid-point updates/s", "value": ntot * args.steps / (ms / 1e3),
            "unit": "updates/s", "n_gpus": ranks.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if ranks.world > 1 else "weak",
            "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32/ff inner / f64 refinement, f64 history",
            "data": "synthetic (manufactured solution)",
            "config": {"workload": "tsfcde_history", "instances": len(probs_all), "n": q0.n,
                       "M": q0.M, "alpha_beta": [[q.alpha, q.beta] for q in probs_all],
                       "history_bytes_per_instance": 8 * q0.n * q0.M,
                       "fast_history": fast, "memory_groups": [len(g) for g in groups],
                       "history_flops": ("blocked FFT convolution in time, as computed" if fast
                                         else "direct sum (2 j n per level)"),
                       "l2": "inputs larger than L2 (history ring %.0f GB per instance)" % (8 * q0.n * q0.M / 1e9)},
            "history_roofline": hist,
            "e2e": e2e,
            "gpu_launches": launches,
            "roofline": roofline("level_kernel", flops, kernel_ms, args.precision),
            "cgs_iterations_mean": float(np.mean(its)), "l2_error_vs_exact_at_T": errs,
            "convergence_order": co, "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(probs[0], args.cpu_budget)
    print(json.dumps(line))


def profile_run(args, p):
    """One march (or --levels levels) of the workload in the launch shape the benchmark times, and
    nothing else: the command the committed ncu summaries under profiles/ were captured with."""
    import paper_1603_00279_gb300 as P
    from paper_1603_00279_gb300 import build
    build.build()
    if isinstance(p, list):
        b = P.Batch(p, p[0].M, preconditioner=args.precond or "strang", precision=args.precision,
                    maxit=args.maxit, algorithm=args.algorithm, autotune=not args.no_autotune)
        st = b.step(p[0].M)
        b.close()
    else:
        s = P.Solver.from_problem(p, source="separable", maxit=args.maxit, precision=args.precision,
                                  autotune=not args.no_autotune,
                                  levels_per_launch=args.levels_per_launch,
                                  fast_history=args.fast_history == "on")
        st = s.step(p.M)
        if args.profile_history and p.M >= 2:
            for _ in range(3):   # the history phase of the last level, direct sum, alone
                s.history_sum(p.M - 1, want=False, direct=True)
        s.close()
    print(json.dumps({"profile_run": True, "levels": st["levels_advanced"],
                      "device_ms": st["device_ms"], "launches": st["device_launches"],
                      "cgs_iterations": st["total_iterations"]}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="precision",
                    help="precision (default: n = 2^20-1, M = 512, FP64 with a mixed leg), large, "
                         "small, mixed (precision workload in mixed precision), batch, history")
    ap.add_argument("--precond", default=None, choices=[None, "strang", "tchan", "none"])
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "mixed"],
                    help="default: fp64, or mixed for the mixed and history workloads")
    ap.add_argument("--levels", type=int, default=None, help="override M (exploration only)")
    ap.add_argument("--maxit", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=8.0,
                    help="--impl reference: seconds of oracle work per step")
    ap.add_argument("--levels-per-launch", type=int, default=64,
                    help="levels per device launch of the single-instance march (0: one launch)")
    ap.add_argument("--traffic-profile", default="level_kernel_precision_n1048575_dram.md",
                    help="profiles/ summary holding the dominant kernel's DRAM bytes per launch")
    ap.add_argument("--no-mixed-leg", dest="mixed_leg", action="store_false",
                    help="precision workload: skip the mixed-precision march and its gap")
    ap.add_argument("--fast-history", default="auto", choices=["auto", "on", "off"],
                    help="history sum as a blocked FFT convolution in time (auto: on for the "
                         "history workload only)")
    ap.add_argument("--profile-history", action="store_true",
                    help="--profile-run: then run the history phase of level M-1 three times")
    ap.add_argument("--profile-run", action="store_true",
                    help="set up and march once in the timed launch shape, print a short line, "
                         "exit (the command behind the ncu summaries in profiles/)")
    ap.add_argument("--instances", type=int, default=None,
                    help="batch workload: instance count (4096); history workload: how many of "
                         "its 16 instances to march (1)")
    ap.add_argument("--no-autotune", action="store_true", help="skip the setup-time FFT-plan tuner")
    ap.add_argument("--algorithm", default="ids", choices=["ids", "ids-const"],
                    help="batch workload: ids-const = constant-coefficient algorithm (Gohberg-Semencul)")
    ap.add_argument("--co", action="store_true",
                    help="history workload: also march M/2 and M/4 levels for CO_tau")
    ap.add_argument("--single-sample", type=int, default=32,
                    help="batch workload: also march this many of its instances one at a time "
                         "through the single-instance ABI (0: skip)")
    args = ap.parse_args()
    global _ARGS
    _ARGS = args
    p = workload(args.workload, args.precond)
    if args.precision is None:
        args.precision = "mixed" if args.workload in ("mixed", "history") else "fp64"
    if args.levels and args.workload not in ("batch", "history"):
        p.M = args.levels
    if args.levels and args.workload == "history":
        for q in p:
            q.M = args.levels
    if args.fast_history == "auto":
        args.fast_history = "on" if args.workload == "history" else "off"
    if args.profile_run:
        if args.workload == "batch" and args.levels:
            for q in p:
                q.M = args.levels
        profile_run(args, p if args.workload != "history" else p[0])
        return
    if args.workload == "history":
        if args.impl == "reference":
            run_reference(args, p[0])
        else:
            run_native_history(args, p)
        return
    if args.workload == "batch":
        if args.levels:
            for q in p:
                q.M = args.levels
        if args.impl == "reference":
            run_reference_batch(args, p)
        else:
            run_native_batch(args, p)
        return
    if args.impl == "reference":
        run_reference(args, p)
    else:
        run_native(args, p)


if __name__ == "__main__":
    main()
