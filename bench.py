#!/usr/bin/env python
"""Benchmark: population evaluation throughput in GPop/s (program nodes x
fitness cases per second / 1e9) on one GB300.

Workload (default): the paper-shaped single problem -- 4,096 postfix programs
of length 8..128 over 10 variables, 100,000 fitness cases X ~ U(1, 10), target
from a random program plus 1% Gaussian noise.  One step = one generation of
the device-resident hot path: both fitness kinds (MSE and 1 - r^2) from one
interpreter pass, a 4-way tournament on 1 - r^2, then crossover and mutation
into the second population buffer.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Under torchrun each rank runs its own replica
of the workload on its GPU (weak scaling, no data-path collective); timing is
the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GPop/s (nodes x cases / s) at 1 GB300 vs plain eval; % of FP32 issue peak"
L2_BYTES = 129 * 1024 * 1024
CSRC = os.path.join(ROOT, "paper_2603_12292_gb300", "csrc")
# The CUDA sources each dominant kernel is built from: an ncu figure below is
# reported only while these files hash to what they were when it was captured.
KERNEL_SOURCES = {
    "eval": ("sr_eval.cu", "sr_interp.cuh", "sr_common.cuh"),
    "grad": ("sr_grad.cu", "sr_interp.cuh", "sr_common.cuh"),
}
# Dominant kernels of the workloads, each from one ncu --set full capture
# summarised under profiles/: the captured workload, DRAM bytes (read +
# write) of the captured launch, the units (node-evaluations) it processed,
# smsp__issue_active, the summary file, and the hash of the kernel's sources
# (source_hash) when it was taken.  Traffic is reported for the captured
# workload, and for another size only where it grows with the units (scale).
KERNEL_NCU = {
    # eval_kernel<MODE_BOTH> on the headline workload, inputs read once
    "paper": {"workload": "paper-4096x100k", "dram_bytes": 173.062e6 + 11.567e6, "units": None,
              "issue_active": 0.839, "scale": False, "sources": "eval",
              "capture": "profiles/eval_kernel_paper-4096x100k.md", "src": "a0bec70a9304581f"},
    # grad_kernel: the tape write-back evicted from L2 grows with the units
    "grad": {"workload": "adjoint-2048x131072", "dram_bytes": 4.489e9 + 18.163e9, "units": 1.3324e10,
             "issue_active": 0.726, "scale": True, "sources": "grad",
             "capture": "profiles/grad_kernel_adjoint-2048x131072.md", "src": "9914c98e792aff67"},
    # eval_kernel<R4>: inputs read once (L2-resident), at the full size
    "beagle": {"workload": "beagle-4096x100k", "dram_bytes": 171.088e6 + 11.973e6, "units": 2.3977e10,
               "issue_active": 0.817, "scale": False, "sources": "eval",
               "capture": "profiles/eval_kernel_r4_beagle-4096x100k.md", "src": "a0bec70a9304581f"},
    # eval_batched_kernel: the first 8 problems; inputs read once
    "batched": {"workload": "batched-8", "dram_bytes": 1625.761e6 + 47.885e6, "units": 4.0723e11,
                "issue_active": 0.816, "scale": False, "sources": "eval",
                "capture": "profiles/eval_batched_kernel_batched-8.md", "src": "a0bec70a9304581f"},
    # eval_kernel<CORR> at Lmax 256: inputs read once
    "large": {"workload": "large-16384x131072", "dram_bytes": 402.477e6 + 20.297e6, "units": 2.5087e11,
              "issue_active": 0.820, "scale": False, "sources": "eval",
              "capture": "profiles/eval_kernel_corr_large-16384x131072.md", "src": "a0bec70a9304581f"},
}


def source_hash(kind: str) -> str:
    """SHA-256 (first 16 hex digits) of the CUDA sources a kernel is built from."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def ncu_record(key: str):
    """The capture of a kernel if it still describes the current sources, and
    its provenance either way: (record or None, provenance dict)."""
    cap = KERNEL_NCU.get(key)
    if cap is None:
        return None, None
    now = source_hash(cap["sources"])
    prov = {"capture": cap["capture"], "src_at_capture": cap["src"], "src_now": now}
    if cap["src"] != now:
        prov["stale"] = ("no capture of the current kernel source" if cap["src"] is None
                         else "the kernel source changed since the capture")
        return None, prov
    return cap, prov


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ops", default="base", choices=["base", "table1"],
                    help="operator set of the paper / beagle populations: base (+ - * / sin cos exp log "
                         "sqrt sq) or table1 (adds 1/x tan asin acos atan tanh, Table 1)")
    ap.add_argument("--selection", default="tournament", choices=["tournament", "microcosm"],
                    help="parent selection of the paper / large workloads: k = 4 tournament, or the "
                         "paper's Monte-Carlo microcosm selection (Sec. 2.1.6: sample 100, keep 0.5)")
    ap.add_argument("--schedule", action="store_true",
                    help="large workload: shrink the population 262,144 -> 131,072 -> 65,536 every two "
                         "generations (the paper's variable population size, Sec. 2.1.7; needs microcosm)")
    ap.add_argument("--small", action="store_true",
                    help="reduced sizes of the adjoint / large / batched workloads (2,048 x 131,072; "
                         "16,384 x 131,072; the first 8 problems), for profiler captures")
    ap.add_argument("--workload", default="paper",
                    choices=["paper", "batched", "adjoint", "large", "plain", "beagle", "opmix"],
                    help="paper (default, the headline): 4096 x 100k; batched: 64 problems in one launch "
                         "vs a loop of single calls; adjoint: Adam constant optimisation; large: "
                         "262,144 x 1M; plain: 256 x 1k, CUDA graph vs eager; beagle: 4096 x 100k with "
                         "1%% invalid targets, the r^4 score of Eq. 2 (and Eq. 3 timed beside it); opmix: the "
                         "paper-shaped population drawn from one operator class at a time")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def host_cores() -> int:
    """Host cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return
        # the timed region starts once the sampler is live (nvidia-smi takes a
        # moment to start), so that its samples fall inside the region
        t0 = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t0 < 3.0:
            time.sleep(0.01)
        self.first = len(self.lines)  # samples from here on fall inside the region

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = self.lines[self.first:]
        for line in inside or self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args, rank, world):
    import oracle
    from paper_2603_12292_gb300 import inputs
    if rank != 0:
        return 0
    for attempt in range(20):  # the same usable-target rule as our arm
        pr = inputs.paper_shaped(attempt=attempt, unary_ops=12 if args.ops == "table1" else 6)
        y64 = oracle.predict(pr.target, pr.target_consts, pr.X, pr.N)
        if np.all(np.isfinite(y64)) and np.abs(y64).max() < 1e15 and np.std(y64) > 1e-6 * (1 + np.abs(y64).max()):
            break
    y = inputs.add_noise(np.random.default_rng(pr.seed + 7), y64, pr.noise)
    # every host core, named explicitly: torchrun sets OMP_NUM_THREADS=1 for its ranks
    cores = host_cores()
    # size each step to ~4 s of CPU work: programs sampled from the population, all cases
    t0 = time.perf_counter()
    oracle.evaluate(pr.programs[:16], pr.lengths[:16], pr.consts[:16], pr.X, y, oracle.CORR, pr.N, nthreads=cores)
    oracle.evaluate(pr.programs[:16], pr.lengths[:16], pr.consts[:16], pr.X, y, oracle.MSE, pr.N, nthreads=cores)
    dt16 = max(time.perf_counter() - t0, 1e-3)
    S = int(min(pr.P, max(16, 16 * 4.0 / dt16)))
    rng = np.random.default_rng(1)
    times, units = [], 0.0
    for step in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(pr.P, S, replace=False))
        t0 = time.perf_counter()
        oracle.evaluate(pr.programs[idx], pr.lengths[idx], pr.consts[idx], pr.X, y, oracle.MSE, pr.N, nthreads=cores)
        oracle.evaluate(pr.programs[idx], pr.lengths[idx], pr.consts[idx], pr.X, y, oracle.CORR, pr.N, nthreads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            units += float(pr.lengths[idx].astype(np.int64).sum()) * pr.N
    total = sum(times)
    value = units / total / 1e9
    sample = f"{S} sampled programs x {pr.N} cases per step, MSE and 1-r^2 (two oracle passes)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GPop/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": pr.name, "programs": pr.P, "cases": pr.N, "vars": pr.nvars,
                       "lengths": "8-128", "fitness": "MSE and 1-r^2"},
            "cpu_baseline": {"value": value, "unit": "GPop/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GPop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2603_12292_gb300 import binding, inputs, shard

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ctx = binding.Context(local_rank)
    stream = torch.cuda.current_stream(dev)

    nun = 12 if args.ops == "table1" else 6
    # the target on the device with the library's own predict, then 1% noise (host, FP64)
    pr, programs, lengths, consts, X, y = _device_problem(
        lambda a: inputs.paper_shaped(attempt=a, unary_ops=nun), dev, binding, ctx)
    binding.sr_reserve(ctx, pr.P, pr.Lmax, pr.N)
    fitness = torch.empty((2, pr.P), dtype=torch.float64, device=dev)
    parents = torch.empty((pr.P, 2), dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    cfg = binding.var_cfg(unary_ops=nun)  # p_cross 0.9, p_point 0.1, p_subtree 0.05, p_const 0.1
    pop = [(programs, lengths, consts),
           (torch.empty_like(programs), torch.empty_like(lengths), torch.empty_like(consts))]
    SEED, K_TOURN = 20260312 + rank, 4  # each rank evolves its own population (an island)
    state = {"gen": 0, "cur": 0}
    ev_eval = []

    def select(f, g):
        if args.selection == "microcosm":
            binding.sr_select_microcosm(ctx, f, pr.P, 100, 0.5, SEED, g, parents=parents)
        else:
            binding.sr_select_tournament(ctx, f, K_TOURN, SEED, g, parents=parents)

    def generation(record_eval=False):
        """One generation: both fitness kinds from one pass, tournament on 1 - r^2, variation."""
        g, cur = state["gen"], state["cur"]
        P_, L_, C_ = pop[cur]
        if record_eval:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        binding.sr_eval(ctx, P_, L_, C_, X, y, pr.N, binding.SR_MSE_CORR, fitness=fitness)
        if record_eval:
            e1.record(stream)
            ev_eval.append((e0, e1))
        select(fitness[1], g)
        binding.sr_vary(ctx, P_, L_, C_, parents, pr.nvars, cfg, SEED, g, out=pop[1 - cur])
        state["gen"], state["cur"] = g + 1, 1 - cur
        return L_

    for _ in range(args.warmup):
        generation()
    torch.cuda.synchronize()
    # the population the timed generations start from: the end-to-end leg
    # below runs the same generations again from it
    start_rows = tuple(t.clone() for t in pop[state["cur"]])
    start_gen = state["gen"]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    nodes = []
    sampler = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = binding.sr_kernel_launches(ctx)
    for i in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        lens_evaluated = generation(record_eval=True)
        ev[i][1].record(stream)
        nodes.append(int(lens_evaluated.sum().item()))  # outside the events
    torch.cuda.synchronize()
    launches = binding.sr_kernel_launches(ctx) - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    eval_ms = [a.elapsed_time(b) for a, b in ev_eval]
    total_ms = float(sum(step_ms))
    units = float(sum(nodes)) * pr.N
    if world > 1:
        total_ms = shard.max_over_ranks(total_ms, dev)
        units = shard.sum_over_ranks(units, dev)
    value = units / (total_ms / 1e3) / 1e9

    # roofline of the dominant kernel (the evaluation call, timed by its own
    # events inside the timed region): FP32 issue bound, one lane-op per node-case
    pk, src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * sm_max * 1e6 / 1e9  # G lane-ops/s
    achieved = float(np.mean([n * pr.N / (ms / 1e3) / 1e9 for n, ms in zip(nodes, eval_ms)]))
    # DRAM bytes per launch and issue-slot use of this kernel: one ncu capture
    # of the same command (profiles/eval_kernel_paper-4096x100k.md)
    cap, prov = ncu_record("paper")
    if args.ops != "base":
        cap = None  # the capture is of the base operator set
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GPop/s",
                "frac": achieved / peak, "traffic": cap["dram_bytes"] if cap else None,
                "kernel": "eval_kernel (sr_eval SR_MSE_CORR)",
                "eval_ms": float(np.mean(eval_ms)),
                "issue_active_ncu": cap["issue_active"] if cap else None, "ncu_provenance": prov,
                "peak_source": f"{sms} SMs x 128 FP32 lanes x {sm_max:.0f} MHz ({src} max clock)"}

    # the evaluation alone on the first timed population, with and without the
    # decoder's variable transforms (outside the timed region, no L2 flush):
    # what the table saves, and that the fitness is the same bits either way
    def eval_rate(mode, reps=5):
        binding.sr_set_transforms(ctx, mode)
        try:
            P_, L_, C_ = start_rows
            f = torch.empty_like(fitness)
            binding.sr_eval(ctx, P_, L_, C_, X, y, pr.N, binding.SR_MSE_CORR, fitness=f)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                binding.sr_eval(ctx, P_, L_, C_, X, y, pr.N, binding.SR_MSE_CORR, fitness=f)
            e1.record(stream)
            torch.cuda.synchronize()
            return float(L_.sum().item()) * pr.N * reps / (e0.elapsed_time(e1) / 1e3) / 1e9, f
        finally:
            binding.sr_set_transforms(ctx, binding.XFORM_AUTO)

    g_on, f_on = eval_rate(binding.XFORM_AUTO)
    g_off, f_off = eval_rate(binding.XFORM_NEVER)
    transforms = {"population": f"generation {start_gen} (the first timed one), sr_eval(SR_MSE_CORR) x5",
                  "eval_gpops": g_on, "eval_gpops_without": g_off,
                  "fitness_bit_identical": bool(torch.equal(f_on.view(torch.int64), f_off.view(torch.int64)))}

    # end to end through the public API with the population held on the host:
    # H2D population, evaluate + select + vary, D2H children and fitness; the
    # same generations as the timed region (same populations, same work)
    P_, L_, C_ = start_rows
    h_prog = P_.cpu().pin_memory()
    h_len = L_.cpu().pin_memory()
    h_con = C_.cpu().pin_memory()
    h_fit = torch.empty((2, pr.P), dtype=torch.float64).pin_memory()
    d_in = (torch.empty_like(programs), torch.empty_like(lengths), torch.empty_like(consts))
    d_out = (torch.empty_like(programs), torch.empty_like(lengths), torch.empty_like(consts))
    h2d = h_prog.numel() + h_len.numel() * 4 + h_con.numel() * 4
    d2h = h2d + h_fit.numel() * 8
    e2e_nodes = []

    def e2e_step(g):
        d_in[0].copy_(h_prog, non_blocking=True)
        d_in[1].copy_(h_len, non_blocking=True)
        d_in[2].copy_(h_con, non_blocking=True)
        binding.sr_eval(ctx, d_in[0], d_in[1], d_in[2], X, y, pr.N, binding.SR_MSE_CORR, fitness=fitness)
        select(fitness[1], g)
        binding.sr_vary(ctx, d_in[0], d_in[1], d_in[2], parents, pr.nvars, cfg, SEED, g, out=d_out)
        h_prog.copy_(d_out[0], non_blocking=True)
        h_len.copy_(d_out[1], non_blocking=True)
        h_con.copy_(d_out[2], non_blocking=True)
        h_fit.copy_(fitness, non_blocking=True)

    for _ in range(2):  # warm the copies, then start again from the same rows
        e2e_step(start_gen)
    torch.cuda.synchronize()
    h_prog.copy_(P_)
    h_len.copy_(L_)
    h_con.copy_(C_)
    e2e_ms = []
    for i in range(args.steps):
        n_in = int(h_len.sum())
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step(start_gen + i)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
        e2e_nodes.append(n_in)
    if e2e_nodes != nodes:
        raise RuntimeError("the end-to-end generations did not repeat the timed ones")
    e2e_units, e2e_total = float(sum(e2e_nodes)) * pr.N, float(sum(e2e_ms))
    if world > 1:
        e2e_total = shard.max_over_ranks(e2e_total, dev)
        e2e_units = shard.sum_over_ranks(e2e_units, dev)
    e2e_val = e2e_units / (e2e_total / 1e3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": "GPop/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": pr.name, "programs": pr.P, "cases": pr.N, "vars": pr.nvars,
                       "lengths": "8-128", "fitness": "MSE and 1-r^2 from one pass",
                       "step": "one generation: sr_eval(SR_MSE_CORR) + "
                               + ("sr_select_microcosm(sample 100, keep 0.5, on 1-r^2)" if args.selection == "microcosm"
                                  else "sr_select_tournament(k=4, on 1-r^2)")
                               + " + sr_vary(p_cross 0.9, p_point 0.1, p_subtree 0.05, p_const 0.1)",
                       "l2": "flushed between timed steps",
                       "decoder": "constant-only subtrees folded; u(x_j) read from a per-call table of "
                                  "the variables' unary transforms; outputs bit for bit those of "
                                  "node-by-node evaluation; GPop/s counts every node as written",
                       "parallelism": f"islands x{world}: one population per rank, own seed, no exchange"},
            "roofline": roofline, "clocks": clocks,
            "e2e": {"value": e2e_val, "unit": "GPop/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches), "decoder_transforms": transforms}

    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pr, y.cpu().numpy())
        line["parity"] = parity_leg(pr, y, X, pop[state["cur"]], ctx, binding, cfg, nun, SEED, state["gen"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def cpu_baseline(pr, y):
    """The oracle as it stands on all host cores, on a bounded sample (~10-20 s)."""
    import oracle
    cores = host_cores()
    t0 = time.perf_counter()
    oracle.evaluate(pr.programs[:16], pr.lengths[:16], pr.consts[:16], pr.X, y, oracle.MSE, pr.N, nthreads=cores)
    dt16 = max(time.perf_counter() - t0, 1e-3)
    S = int(min(pr.P, max(16, 16 * 6.0 / dt16)))
    idx = np.sort(np.random.default_rng(2).choice(pr.P, S, replace=False))
    t0 = time.perf_counter()
    oracle.evaluate(pr.programs[idx], pr.lengths[idx], pr.consts[idx], pr.X, y, oracle.MSE, pr.N, nthreads=cores)
    oracle.evaluate(pr.programs[idx], pr.lengths[idx], pr.consts[idx], pr.X, y, oracle.CORR, pr.N, nthreads=cores)
    dt = time.perf_counter() - t0
    units = float(pr.lengths[idx].astype(np.int64).sum()) * pr.N
    return {"value": units / dt / 1e9, "unit": "GPop/s", "cores": cores, "kind": "oracle",
            "sample": f"{S} of {pr.P} programs x {pr.N} cases, MSE and 1-r^2 (two passes), {dt:.1f} s"}


def parity_leg(pr, y_dev, X_dev, population, ctx, binding, vcfg, nun, seed, gen, sample=512):
    """The error report of this run against the FP64 oracle, outside the
    timed region, on the population the timed generations produced: the
    device fitness (both kinds) of a sample of its programs against the
    oracle's, with the oracle's certificates (oracle.parity_report), and one
    more generation's selection and variation from the device fitness,
    bit for bit against the oracle's on the same fitness."""
    import torch

    import oracle
    P_, L_, C_ = population
    f = binding.sr_eval(ctx, P_, L_, C_, X_dev, y_dev, pr.N, binding.SR_MSE_CORR)
    parents = binding.sr_select_tournament(ctx, f[1].contiguous(), 4, seed, gen)
    kids = binding.sr_vary(ctx, P_, L_, C_, parents, pr.nvars, vcfg, seed, gen)
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    prog, lens, cons = P_.cpu().numpy(), L_.cpu().numpy(), C_.cpu().numpy()
    y = y_dev.cpu().numpy()
    par_or = oracle.tournament(f[1], 4, seed, gen)
    kids_or = oracle.vary(prog, lens, cons, par_or, cons.shape[1], pr.nvars, seed=seed, gen=gen, unary_ops=nun)
    t0 = time.perf_counter()
    idx = np.sort(np.random.default_rng(3).choice(pr.P, min(sample, pr.P), replace=False))
    errb, errp, cfl, f0 = oracle.condition_fo(prog[idx], lens[idx], cons[idx], pr.X, y, pr.N,
                                              nthreads=host_cores())
    reps = {name: oracle.parity_report(k, f[k, idx], f0[k], errb[k], errp[k], cfl[k], y)
            for k, name in ((oracle.MSE, "mse"), (oracle.CORR, "corr"))}
    return {"sample": f"{len(idx)} of the {pr.P} programs after the timed generations, all {pr.N} cases, "
                      f"oracle {time.perf_counter() - t0:.1f} s on {host_cores()} cores",
            "tolerance": "|f - f_oracle| <= 1e-4 |f_oracle| + floor (1e-7 var(y) MSE, 1e-6 1-r^2) on certified "
                         "programs; max_rel_tol / p99_rel_tol are |f - f_oracle| / tol over them",
            **reps,
            "parents_bit_exact": bool(np.array_equal(parents.cpu().numpy(), par_or)),
            "offspring_bit_exact": bool(all(np.array_equal(a.cpu().numpy().view(np.uint8), b.view(np.uint8))
                                            for a, b in zip(kids, kids_or)))}


# ------------------------------------------------------------------ other workloads
def _timed(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def _alu_peak(dev):
    """FP32 lane-op peak of the device: SMs x 128 lanes x the measured max SM clock."""
    import torch
    pk, src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * sm_max * 1e-3, f"{sms} SMs x 128 FP32 lanes x {sm_max:.0f} MHz ({src} max clock)"


def _roofline(dev, achieved, kernel, timing, workload, ncu_key=None, units_per_launch=None):
    """ALU roofline of a workload's dominant kernel.  achieved: GPop/s of that
    kernel from CUDA events; traffic: DRAM bytes per launch from its ncu
    capture (scaled by units where it grows with them), else null."""
    peak, src = _alu_peak(dev)
    cap, prov = ncu_record(ncu_key) if ncu_key else (None, None)
    same = cap is not None and workload.split(":")[0] == cap["workload"]
    traffic = None
    if cap is not None and (same or cap["scale"]):
        traffic = cap["dram_bytes"] * (units_per_launch / cap["units"] if units_per_launch else 1.0)
    # the DRAM side of the same launch: traffic over the launch time (units /
    # achieved), against the measured copy bandwidth
    hbm = None
    if traffic is not None and units_per_launch and achieved > 0:
        pk, psrc = peaks()
        gbs = traffic / (units_per_launch / (achieved * 1e9)) / 1e9
        hbm = {"gbs": gbs, "peak_gbs": pk["hbm_gbs"], "frac": gbs / pk["hbm_gbs"], "peak_source": psrc}
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GPop/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kernel, "timing": timing,
            "issue_active_ncu": cap["issue_active"] if same else None, "ncu_provenance": prov,
            "peak_source": src, "hbm": hbm}


class _Region:
    """Clock samples and the library's launch count over a timed region."""

    def __init__(self, binding, ctx, index):
        self.binding, self.ctx, self.sampler = binding, ctx, ClockSampler(index)

    def __enter__(self):
        import torch
        torch.cuda.synchronize()
        self.sampler.start()
        self.l0 = self.binding.sr_kernel_launches(self.ctx)
        return self

    def __exit__(self, *exc):
        import torch
        torch.cuda.synchronize()
        self.launches = int(self.binding.sr_kernel_launches(self.ctx) - self.l0)
        self.clocks = self.sampler.stop()
        return False


def _device_problem(make, dev, binding, ctx, noise_seed=7):
    """A problem from make(attempt) whose target, evaluated by the library's
    own predict, is finite, not constant and below 1e15 in magnitude (the
    recipe redraws with the next attempt otherwise), and its device copies
    with y = that output plus the problem's noise (FP64 on the host).
    Returns (problem, programs, lengths, consts, X, y)."""
    import torch
    from paper_2603_12292_gb300 import inputs
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    for attempt in range(20):
        pr = make(attempt)
        X = t(pr.X)
        tgt = np.zeros((1, max(pr.Lmax, len(pr.target))), np.uint8)
        tgt[0, : len(pr.target)] = pr.target
        yh = binding.sr_predict(ctx, t(tgt), t(np.array([len(pr.target)], np.int32)),
                                t(pr.target_consts[None, :]), X, pr.N)[0, : pr.N].double().cpu().numpy()
        if np.all(np.isfinite(yh)) and np.abs(yh).max() < 1e15 and np.std(yh) > 1e-6 * (1 + np.abs(yh).max()):
            break
    else:
        raise RuntimeError(f"no usable target for {pr.name}")
    y = inputs.add_noise(np.random.default_rng(pr.seed + noise_seed), yh, pr.noise) if pr.noise \
        else yh.astype(np.float32)
    return pr, t(pr.programs), t(pr.lengths), t(pr.consts), X, t(y)


def run_workload(args, local_rank):
    import torch

    import __graft_entry__
    from paper_2603_12292_gb300 import binding, inputs
    from paper_2603_12292_gb300.evolve import EvolveConfig, Evolver, Population

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ctx = binding.Context(local_rank)
    stream = torch.cuda.current_stream(dev)
    line = {"higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "vs_baseline": None, "steps": args.steps, "warmup": args.warmup}

    if args.workload == "batched":
        from paper_2603_12292_gb300.autotune import Autotuner
        tuner = Autotuner(ctx)

        def build(shapes):
            pops = []
            for sh in shapes:
                pr, pg, ln, cs, X, y = _device_problem(lambda a, sh=sh: inputs.batched_problem(sh, attempt=a),
                                                       dev, binding, ctx)
                kind = binding.SR_CORR if sh["kind"] else binding.SR_MSE
                cfg = EvolveConfig(select_kind=kind, eval_kind=kind)
                pops.append(Population(pg, ln, cs, X, y, pr.N, cfg))
            return pops

        nodes = lambda pops: sum(float(p.current[1].sum()) * p.N for p in pops)

        def compare_eval(pops):
            """One evaluation of every problem: a loop of sr_eval calls, one
            batched call with the library's automatic shape, and one with the
            autotuned shape (cases per item x CTAs per SM)."""
            def plain_loop():
                for p in pops:
                    binding.sr_eval(ctx, *p.current, p.X, p.y, p.N, p.cfg.eval_kind, fitness=p.fitness[0])
            probs = [binding.make_problem(*p.current, p.X, p.y, p.N, p.cfg.eval_kind, fitness=p.fitness[0])
                     for p in pops]
            batched = lambda: binding.sr_eval_batched(ctx, probs)
            for f in (plain_loop, batched):
                for _ in range(max(1, args.warmup)):
                    f()
            t_plain = _timed(plain_loop, args.steps, stream)
            binding.sr_set_occupancy(ctx, 0, 0)
            t_auto = _timed(batched, args.steps, stream)
            best = tuner.tune_batched(probs)
            t_tuned = _timed(batched, args.steps, stream)
            n = nodes(pops)
            return {"problems": len(pops), "node_cases": n, "plain_loop_gpops": n / t_plain / 1e6,
                    "batched_auto_gpops": n / t_auto / 1e6, "batched_tuned_gpops": n / t_tuned / 1e6,
                    "batched_over_plain": t_plain / t_tuned, "tuned_over_auto": t_auto / t_tuned,
                    "tuned": {"cases_per_tile": best["tile"] or "automatic", "ctas_per_sm": best["ctas"]},
                    "ms": {"plain_loop": t_plain, "batched_auto": t_auto, "batched_tuned": t_tuned}}

        def compare_adam(pops):
            """One Adam step on every problem's constants: a loop of
            sr_eval_grad + sr_adam_step per problem, against one
            sr_eval_grad_batched + one sr_adam_step_batched."""
            acfg = binding.adam_cfg()
            bufs = []
            for p in pops:
                P_, L_, C_ = p.current
                g = torch.empty((P_.shape[0], C_.shape[1]), dtype=torch.float64, device=dev)
                bufs.append((torch.empty(P_.shape[0], dtype=torch.float64, device=dev), g, torch.zeros_like(g),
                             torch.zeros_like(g), C_.clone()))
            st = {"t": 0}

            def loop():
                st["t"] += 1
                for p, (mse, g, m, v, c) in zip(pops, bufs):
                    P_, L_, _ = p.current
                    binding.sr_eval_grad(ctx, P_, L_, c, p.X, p.y, p.N, mse=mse, dconst=g)
                    binding.sr_adam_step(ctx, c, g, m, v, st["t"], acfg)
            gp = [binding.make_grad_problem(p.current[0], p.current[1], c, p.X, p.y, p.N, mse=mse, dconst=g)
                  for p, (mse, g, m, v, c) in zip(pops, bufs)]
            tables = [(c, g, m, v) for (mse, g, m, v, c) in bufs]

            def batched():
                st["t"] += 1
                binding.sr_eval_grad_batched(ctx, gp)
                binding.sr_adam_step_batched(ctx, tables, st["t"], acfg)
            for f in (loop, batched):
                for _ in range(max(1, args.warmup)):
                    f()
            t_loop = _timed(loop, args.steps, stream)
            t_b = _timed(batched, args.steps, stream)
            n = nodes(pops)
            return {"problems": len(pops), "loop_steps_per_s": 1e3 / t_loop, "batched_steps_per_s": 1e3 / t_b,
                    "batched_over_loop": t_loop / t_b, "loop_grad_gpops": n / t_loop / 1e6,
                    "batched_grad_gpops": n / t_b / 1e6}

        main_shapes = inputs.batched_shapes()[: 8 if args.small else None]
        pops = build(main_shapes)
        small = build(inputs.small_batch_shapes())
        r_main = compare_eval(pops)
        r_small = compare_eval(small)
        r_adam = compare_adam(small)
        # the whole generation loop of the main batch, batched, autotuned and
        # captured as a CUDA graph
        ev = Evolver(ctx, pops, batched=True)
        ev.autotune(tuner)
        l0 = binding.sr_kernel_launches(ctx)
        ev.step()  # one eager generation: the launches a replayed generation makes
        per_gen = binding.sr_kernel_launches(ctx) - l0
        ev.capture(2)
        torch.cuda.synchronize()
        gens = 2 * max(1, args.steps // 2)
        n_gen = nodes(pops)
        with _Region(binding, ctx, local_rank) as region:
            t_graph = _timed(lambda: ev.run(gens), 1, stream) / gens
        binding.sr_set_occupancy(ctx, 0, 0)
        line.update(metric=f"GPop/s, {len(main_shapes)} problems per generation (batched + graph vs plain loop)",
                    value=n_gen / (t_graph / 1e3) / 1e9, unit="GPop/s", ms_per_step=t_graph,
                    scaling="weak",
                    config={"workload": f"batched-{len(main_shapes)}: nvars 1-10, N log-uniform 1k-1M, "
                                        "P 512-8192, L 4-256, MSE/1-r^2 mixed",
                            "problems": len(pops), "node_cases_per_eval": r_main["node_cases"],
                            "step": "one generation: sr_eval_batched (autotuned) + tournament + variation per "
                                    "problem, CUDA-graph replay"},
                    roofline=_roofline(dev, r_main["batched_tuned_gpops"], "eval_batched_kernel (sr_eval_batched)",
                                       "one batched evaluation, CUDA events over a loop of calls",
                                       f"batched-{len(main_shapes)}", "batched", r_main["node_cases"]),
                    clocks=region.clocks, gpu_launches=int(per_gen * gens),
                    batched_eval=r_main, small_batch_eval=dict(r_small, workload="small-64: nvars 1-10, N 316-10k, "
                                                                "P 64-1024, L 4-64, MSE/1-r^2 mixed"),
                    small_batch_adam=dict(r_adam, workload="small-64, K = 4, one Adam step per problem"),
                    batched_over_plain=r_main["batched_over_plain"],
                    generation_graph_ms=t_graph)
    elif args.workload == "adjoint":
        pr, pg, ln, cs, X, y = _device_problem(
            lambda a: inputs.adjoint(attempt=a, P=2048, N=131072) if args.small else inputs.adjoint(attempt=a),
            dev, binding, ctx)
        P, K, N = pr.P, pr.K, pr.N
        mse = torch.empty(P, dtype=torch.float64, device=dev)
        g = torch.empty((P, K), dtype=torch.float64, device=dev)
        m, v = torch.zeros_like(g), torch.zeros_like(g)
        cfg = binding.adam_cfg()
        state = {"t": 0}
        grad_ev = []
        def adam_step(record=False):
            state["t"] += 1
            if record:
                grad_ev.append((torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)))
                grad_ev[-1][0].record(stream)
            binding.sr_eval_grad(ctx, pg, ln, cs, X, y, N, mse=mse, dconst=g)
            if record:
                grad_ev[-1][1].record(stream)
            binding.sr_adam_step(ctx, cs, g, m, v, state["t"], cfg)
        # plain alternative: central differences with 2K + 1 plain evaluations
        f0 = torch.empty(P, dtype=torch.float64, device=dev)
        fp, fm = torch.empty_like(f0), torch.empty_like(f0)
        c2 = cs.clone()
        def fd_step():
            binding.sr_eval(ctx, pg, ln, cs, X, y, N, binding.SR_MSE, fitness=f0)
            for k in range(K):
                c2.copy_(cs)
                c2[:, k] += 1e-3
                binding.sr_eval(ctx, pg, ln, c2, X, y, N, binding.SR_MSE, fitness=fp)
                c2[:, k] -= 2e-3
                binding.sr_eval(ctx, pg, ln, c2, X, y, N, binding.SR_MSE, fitness=fm)
                g[:, k] = (fp - fm) / 2e-3
            state["t"] += 1
            binding.sr_adam_step(ctx, cs, g, m, v, state["t"], cfg)
        for _ in range(max(1, args.warmup)):
            adam_step()
        steps = max(1, args.steps)
        with _Region(binding, ctx, local_rank) as region:
            t_adj = _timed(lambda: adam_step(True), steps, stream)
        grad_ms = float(np.mean([a.elapsed_time(b) for a, b in grad_ev]))
        fd_step()  # untimed: first-call costs of the plain path stay out of the comparison
        t_fd = _timed(fd_step, 1, stream)
        nodes = float(ln.sum()) * N
        line.update(metric="constant-optimisation steps/s (adjoint + Adam) vs plain finite differences",
                    value=1e3 / t_adj, unit="steps/s", ms_per_step=t_adj, scaling="weak",
                    config={"workload": f"{pr.name}: K=8, L<=96, 5 vars, Adam"},
                    roofline=_roofline(dev, nodes / (grad_ms / 1e3) / 1e9, "grad_kernel (sr_eval_grad)",
                                       "sr_eval_grad call inside each timed Adam step, CUDA events",
                                       pr.name, "grad", nodes),
                    clocks=region.clocks, gpu_launches=region.launches,
                    grad_ms=grad_ms, grad_gpops=nodes / (t_adj / 1e3) / 1e9,
                    fd_steps_per_s=1e3 / t_fd, adjoint_over_fd=t_fd / t_adj)
    elif args.workload == "large":
        pr, pg, ln, cs, X, y = _device_problem(
            lambda a: inputs.large(attempt=a, P=16384, N=131072) if args.small else inputs.large(attempt=a),
            dev, binding, ctx)
        sched = None
        if args.schedule:
            w0 = max(1, args.warmup)
            sched = ((0, pr.P), (w0 + 2, pr.P // 2), (w0 + 4, pr.P // 4))
        cfg = EvolveConfig(select_kind=binding.SR_CORR, eval_kind=binding.SR_CORR, selection=args.selection,
                           schedule=sched)
        ev = Evolver(ctx, [Population(pg, ln, cs, X, y, pr.N, cfg)])
        for _ in range(max(1, args.warmup)):
            ev.step()
        torch.cuda.synchronize()
        steps = max(1, args.steps)
        ms, nodes, sizes = [], [], []
        ev.eval_events = []
        with _Region(binding, ctx, local_rank) as region:
            for _ in range(steps):
                nodes.append(float(ev.pops[0].current[1].sum()) * pr.N)
                sizes.append(ev.pops[0].size)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ev.step()
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
        eval_ms = [a.elapsed_time(b) for a, b in ev.eval_events]
        line.update(metric="GPop/s (nodes x cases / s), one generation (1-r^2, selection, variation)",
                    value=sum(nodes) / (sum(ms) / 1e3) / 1e9, unit="GPop/s", ms_per_step=sum(ms) / steps,
                    scaling="weak",
                    config={"workload": pr.name, "programs": pr.P, "cases": pr.N, "lengths": "4-256",
                            "selection": args.selection, "population_sizes": sizes},
                    roofline=_roofline(dev, float(np.mean([n / (t / 1e3) / 1e9 for n, t in zip(nodes, eval_ms)])),
                                       "eval_kernel (sr_eval SR_CORR)",
                                       "sr_eval call inside each timed generation, CUDA events",
                                       pr.name, "large", float(np.mean(nodes))),
                    clocks=region.clocks, gpu_launches=region.launches,
                    eval_ms=float(np.mean(eval_ms)))
    elif args.workload == "beagle":
        nun = 12 if args.ops == "table1" else 6
        pr, pg, ln, cs, X, y = _device_problem(lambda a: inputs.paper_shaped(attempt=a, unary_ops=nun),
                                               dev, binding, ctx)
        # 1 % invalid targets (NaN, +inf, -inf in turn) at seeded cases
        bad = np.sort(np.random.default_rng(pr.seed + 11).choice(pr.N, pr.N // 100, replace=False))
        yv = y.clone()
        vals = torch.tensor([float("nan"), float("inf"), float("-inf")], dtype=torch.float32, device=dev)
        yv[torch.from_numpy(bad).to(dev)] = vals[torch.arange(len(bad), device=dev) % 3]
        P, M, SEED = pr.P, 1000, 20260312
        score = torch.empty(P, dtype=torch.float64, device=dev)
        counts = torch.empty((P, 2), dtype=torch.int32, device=dev)
        parents = torch.empty((P, 2), dtype=torch.int32, device=dev)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        vcfg = binding.var_cfg(unary_ops=nun)
        pop = [(pg, ln, cs), (torch.empty_like(pg), torch.empty_like(ln), torch.empty_like(cs))]
        state = {"gen": 0, "cur": 0}

        score_ev = []

        def generation(record=False):
            g, cur = state["gen"], state["cur"]
            P_, L_, C_ = pop[cur]
            if record:
                score_ev.append((torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)))
                score_ev[-1][0].record(stream)
            binding.sr_eval_score(ctx, P_, L_, C_, X, yv, pr.N, binding.SR_SCORE_R4, M, score=score,
                                  pair_counts=counts)
            if record:
                score_ev[-1][1].record(stream)
            binding.sr_select_tournament_max(ctx, score, 4, SEED, g, parents=parents)
            binding.sr_vary(ctx, P_, L_, C_, parents, pr.nvars, vcfg, SEED, g, out=pop[1 - cur])
            state["gen"], state["cur"] = g + 1, 1 - cur

        for _ in range(max(3, args.warmup)):
            generation()
        torch.cuda.synchronize()
        steps = max(1, args.steps)
        ms, nodes = [], []
        with _Region(binding, ctx, local_rank) as region:
            for _ in range(steps):
                nodes.append(float(pop[state["cur"]][1].sum()) * pr.N)
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                generation(record=True)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
        score_ms = [a.elapsed_time(b) for a, b in score_ev]
        # evaluation alone on the current population: Eq. 2, Eq. 3, and MSE + 1 - r^2
        P_, L_, C_ = pop[state["cur"]]
        n_cur = float(L_.sum()) * pr.N
        f2 = torch.empty((2, P), dtype=torch.float64, device=dev)
        t_r4 = _timed(lambda: binding.sr_eval_score(ctx, P_, L_, C_, X, yv, pr.N, binding.SR_SCORE_R4, M,
                                                    score=score, pair_counts=counts), steps, stream)
        t_p2p = _timed(lambda: binding.sr_eval_score(ctx, P_, L_, C_, X, yv, pr.N, binding.SR_SCORE_P2P, M,
                                                     score=score, pair_counts=counts), steps, stream)
        t_both = _timed(lambda: binding.sr_eval(ctx, P_, L_, C_, X, y, pr.N, binding.SR_MSE_CORR, fitness=f2),
                        steps, stream)
        line.update(metric="GPop/s, one generation scored by Beagle's r^4 score (Eq. 2) with invalid targets",
                    value=sum(nodes) / (sum(ms) / 1e3) / 1e9, unit="GPop/s", ms_per_step=sum(ms) / steps,
                    scaling="weak",
                    config={"workload": f"beagle-4096x100k{'-table1' if nun == 12 else ''}: paper shapes, "
                                        "1% invalid targets, M = 1000",
                            "step": "sr_eval_score(R4) + sr_select_tournament_max(k=4) + sr_vary",
                            "l2": "flushed between timed generations"},
                    roofline=_roofline(dev, float(np.mean([n / (t / 1e3) / 1e9 for n, t in zip(nodes, score_ms)])),
                                       "eval_kernel (sr_eval_score SR_SCORE_R4)",
                                       "sr_eval_score call inside each timed generation, CUDA events",
                                       f"beagle-4096x100k{'-table1' if nun == 12 else ''}", "beagle",
                                       float(np.mean(nodes))),
                    clocks=region.clocks, gpu_launches=region.launches,
                    r4_eval_gpops=n_cur / (t_r4 / 1e3) / 1e9, p2p_eval_gpops=n_cur / (t_p2p / 1e3) / 1e9,
                    mse_corr_eval_gpops=n_cur / (t_both / 1e3) / 1e9)
    elif args.workload == "opmix":
        # one evaluation (both kinds from one pass) of the paper-shaped
        # population drawn from one operator class at a time
        classes, runs = {}, {}
        for cls in inputs.OPMIX_CLASSES:
            pr, pg, ln, cs, X, y = _device_problem(lambda a, c=cls: inputs.opmix(c, attempt=a), dev, binding, ctx)
            f2 = torch.empty((2, pr.P), dtype=torch.float64, device=dev)
            runs[cls] = (lambda pg=pg, ln=ln, cs=cs, X=X, y=y, f2=f2, N=pr.N:
                         binding.sr_eval(ctx, pg, ln, cs, X, y, N, binding.SR_MSE_CORR, fitness=f2))
            for _ in range(max(1, args.warmup)):
                runs[cls]()
            classes[cls] = {"units": float(ln.sum()) * pr.N, "mean_length": float(ln.float().mean())}
        with _Region(binding, ctx, local_rank) as region:
            for cls, run in runs.items():
                t = _timed(run, max(1, args.steps), stream)
                g = classes[cls].pop("units") / t / 1e6
                classes[cls].update(gpops=g, ms=t, frac_of_alu_peak=g / _alu_peak(dev)[0])
        line.update(metric="GPop/s per operator class (paper-shaped population, one sr_eval of both kinds)",
                    value=classes["base"]["gpops"], unit="GPop/s", ms_per_step=classes["base"]["ms"],
                    scaling="weak",
                    config={"workload": "opmix: 4,096 programs of length 8-128 x 100,000 cases per class",
                            "classes": {c: ({k: v for k, v in d.items()} or "all base operators")
                                        for c, d in inputs.OPMIX_CLASSES.items()}},
                    roofline=_roofline(dev, classes["base"]["gpops"], "eval_kernel (sr_eval SR_MSE_CORR)",
                                       "a loop of sr_eval calls per class, CUDA events", "opmix-base"),
                    opmix=classes, clocks=region.clocks, gpu_launches=region.launches)
    else:  # plain: launch-bound, CUDA graph vs eager
        pr, pg, ln, cs, X, y = _device_problem(lambda a: inputs.plain(attempt=a), dev, binding, ctx)
        pe = Population(pg.clone(), ln.clone(), cs.clone(), X, y, pr.N,
                        EvolveConfig(select_kind=binding.SR_MSE, eval_kind=binding.SR_MSE))
        pgr = Population(pg.clone(), ln.clone(), cs.clone(), X, y, pr.N,
                         EvolveConfig(select_kind=binding.SR_MSE, eval_kind=binding.SR_MSE))
        eager, graph = Evolver(ctx, [pe]), Evolver(ctx, [pgr])
        for _ in range(max(3, args.warmup)):
            eager.step()
        l0 = binding.sr_kernel_launches(ctx)
        eager.step()  # one eager generation: the launches a replayed generation makes
        per_gen = binding.sr_kernel_launches(ctx) - l0
        graph.capture(2)
        graph.run(4)
        torch.cuda.synchronize()
        gens = 2 * max(5, args.steps)
        t_e = _timed(lambda: [eager.step() for _ in range(gens)], 1, stream) / gens
        gens_g = 2 * max(1000, args.steps)  # long enough for the clock sampler
        with _Region(binding, ctx, local_rank) as region:
            t_g = _timed(lambda: graph.run(gens_g), 1, stream) / gens_g
        n = float(pgr.current[1].sum()) * pr.N
        P_, L_, C_ = pgr.current
        f1 = torch.empty(pr.P, dtype=torch.float64, device=dev)
        t_eval = _timed(lambda: binding.sr_eval(ctx, P_, L_, C_, X, y, pr.N, binding.SR_MSE, fitness=f1),
                        gens, stream)
        line.update(metric="generations/s, 256 x 1k (CUDA graph vs eager launches)",
                    value=1e3 / t_g, unit="generations/s", ms_per_step=t_g, scaling="weak",
                    config={"workload": pr.name},
                    roofline=_roofline(dev, n / (t_eval / 1e3) / 1e9, "eval_kernel (sr_eval SR_MSE)",
                                       "sr_eval calls in a loop, CUDA events; launch-bound at 1,000 cases",
                                       pr.name),
                    clocks=region.clocks, gpu_launches=int(per_gen * gens_g),
                    eager_generations_per_s=1e3 / t_e,
                    graph_gpops=n / (t_g / 1e3) / 1e9, graph_over_eager=t_e / t_g)
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    args = parse()
    if args.workload != "paper" and args.impl == "ours":
        return run_workload(args, int(os.environ.get("LOCAL_RANK", "0")))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        if args.impl == "reference":
            return run_reference(args, rank, world)
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
        try:
            return run_ours(args, rank, world, local_rank)
        finally:
            dist.destroy_process_group()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
