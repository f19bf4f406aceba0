#!/usr/bin/env python
"""Benchmark of the fused payoff-expression Monte Carlo engine.

One step prices one contract of the selected workload (default: the daily
knock-out barrier on the worst-of, 3 correlated GBM underlyings, 365 daily
dates, 2^22 paths -- the largest single-GPU configuration): Philox normals
-> Brownian bridge -> correlated GBM -> payoff bytecode -> mean / variance,
all in one kernel launch.

Prints one JSON line (rank 0):
  value   -- path-date evaluations per second over all ranks, kernel time
             from CUDA events on the launch stream, inputs resident on the
             device, L2 flushed (256 MiB write) between steps;
  e2e     -- the same metric through the C ABI as a user calls it: load the
             payoff bytecode from host memory (host-to-device copy), price,
             read the result back to the host, release the contract;
  roofline, cpu_baseline (the FP64 oracle on host cores), clocks, ...
``--impl reference`` times the oracle instead (the reference arm).
Multi-GPU (torchrun): each rank prices its own disjoint path range of the
same contract (no data-path collective; weak scaling); after the timed
region the ranks' (sum, sum of squares, n) are merged in rank order on the
host (merge.allgather_sums over a gloo group) and the merged price printed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "path·date evals/sec & contracts priced/sec at 1e-4 rel. std-err vs plain MC"
UNIT = "path·date/s"
TARGET_REL_SE = 1e-4
KERNEL_SRCS = [os.path.join(ROOT, "paper_2108_03076_gb300", "csrc", f)
               for f in ("pc_kernels.cu", "pc_eval.cuh", "pc_eval_state.inc", "pc_ops.inc", "pc_price.cuh",
                         "pc_device.cuh", "pc_types.h")]
# a specialised kernel is identified by the CUDA source generated for the
# program (pc_debug_jit_source) and the device headers that source includes
JIT_SRCS = [os.path.join(ROOT, "paper_2108_03076_gb300", "csrc", f)
            for f in ("pc_types.h", "pc_device.cuh", "pc_price.cuh", "pc_eval_state.inc", "pc_ops.inc")]
GREEKS_SRCS = [os.path.join(ROOT, "paper_2108_03076_gb300", "csrc", f)
               for f in ("pc_greeks.cu", "pc_greeks.cuh", "pc_greeks_state.inc", "pc_greeks_ops.inc",
                         "pc_device.cuh", "pc_types.h")]
JIT_GREEKS_SRCS = [os.path.join(ROOT, "paper_2108_03076_gb300", "csrc", f)
                   for f in ("pc_types.h", "pc_device.cuh", "pc_greeks.cuh", "pc_greeks_state.inc",
                             "pc_greeks_ops.inc")]
ADJOINT_SRCS = [os.path.join(ROOT, "paper_2108_03076_gb300", "csrc", f)
                for f in ("pc_adjoint.cu", "pc_adjoint.cuh", "pc_device.cuh", "pc_types.h")]
PORTFOLIO = "portfolio_1024"
LEARNED = "learned_cv_worst_of_autocall"
PORTFOLIO_SEED = 0x5EED0004


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def alg_ops_per_path(info) -> dict:
    """Algorithmic thread-operations of generating one full path (all dates),
    counted on the method's n d normals (n d / 4 Philox blocks, n d / 2
    Box-Muller pairs, which is what the kernel draws):
    Philox4x32-10: 10 rounds x (2 mul.lo + 2 mul.hi + 2 three-way xor) = 60;
    Box-Muller pair: 2 shifts, 2 int->float, 2 FMA (u_a, angle), lg2, mul,
    sqrt, sin, cos, 2 mul = 13 (4 on the MUFU pipe);
    bridge: d ops for the first node, 3d for each other node;
    correlation + GBM per date: d(d+1)/2 FMA + d ex2 + d mul.
    The payoff's own arithmetic is not counted (a lower bound)."""
    d, n = info.d, info.n_dates
    blocks, pairs = n * d / 4.0, n * d / 2.0
    ops = (60 * blocks + 13 * pairs + (3 * n * d - 2 * d) + n * (d * (d + 1) // 2 + 2 * d))
    mufu = 4 * pairs + n * d
    return {"ops": ops, "mufu": mufu}


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons while running.

    The sampler is up (first sample read) before the region starts and
    stops after a sample taken once the region has ended, so a region
    shorter than the sampling period still has its neighbours recorded
    (`in_region` counts the samples taken inside it)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.samples = []  # (host time, line)
        self.t0 = self.t1 = None
        self.cv = threading.Condition()

    def _read(self):
        for l in self.proc.stdout:
            if l.strip():
                with self.cv:
                    self.samples.append((time.perf_counter(), l))
                    self.cv.notify_all()

    def _wait(self, pred, timeout):
        with self.cv:
            self.cv.wait_for(pred, timeout)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
            self._wait(lambda: len(self.samples) > 0, 5.0)
        except OSError:
            self.proc = None
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *exc):
        self.t1 = time.perf_counter()
        if self.proc is not None:
            self._wait(lambda: any(t > self.t1 for t, _ in self.samples), 2.0)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
        with self.cv:
            self.lines = [l for _, l in self.samples]
            self.in_region = sum(1 for t, _ in self.samples if self.t0 <= t <= self.t1)

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "in_region": getattr(self, "in_region", 0)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


PROFILED = {  # kernel kind: (profiles/ file prefix, sources, specialised-kernel kind or None)
    "interpreter": ("price_kernel", KERNEL_SRCS, None),
    "adjoint": ("adjoint_kernel", ADJOINT_SRCS, None),
    "specialised": ("jit_price_kernel", JIT_SRCS, 0),
    "greeks": ("greeks_kernel", GREEKS_SRCS, None),
    "greeks_specialised": ("jit_greeks_kernel", JIT_GREEKS_SRCS, 32),
}


def kernel_sha(w, kind: str) -> str:
    """Hash of what the workload's kernel of this kind is compiled from: the
    sources, and for a specialised kernel the CUDA source generated for the
    workload's program."""
    _, srcs, jit_kind = PROFILED[kind]
    h = hashlib.sha256()
    if jit_kind is not None:
        import paper_2108_03076_gb300 as pc
        words, consts = pc.pc_assemble(w.il_text)
        h.update(pc.pc_debug_jit_source(words, consts, w.tparams, w.market.d, 0, 1, jit_kind).encode())
    for src in srcs:
        with open(src, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profile_record(w, kind: str) -> dict:
    """The committed ncu summary of the workload's kernel (profiles/*.json)
    if it was taken on the current kernel source, else {}."""
    path = os.path.join(ROOT, "profiles", f"{PROFILED[kind][0]}_{w.name}.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p if p.get("kernel_sha256") == kernel_sha(w, kind) else {}
    except (OSError, ValueError):
        return {}


def profile_traffic(w, kind: str):
    """DRAM bytes of one launch of the workload, from the committed ncu
    summary if it was taken on the current kernel source (else None).  A
    summary taken on fewer paths is scaled by the paths, unless it records
    that the kernel's traffic does not grow with them ("traffic": "fixed":
    only the program, model tables and partial sums reach DRAM)."""
    p = profile_record(w, kind)
    b, n = p.get("dram_bytes_per_launch"), p.get("n_paths")
    if b is None or not n or p.get("traffic") == "fixed":
        return b
    return b * w.n_paths / n


def oracle_run(w, n_paths: int, offset: int = 0):
    from oracle import il_text, mc
    from oracle.paths import Market
    prog = il_text.parse(w.il_text)
    env = {f"${i}": v for i, v in enumerate(w.tparams)}
    t = time.perf_counter()
    x = mc.payoffs(prog, Market(**vars(w.market)), env, 0, 1, n_paths, w.seed, 0, offset)
    return time.perf_counter() - t, x


def _oracle_chunk(task):
    """Worker of the all-core oracle timing: paths [off, off + n)."""
    w, n, off = task
    oracle_run(w, n, off)
    return n


def cpu_baseline(w, budget_s: float = 12.0) -> dict:
    """The oracle as it stands, on chunks of the workload's paths: one
    process until the time budget is used, then every host core (a spawned
    process pool over path ranges, sized to about the same wall time);
    rates in path-dates/s, the all-core one reported as the value."""
    chunk = 1 << 14
    done, el = 0, 0.0
    while el < budget_s and done < w.n_paths:
        dt, _ = oracle_run(w, min(chunk, w.n_paths - done), done)
        el += dt
        done += min(chunk, w.n_paths - done)
    rate1 = done * w.market.n / el
    out = {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle", "value_1_core": rate1,
           "sample": f"paths 0..{done - 1} of the workload ({done} paths, {el:.1f} s, numpy FP64, 1 thread)"}
    cores = os.cpu_count() or 1
    if cores > 1:
        import multiprocessing as mp
        per = max(1, int(rate1 / w.market.n * budget_s / chunk))      # chunks one core does in the budget
        tasks = [(w, chunk, (i * chunk) % max(w.n_paths - chunk, 1)) for i in range(per * cores)]
        # spawn: the parent holds a CUDA context, a forked child would not start cleanly
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_chunk, [(w, 256, 0)] * cores)            # imports and first call
            t0 = time.perf_counter()
            n_all = sum(pool.map(_oracle_chunk, tasks, chunksize=1))
            el_all = time.perf_counter() - t0
        out.update({"value": n_all * w.market.n / el_all, "cores": cores,
                    "sample": out["sample"] + f"; then {n_all} paths over {cores} spawned processes "
                              f"in {el_all:.1f} s wall"})
    return out


def run_reference(args, w):
    """The oracle as it stands on the host cores: each step prices one chunk
    per core (a spawned process pool over path ranges) of about 80 k
    path-dates (2^14 paths of the 5-date autocall): enough to hide the
    pool's dispatch, short enough for a thousand steps in about a minute."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    chunk = max(256, ((1 << 14) * 5 // max(w.market.n, 1)) // 256 * 256)
    cores = os.cpu_count() or 1
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(cores) as pool:
        off = 0

        def step():
            nonlocal off
            tasks = [(w, chunk, (off + i * chunk) % max(w.n_paths - chunk, 1)) for i in range(cores)]
            off += cores * chunk
            t = time.perf_counter()
            n = sum(pool.map(_oracle_chunk, tasks, chunksize=1))
            return time.perf_counter() - t, n

        for _ in range(args.warmup):
            step()
        total, paths = 0.0, 0
        for _ in range(args.steps):
            dt, n = step()
            total += dt
            paths += n
    value = paths * w.market.n / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(w, None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{chunk} paths per core per step of the workload, {cores} spawned "
                                       "processes (numpy FP64)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config(w, info) -> dict:
    return {"workload": w.name, "n_paths": w.n_paths, "n_dates": w.market.n,
            "underlyings": w.market.d, "il_nodes": info, "seed": w.seed,
            "l2": "flushed between steps by a 256 MiB device write"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="daily_barrier_3u_365d",
                    choices=sorted(W.ALL) + sorted(W.GREEKS) + [PORTFOLIO, LEARNED])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--interpret", action="store_true",
                    help="time the interpreting kernel instead of the contract's specialised kernel")
    ap.add_argument("--paths", type=int, default=0,
                    help="price this many paths instead of the workload's own count (small profiling runs; "
                         "the line's config records it)")
    args = ap.parse_args()
    if args.workload == PORTFOLIO:
        return run_portfolio(args)
    if args.workload == LEARNED:
        return run_learned(args)
    if args.workload in W.GREEKS:
        return run_greeks(args)
    w = W.ALL[args.workload](args.paths) if args.paths > 0 else W.ALL[args.workload]()
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import paper_2108_03076_gb300 as pc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        from paper_2108_03076_gb300 import build
        build.build()
    if ws > 1:
        dist.barrier()
    # a dedicated stream: the engine and the timing events must share it (the
    # legacy default stream has handle 0, which pc_create reads as "none")
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = pc.pc_create(local, stream.cuda_stream)
    spec = w.market
    model = pc.pc_model_create(ctx, spec.S0, spec.sigma, spec.corr, spec.r, spec.days)
    words, consts = pc.pc_assemble(w.il_text)
    info = pc.pc_verify_payoff(words, consts, w.tparams)
    contract = pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
    minfo = pc.pc_model_query(model)
    linfo = pc.pc_price_info(model, contract, w.n_paths)
    offset = rank * w.n_paths
    jit_s = None
    if not args.interpret:
        # the paper's per-instrument compilation: a kernel specialised to this
        # program, compiled once (outside the timed region)
        pc.pc_set_jit(ctx, True)
        t0 = time.perf_counter()
        pc.pc_jit_compile(model, contract)
        jit_s = time.perf_counter() - t0
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        pc.pc_price_async(model, contract, w.n_paths, offset, w.seed, 0, out.data_ptr())
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            pc.pc_price_async(model, contract, w.n_paths, offset, w.seed, 0, out.data_ptr())
            b.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    kernel_ms = [a.elapsed_time(b) for a, b in evs]
    t_dev = sum(kernel_ms) / 1e3
    sums = out.cpu().numpy()
    interp_ms = None
    if not args.interpret:
        # the interpreting kernel on the same inputs, for comparison
        pc.pc_set_jit(ctx, False)
        ims = []
        for _ in range(max(3, min(args.steps, 50))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pc.pc_price_async(model, contract, w.n_paths, offset, w.seed, 0, out.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
            ims.append(a.elapsed_time(b))
        interp_ms = statistics.median(ims)
        pc.pc_set_jit(ctx, True)
    # cutPayoff (Sec. 4.1) of the same contract priced at now = 0: every
    # payoff guarded by if(t < now, 0, .) -- the paper's "-Cut" timings
    cw, ck = pc.pc_cut_payoff(words, consts)
    kcut = pc.pc_load_payoff(ctx, cw, ck, w.tparams, 0, 1)
    if not args.interpret:
        pc.pc_jit_compile(model, kcut)
    cut_out = torch.zeros(4, dtype=torch.float64, device="cuda")
    cms = []
    for i in range(3 + max(3, min(args.steps, 20))):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pc.pc_price_async(model, kcut, w.n_paths, offset, w.seed, 0, cut_out.data_ptr())
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            cms.append(a.elapsed_time(b))
    cut_ms = statistics.median(cms)
    cut_same = bool(np.array_equal(cut_out.cpu().numpy()[:3], sums[:3]))
    pc.pc_contract_destroy(kcut)
    merged = None
    if ws > 1:
        from paper_2108_03076_gb300 import merge
        gloo = dist.new_group(backend="gloo")
        tot = merge.allgather_sums(np.asarray(sums[:3]), group=gloo)[0]
        mp_, mse = merge.estimate(tot)
        merged = {"price": mp_, "stderr": mse, "n_paths": int(tot[2]),
                  "note": "ranks' (sum, sum of squares, n) merged in rank order over gloo"}
    mean = sums[0] / w.n_paths
    var = max(0.0, (sums[1] - w.n_paths * mean * mean) / (w.n_paths - 1))

    # end to end through the public API with host buffers
    n_e2e = max(3, min(args.e2e_steps, args.steps))
    for _ in range(3):
        k = pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
        pc.pc_price(model, k, w.n_paths, w.seed)
        pc.pc_contract_destroy(k)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        k = pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
        price, se = pc.pc_price(model, k, w.n_paths, w.seed)
        pc.pc_contract_destroy(k)
    t_e2e = time.perf_counter() - t0

    if ws > 1:
        t = torch.tensor([t_dev, t_e2e / n_e2e], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev, e2e_step = float(t[0]), float(t[1])
    else:
        e2e_step = t_e2e / n_e2e

    path_dates = w.n_paths * spec.n
    value = ws * path_dates * args.steps / t_dev
    e2e_value = ws * path_dates / e2e_step
    cv = math.sqrt(var) / abs(mean) if mean else float("inf")
    paths_needed = (cv / TARGET_REL_SE) ** 2
    contracts_per_s = ws * (w.n_paths * args.steps / t_dev) / paths_needed

    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    clock_hz = 1e6 * float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 128 * clock_hz
    peak_mufu = props.multi_processor_count * 16 * clock_hz
    ops = alg_ops_per_path(minfo)
    launch_s = t_dev / args.steps
    achieved = ops["ops"] * w.n_paths / launch_s
    kind = "interpreter" if args.interpret or info.n_insn > pc.JIT_MAX_INSNS else "specialised"
    traffic = profile_traffic(w, kind)
    prof = profile_record(w, kind)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {**config(w, info.n_nodes), "parallelism": f"path ranges x{ws}",
                       "kernel": ("interpreter" if args.interpret else
                                  "specialised to the program (run-time compiled, NVRTC)"
                                  if info.n_insn <= pc.JIT_MAX_INSNS else
                                  f"interpreter ({info.n_insn} instructions: above the "
                                  f"{pc.JIT_MAX_INSNS} that are specialised)")
                                 + (", window of dates in HBM" if linfo.hbm_window else "")},
            # where the window of simulated dates lives (a program that looks
            # far back keeps it in HBM: bytes of the launch's buffer, bytes
            # each path writes per simulated date)
            "window": {"dates": linfo.window, "placement": "hbm" if linfo.hbm_window else "shared",
                       "hbm_bytes": int(linfo.hbm_window_bytes),
                       "bytes_written_per_path_date": int(linfo.window_bytes_written_per_path_date)},
            "interpreter_ms_per_step": interp_ms, "specialised_compile_s": jit_s,
            "cut_payoff": {"ms_per_step": cut_ms, "overhead": cut_ms / (1e3 * t_dev / args.steps) - 1.0,
                           "sums_equal_uncut": cut_same,
                           "note": "cutPayoff (Sec. 4.1) of the contract, loaded once, priced at now = 0 "
                                   "(Table 1's -Cut column): median of launches after 3 warm-up"},
            "merged": merged,
            "contracts_per_sec_at_1e-4_rel_se": contracts_per_s,
            "price": mean, "stderr": math.sqrt(var / w.n_paths),
            "paths_for_1e-4_rel_se": paths_needed,
            "gpu_launches": args.steps,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(words.nbytes + consts.nbytes + 4 * len(w.tparams)),
                    "d2h_bytes_per_step": 40,
                    "note": "pc_load_payoff + pc_price + pc_contract_destroy per step, host wall clock "
                            "(a reloaded program finds its compiled kernel in the context's cache)"},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Tops/s", "frac": achieved / peak_ops, "traffic": traffic,
                         "mufu_frac": ops["mufu"] * w.n_paths / launch_s / peak_mufu,
                         # the busiest pipe's issue rate and the issue-active fraction from the
                         # committed ncu capture of this kernel source (null if none)
                         "ncu_max_pipe": prof.get("ncu_max_pipe"),
                         "ncu_max_pipe_frac": prof.get("ncu_max_pipe_frac"),
                         "ncu_issue_active": prof.get("ncu_issue_active"),
                         "alg_ops_per_path": ops["ops"],
                         "peak_basis": f"{props.multi_processor_count} SMs x 128 lanes x "
                                       f"{clock_hz / 1e6:.0f} MHz issue (MUFU: x16)"},
            "clocks": clk.summary(),
        }
        if linfo.hbm_window:
            # the window in HBM: every simulated date is written once and the
            # program reads it back -- algorithmically n d floats out and in
            # per path; bound by HBM when that fraction exceeds the issue one
            hbm_peak = 1e9 * float(peaks.get("hbm_gbs", 6800.0))
            alg_bytes = 2.0 * 4.0 * spec.n * spec.d * w.n_paths
            hbm_frac = alg_bytes / launch_s / hbm_peak
            line["roofline"]["hbm"] = {"achieved": alg_bytes / launch_s / 1e9, "peak": hbm_peak / 1e9,
                                       "unit": "GB/s", "frac": hbm_frac, "alg_bytes_per_launch": alg_bytes,
                                       "peak_basis": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks
                                       else "fallback 6.8 TB/s"}
            if hbm_frac > line["roofline"]["frac"]:
                line["roofline"].update({"bound": "hbm", "achieved": alg_bytes / launch_s / 1e9,
                                         "peak": hbm_peak / 1e9, "unit": "GB/s", "frac": hbm_frac})
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)

    pc.pc_contract_destroy(contract)
    pc.pc_model_destroy(model)
    pc.pc_destroy(ctx)
    if ws > 1:
        dist.destroy_process_group()



# ---------------------------------------------------------------------------
# Portfolio: 1024 templated contracts priced by one replay of a batch plan
# ---------------------------------------------------------------------------


def portfolio_config(items, ws) -> dict:
    from collections import Counter
    return {"workload": PORTFOLIO, "contracts": len(items),
            "total_paths": sum(it.n_paths for it in items),
            "path_dates": sum(it.n_paths * it.market.n for it in items),
            "templates": dict(Counter(it.template for it in items)),
            "underlyings": "1-4", "dates": "1-365", "seed": PORTFOLIO_SEED,
            "parallelism": f"contracts x{ws}",
            "l2": "flushed between steps by a 256 MiB device write"}


def portfolio_reference(args, items):
    """The oracle on a bounded sample per step: 512 paths of each of the
    next contracts in portfolio order until 2 s of CPU time are used."""
    from oracle import il_text, mc
    from oracle.paths import Market
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    i = 0

    def step(budget=2.0):
        nonlocal i
        pd, el = 0, 0.0
        while el < budget:
            it = items[i % len(items)]
            n = min(512, it.n_paths)
            env = {f"${k}": v for k, v in enumerate(it.tparams)}
            t = time.perf_counter()
            mc.payoffs(il_text.parse(it.il_text), Market(**vars(it.market)), env, 0, 1, n,
                       PORTFOLIO_SEED, i % len(items), 0)
            el += time.perf_counter() - t
            pd += n * it.market.n
            i += 1
        return pd, el
    for _ in range(args.warmup):
        step(0.2)
    tot_pd, tot_t = 0, 0.0
    for _ in range(args.steps):
        pd, el = step()
        tot_pd += pd
        tot_t += el
    pd_rate = tot_pd / tot_t
    # contracts priced per second at the portfolio's own path budgets
    value = pd_rate * len(items) / sum(it.n_paths * it.market.n for it in items)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "contracts/s",
            "path_date_evals_per_sec": pd_rate,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": portfolio_config(items, ws),
            "cpu_baseline": {"value": value, "unit": "contracts/s", "cores": 1, "kind": "oracle",
                             "sample": "512 paths of each contract in portfolio order, 2 s per "
                                       "step; rate scaled to the full path budgets"},
            "e2e": {"value": value, "unit": "contracts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def portfolio_cpu_baseline(items, budget_s: float = 12.0) -> dict:
    """The oracle as it stands, single process: 512 paths of each contract in
    portfolio order until the time budget is used; its path-date rate scaled
    to contracts/s at the portfolio's own path budgets."""
    from oracle import il_text, mc
    from oracle.paths import Market
    pd, el, i = 0, 0.0, 0
    while el < budget_s and i < len(items):
        it = items[i]
        n = min(512, it.n_paths)
        env = {f"${k}": v for k, v in enumerate(it.tparams)}
        t = time.perf_counter()
        mc.payoffs(il_text.parse(it.il_text), Market(**vars(it.market)), env, 0, 1, n, PORTFOLIO_SEED, i, 0)
        el += time.perf_counter() - t
        pd += n * it.market.n
        i += 1
    value = (pd / el) * len(items) / sum(it.n_paths * it.market.n for it in items)
    return {"value": value, "unit": "contracts/s", "cores": 1, "kind": "oracle",
            "sample": f"512 paths of contracts 0..{i - 1} ({pd} path-dates, {el:.1f} s, numpy FP64, 1 thread), "
                      "rate scaled to the portfolio's path budgets"}


def learned_cpu_baseline(w, budget_s: float = 12.0) -> dict:
    """The oracle's plain Monte Carlo on chunks of 2^13 paths until the time
    budget is used, scaled to the paths a 1e-4 relative standard error
    needs (no control variate: the oracle prices plainly)."""
    import numpy as np
    xs, el, off = [], 0.0, 0
    while el < budget_s:
        dt, x = oracle_run(w, 1 << 13, off)
        el += dt
        xs.append(x)
        off += 1 << 13
    x = np.concatenate(xs)
    need = (x.std() / abs(x.mean()) / TARGET_REL_SE) ** 2
    return {"value": (len(x) / el) / need, "unit": "contracts/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(x)} paths of the contract ({el:.1f} s, numpy FP64, 1 thread), plain MC rate "
                      "scaled to the paths a 1e-4 relative standard error needs"}


def run_portfolio(args):
    items = W.portfolio()
    if args.impl == "reference":
        return portfolio_reference(args, items)
    import numpy as np
    import torch
    import paper_2108_03076_gb300 as pc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        from paper_2108_03076_gb300 import build
        build.build()
    if ws > 1:
        dist.barrier()
    mine = items[rank::ws]          # contracts are independent: shard them
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = pc.pc_create(local, stream.cuda_stream)
    # the costliest contracts on their run-time specialised kernels
    pc.pc_set_jit(ctx, not args.interpret)
    models, contracts, programs = [], [], []
    for it in mine:
        s = it.market
        models.append(pc.pc_model_create(ctx, s.S0, s.sigma, s.corr, s.r, s.days))
        w_, k_ = pc.pc_assemble(it.il_text)
        programs.append((w_, k_, it.tparams))
        contracts.append(pc.pc_load_payoff(ctx, w_, k_, it.tparams, 0, 1))
    n_paths = [it.n_paths for it in mine]
    plan = pc.pc_batch_create(models, contracts, n_paths, PORTFOLIO_SEED)
    pc.pc_batch_tune(plan, 2)
    binfo = pc.pc_batch_query(plan)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        pc.pc_batch_launch(plan)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            pc.pc_batch_launch(plan)
            b.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t_dev = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    price, se = pc.pc_batch_results(plan, len(mine))

    # the other arrangement, timed beside it: one launch of the kernel for
    # every underlying count instead of one launch per group
    pc.pc_batch_set_single_launch(plan, True)
    pc.pc_batch_tune(plan, 2)
    sinfo = pc.pc_batch_query(plan)
    s_ms = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pc.pc_batch_launch(plan)
        b.record(stream)
        torch.cuda.synchronize()
        s_ms.append(a.elapsed_time(b))
    s_price, _ = pc.pc_batch_results(plan, len(mine))
    single = {"ms_per_step": statistics.median(s_ms), "block": sinfo.config.block,
              "unit_split": sinfo.config.unit_split, "prices_equal_grouped": bool(np.array_equal(s_price, price)),
              "note": "pc_batch_set_single_launch: one persistent launch for every contract, tuned the same way"}
    pc.pc_batch_set_single_launch(plan, False)

    # end to end through the public API: load every program from host
    # memory, price the portfolio in one call, read the prices back
    # (the programs' words held concatenated on the host, as a caller keeps
    # its portfolio; one pc_load_payoffs call loads them all)
    n_e2e = max(2, min(args.e2e_steps, 5))
    pset = pc.ProgramSet(programs)
    ks = pc.pc_load_payoffs(ctx, pset)
    pc.pc_price_batch(models, ks, n_paths, PORTFOLIO_SEED)
    for k in ks:
        pc.pc_contract_destroy(k)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        ks = pc.pc_load_payoffs(ctx, pset)
        pc.pc_price_batch(models, ks, n_paths, PORTFOLIO_SEED)
        for k in ks:
            pc.pc_contract_destroy(k)
    e2e_step = (time.perf_counter() - t0) / n_e2e

    if ws > 1:
        t = torch.tensor([t_dev, e2e_step], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev, e2e_step = float(t[0]), float(t[1])
    step_s = t_dev / args.steps
    path_dates = sum(it.n_paths * it.market.n for it in items)
    ops = 0
    mufu = 0
    for m, it in zip(models, mine):
        o = alg_ops_per_path(pc.pc_model_query(m))
        ops += o["ops"] * it.n_paths
        mufu += o["mufu"] * it.n_paths
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    clock_hz = 1e6 * float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 128 * clock_hz
    rel = np.abs(se / np.where(price != 0, price, np.nan))
    if rank == 0:
        line = {
            "metric": METRIC, "value": ws * len(mine) / step_s,
            "unit": "contracts/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * step_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": portfolio_config(items, ws),
            "value_note": "contracts priced per second at their own path budgets "
                          "(2^12-2^18); median rel. std-err of those prices below",
            "path_date_evals_per_sec": ws * sum(it.n_paths * it.market.n for it in mine) / step_s,
            "median_rel_stderr": float(np.nanmedian(rel)),
            "path_dates_per_step": path_dates,
            "gpu_launches": args.steps * (binfo.n_groups + binfo.n_specialised),
            "batch": {"groups": binfo.n_groups, "specialised_contracts": binfo.n_specialised,
                      "units": binfo.n_units, "tiles": binfo.n_tiles,
                      "block": binfo.config.block, "unit_split": binfo.config.unit_split,
                      "paths_per_thread": binfo.paths_per_thread, "tuned_ms": binfo.last_ms},
            "single_launch": single,
            "e2e": {"value": ws * len(mine) / e2e_step, "unit": "contracts/s",
                    "h2d_bytes_per_step": int(sum(w_.nbytes + k_.nbytes + 4 * len(tp)
                                                  for (w_, k_, tp) in programs)),
                    "d2h_bytes_per_step": 16 * len(mine) + 40,
                    "note": "pc_load_payoffs (one call for every contract) + pc_price_batch (no graph) + "
                            "pc_contract_destroy per step, host wall clock"},
            "roofline": {"bound": "alu", "achieved": ops / step_s / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Tops/s", "frac": ops / step_s / peak_ops, "traffic": None,
                         "mufu_frac": mufu / step_s / (props.multi_processor_count * 16 * clock_hz),
                         "peak_basis": f"{props.multi_processor_count} SMs x 128 lanes x "
                                       f"{clock_hz / 1e6:.0f} MHz issue (MUFU: x16)"},
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = portfolio_cpu_baseline(items)
        print(json.dumps(line), flush=True)
    pc.pc_batch_destroy(plan)
    for k in contracts:
        pc.pc_contract_destroy(k)
    for m in models:
        pc.pc_model_destroy(m)
    pc.pc_destroy(ctx)
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Pathwise sensitivities: delta and vega of every underlying
# ---------------------------------------------------------------------------


def greeks_oracle_rate(w, budget_s: float) -> tuple:
    """The oracle's pathwise derivatives (oracle.pathwise: payoff and its
    S0 / sigma derivatives per path, every underlying) on chunks of 2^10
    paths until the budget is used: (path-date tangent evaluations per s,
    paths, seconds)."""
    from oracle import il_text
    from oracle import pathwise as OP
    from oracle.paths import Market
    il = il_text.parse(w.il_text)
    mk = Market(**vars(w.market))
    env = {f"${i}": v for i, v in enumerate(w.tparams)}
    done, el = 0, 0.0
    while el < budget_s:
        t = time.perf_counter()
        for g in range(mk.d):
            OP.pathwise(il, mk, env, 0, 1, 1 << 10, w.seed, g, offset=done)
        el += time.perf_counter() - t
        done += 1 << 10
    return mk.d * done * mk.n / el, done, el


def run_greeks(args):
    w = W.GREEKS[args.workload](args.paths) if args.paths > 0 else W.GREEKS[args.workload]()
    spec = w.market
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        greeks_oracle_rate(w, 0.5)
        rate, done, el = greeks_oracle_rate(w, 12.0)
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": greeks_config(w, ws),
                "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"{done} paths x {spec.d} underlyings (central differences of the "
                                           "FP64 payoff on common paths), 1 thread"},
                "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import torch
    import paper_2108_03076_gb300 as pc
    torch.cuda.set_device(local)
    from paper_2108_03076_gb300 import build
    build.build()
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = pc.pc_create(local, stream.cuda_stream)
    model = pc.pc_model_create(ctx, spec.S0, spec.sigma, spec.corr, spec.r, spec.days)
    words, consts = pc.pc_assemble(w.il_text)
    contract = pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
    d = spec.d
    specialised = not args.interpret and pc.pc_verify_payoff(words, consts, w.tparams).n_insn <= pc.JIT_MAX_INSNS
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    interp_ms = None
    if specialised:
        # the interpreting tangent kernel on the same inputs, for comparison
        for _ in range(args.warmup):
            pc.pc_greeks(model, contract, w.n_paths, w.seed, d)
        im = []
        for _ in range(max(3, min(args.steps, 20))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pc.pc_greeks(model, contract, w.n_paths, w.seed, d)
            b.record(stream)
            torch.cuda.synchronize()
            im.append(a.elapsed_time(b))
        interp_ms = statistics.median(im)
        pc.pc_set_jit(ctx, True)   # compiled on the first warm-up call
    for _ in range(args.warmup):
        res = pc.pc_greeks(model, contract, w.n_paths, w.seed, d)
    steps = max(3, min(args.steps, 200))
    ms = []
    with ClockSampler(local) as clk:
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            res = pc.pc_greeks(model, contract, w.n_paths, w.seed, d)      # d tangent launches, blocking
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    t_tan = statistics.median(ms) / 1e3
    price, delta, vega, se = res
    # the adjoint: every underlying's delta and vega from one launch
    v = 1 + 2 * d
    adj_out = torch.zeros(2 * v + 1, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        pc.pc_greeks_adjoint_async(model, contract, w.n_paths, 0, w.seed, 0, adj_out.data_ptr())
    torch.cuda.synchronize()
    ams = []
    with ClockSampler(local) as clk:
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pc.pc_greeks_adjoint_async(model, contract, w.n_paths, 0, w.seed, 0, adj_out.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
            ams.append(a.elapsed_time(b))
    t_step = statistics.median(ams) / 1e3
    sums = adj_out.cpu().numpy()
    adj_mean = sums[0:2 * v:2] / w.n_paths
    adj_se = np.sqrt(np.maximum(0.0, (sums[1:2 * v:2] - w.n_paths * adj_mean ** 2) / (w.n_paths - 1))
                     / w.n_paths)
    # the two methods agree within their standard errors (same paths)
    agree = bool(np.all(np.abs(adj_mean[1:] - np.concatenate([delta, vega]))
                        <= 1e-3 * np.abs(adj_mean[1:]) + 3e-2 * adj_se[1:] + 1e-9))
    # end to end through the public API: load, sensitivities, drop
    t0 = time.perf_counter()
    for _ in range(5):
        k = pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
        pc.pc_greeks_adjoint(model, k, w.n_paths, w.seed, d)
        pc.pc_contract_destroy(k)
    e2e_step = (time.perf_counter() - t0) / 5
    path_dates = w.n_paths * spec.n
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    clock_hz = 1e6 * float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 128 * clock_hz
    ops = alg_ops_per_path(pc.pc_model_query(model))
    prof = profile_record(w, "adjoint")
    traffic = profile_traffic(w, "adjoint")
    line = {
        "metric": METRIC, "value": ws * path_dates / t_step, "unit": UNIT, "n_gpus": ws, "steps": steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**greeks_config(w, ws), "kernel": "adjoint (interpreter, one launch)"},
        "value_note": "path-dates per second with the price and every underlying's delta and vega "
                      "(one adjoint launch per step)",
        "price": float(adj_mean[0]), "delta": list(adj_mean[1:1 + d]), "vega": list(adj_mean[1 + d:]),
        "stderr": list(adj_se),
        "tangent": {"ms_per_step": 1e3 * t_tan, "launches_per_step": d,
                    "kernel": "specialised to the program (run-time compiled, NVRTC)" if specialised
                    else "interpreter",
                    "interpreter_ms_per_step": interp_ms, "value": ws * path_dates / t_tan,
                    "delta": list(delta), "vega": list(vega), "agrees_with_adjoint": agree},
        "adjoint_speedup_over_tangent": t_tan / t_step,
        "gpu_launches": steps,
        "e2e": {"value": ws * path_dates / e2e_step, "unit": UNIT,
                "h2d_bytes_per_step": int(words.nbytes + consts.nbytes + 4 * len(w.tparams)),
                "d2h_bytes_per_step": 8 * (2 * v + 1),
                "note": "pc_load_payoff + pc_greeks_adjoint + pc_contract_destroy per step, host wall clock"},
        "roofline": {"bound": "alu", "achieved": ops["ops"] * w.n_paths / t_step / 1e12,
                     "peak": peak_ops / 1e12, "unit": "Tops/s",
                     "frac": ops["ops"] * w.n_paths / t_step / peak_ops, "traffic": traffic,
                     "ncu_max_pipe": prof.get("ncu_max_pipe"),
                     "ncu_max_pipe_frac": prof.get("ncu_max_pipe_frac"),
                     "ncu_issue_active": prof.get("ncu_issue_active"),
                     "alg_ops_per_path": ops["ops"],
                     "note": "path generation counted once (the adjoint tape and sweep are not: a "
                             "lower bound)",
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 lanes x "
                                   f"{clock_hz / 1e6:.0f} MHz issue"},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline and ws == 1:
        rate, done, el = greeks_oracle_rate(w, 12.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{done} paths x {d} underlyings ({el:.1f} s, FP64 central "
                                          "differences on common paths, 1 thread)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    pc.pc_contract_destroy(contract)
    pc.pc_model_destroy(model)
    pc.pc_destroy(ctx)


def greeks_config(w, ws) -> dict:
    return {"workload": w.name, "n_paths": w.n_paths, "n_dates": w.market.n, "underlyings": w.market.d,
            "sensitivities": "pathwise delta and vega of every underlying (adjoint: one launch; "
                             "tangent mode, one launch per underlying, timed beside it)",
            "seed": w.seed, "parallelism": f"replicas x{ws}",
            "l2": "flushed between steps by a 256 MiB device write"}


# ---------------------------------------------------------------------------
# Learned control variate: time to a 1e-4 relative standard error
# ---------------------------------------------------------------------------


def learned_config(ws, interpret: bool = False) -> dict:
    return {"workload": LEARNED, "contract": "worst_of_autocall_3u_5d", "target_rel_se": TARGET_REL_SE,
            "kernel": ("interpreter in both arms" if interpret else
                       "specialised to the program (run-time compiled) in both arms"),
            "network": "16-256-256-256-5 softplus, BF16 weights, FP32 accumulation",
            "training_set": "8192 engine-priced states x 128 paths (+6 bumped plans for hedge ratios)",
            "training_steps": 6000, "table_grid": 12,
            "betas": "calibrated once per template on a pilot run with its own seed",
            "parallelism": f"replicas x{ws}",
            "l2": "flushed between steps by a 256 MiB device write"}


def run_learned(args):
    w = W.worst_of_autocall()
    if args.impl == "reference":
        # the oracle, plain Monte Carlo, on a bounded sample; contracts/s at the target
        ws, rank, _ = dist_env()
        if rank != 0:
            return
        dt, x = oracle_run(w, 1 << 14)
        for _ in range(args.warmup):
            oracle_run(w, 1 << 12)
        tot, n = 0.0, 0
        for s_ in range(args.steps):
            dt, x = oracle_run(w, 1 << 13, s_ << 13)
            tot += dt
            n += 1 << 13
        cvx = x.std() / abs(x.mean())
        need = (cvx / TARGET_REL_SE) ** 2
        value = (n / tot) / need
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "contracts/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": learned_config(ws, args.interpret),
                "cpu_baseline": {"value": value, "unit": "contracts/s", "cores": 1, "kind": "oracle",
                                 "sample": "8192 paths per step, plain MC rate scaled to the paths a "
                                           "1e-4 relative standard error needs"},
                "e2e": {"value": value, "unit": "contracts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import torch
    import paper_2108_03076_gb300 as pc
    from paper_2108_03076_gb300 import learned_cv as LCV
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2108_03076_gb300 import build
    build.build()
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = pc.pc_create(local, stream.cuda_stream)
    # both arms on the same evaluator: the plain pricing kernel and the
    # control-variate kernel specialised to the program, or both interpreted
    pc.pc_set_jit(ctx, not args.interpret)
    spec = w.market
    model = pc.pc_model_create(ctx, spec.S0, spec.sigma, spec.corr, spec.r, spec.days)
    words, consts = pc.pc_assemble(w.il_text)
    contract = pc.pc_load_payoff(ctx, words, consts, w.tparams, 0, 1)
    if not args.interpret:
        pc.pc_jit_compile(model, contract)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    t0 = time.perf_counter()
    data = LCV.engine_training_set(ctx, 8192, 128, 0x7A1)
    t_data = time.perf_counter() - t0
    net = LCV.LearnedCV(ctx, seed=5)
    a, b = ev(), ev()
    a.record(stream)
    net.train(data, 6000)
    b.record(stream)
    torch.cuda.synchronize()
    t_train = a.elapsed_time(b) / 1e3
    # betas fixed once for the template (a pilot run on its own seed): any
    # fixed betas keep the estimate unbiased
    betas = net.calibrate(model, contract)
    # the first build sizes the network's scratch and captures the build;
    # pricing rebuilds into the same buffer (a replay)
    desc, tabs = net.tables(model)
    tt = []
    for _ in range(5):
        a, b = ev(), ev()
        a.record(stream)
        net.tables(model, out=tabs, asynchronous=True)
        b.record(stream)
        torch.cuda.synchronize()
        tt.append(a.elapsed_time(b))
    t_tables = statistics.median(tt) / 1e3
    # variances on an independent run: plain, first-order hedge, with second order
    VS = 0x5EED7001
    d1, t1 = net.tables(model, gamma=False)   # same tables, first-order control only
    (_, s_delta), (pp, sp) = pc.pc_price_cv(model, contract, d1, t1.data_ptr(), 1 << 18, VS)
    (_, s_gamma), _ = pc.pc_price_cv(model, contract, desc, tabs.data_ptr(), 1 << 18, VS)
    n_plain = int(math.ceil((sp * math.sqrt(1 << 18) / (TARGET_REL_SE * abs(pp))) ** 2))
    n_for = lambda s_: int(math.ceil((s_ * math.sqrt(1 << 18) / (TARGET_REL_SE * abs(pp))) ** 2))  # noqa: E731

    def cv_ms(dsc, tb, n):
        for _ in range(2):
            pc.pc_price_cv(model, contract, dsc, tb.data_ptr(), n, w.seed)
        ts = []
        for _ in range(5):
            a, b = ev(), ev()
            a.record(stream)
            pc.pc_price_cv(model, contract, dsc, tb.data_ptr(), n, w.seed)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    # the arm that reaches the target in less GPU time: the second-order
    # term removes more variance, the first-order kernel is cheaper per path
    arm_ms = {"first_order": cv_ms(d1, t1, n_for(s_delta)), "second_order": cv_ms(desc, tabs, n_for(s_gamma))}
    if arm_ms["first_order"] <= arm_ms["second_order"]:
        desc, tabs = d1, t1
    scv_b = s_delta if desc is d1 else s_gamma
    n_cv = n_for(scv_b)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    gamma = bool(desc.use_gamma)
    for _ in range(args.warmup):
        pc.pc_price_async(model, contract, n_plain, 0, w.seed, 0, out.data_ptr())
        dstep, _ = net.tables(model, gamma=gamma, out=tabs, asynchronous=True)
        pc.pc_price_cv(model, contract, dstep, tabs.data_ptr(), n_cv, w.seed)
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 50))
    tp_ms, tc_ms, res = [], [], None
    with ClockSampler(local) as clk:
        for _ in range(steps):
            flush.zero_()
            a, b = ev(), ev()
            a.record(stream)
            pc.pc_price_async(model, contract, n_plain, 0, w.seed, 0, out.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
            tp_ms.append(a.elapsed_time(b))
            flush.zero_()
            # one control-variate step: the tables from the network (enqueued,
            # delta0 left on the device) and the pricing, in one timed window
            a, b = ev(), ev()
            a.record(stream)
            dstep, _ = net.tables(model, gamma=gamma, out=tabs, asynchronous=True)
            res = pc.pc_price_cv(model, contract, dstep, tabs.data_ptr(), n_cv, w.seed)
            b.record(stream)
            torch.cuda.synchronize()
            tc_ms.append(a.elapsed_time(b))
    sums = out.cpu().numpy()
    plain_price = sums[0] / n_plain
    plain_se = math.sqrt(max(0.0, (sums[1] - n_plain * plain_price ** 2) / (n_plain - 1)) / n_plain)
    (cv_price, cv_se), _ = res
    t_plain = statistics.median(tp_ms) / 1e3
    t_cv = statistics.median(tc_ms) / 1e3
    # e2e through the public API: tables from the trained network + priced to the target
    t2 = torch.empty_like(tabs)
    for _ in range(2):
        d2, t2 = net.tables(model, gamma=gamma, out=t2, asynchronous=True)
        pc.pc_price_cv(model, contract, d2, t2.data_ptr(), n_cv, w.seed)
    t0 = time.perf_counter()
    for _ in range(5):
        d2, t2 = net.tables(model, gamma=gamma, out=t2, asynchronous=True)
        pc.pc_price_cv(model, contract, d2, t2.data_ptr(), n_cv, w.seed)
    e2e = (time.perf_counter() - t0) / 5
    # surrogate: the network's value at the spot
    x = LCV.features(np.zeros((1, 3)), np.zeros(1, bool), np.zeros(1), 5, np.array(spec.sigma)[None, :], 0.5,
                     spec.r, np.ones(1), 0.05, 1.0, 0.6)
    surrogate = float(net.predict(x)[0, 0])
    line = {
        "metric": METRIC, "value": ws / t_cv, "unit": "contracts/s", "n_gpus": ws, "steps": steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_cv, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 paths, bf16 network", "data": "synthetic",
        "config": learned_config(ws, args.interpret),
        "value_note": "contracts priced per second at a 1e-4 relative standard error with the learned "
                      "control variate (hedge tables from the network + control-variate pricing)",
        "plain_mc": {"contracts_per_sec": ws / t_plain, "paths": n_plain, "ms": 1e3 * t_plain,
                     "price": plain_price, "stderr": plain_se},
        "learned_cv": {"paths": n_cv, "ms_step": statistics.median(tc_ms), "ms_tables": 1e3 * t_tables,
                       "price": cv_price, "stderr": cv_se,
                       "second_order_term": bool(desc.use_gamma), "beta": desc.beta, "beta2": desc.beta2,
                       "variance_ratio": (sp / scv_b) ** 2,
                       "variance_ratio_first_order_only": (sp / s_delta) ** 2,
                       "arm_pricing_ms": arm_ms},
        "gpu_time_ratio_plain_over_cv": t_plain / t_cv,
        "training": {"data_s_wall": t_data, "train_s_gpu": t_train, "samples": len(data.x)},
        "surrogate": {"value": surrogate, "mc_price": plain_price,
                      "rel_error": abs(surrogate - plain_price) / abs(plain_price)},
        # per step one plain launch and the control-variate step (the fused
        # table build, the slopes, the pricing), plus the five timed table
        # builds (2 kernels each)
        "gpu_launches": steps * 4 + 5 * 2,
        "e2e": {"value": ws / e2e, "unit": "contracts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 48,
                "note": "pc_cv_tables_async + pc_price_cv on resident model/contract, host wall clock"},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = learned_cpu_baseline(w)
    print(json.dumps(line), flush=True)
    net.close()
    pc.pc_contract_destroy(contract)
    pc.pc_model_destroy(model)
    pc.pc_destroy(ctx)

if __name__ == "__main__":
    main()
