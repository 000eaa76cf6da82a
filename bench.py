"""Benchmark: exact samples/s of the pilot-wave sampler on one GB300.

Workload (default): noisy QAOA p=2 on the 8x8 grid (64 qubits), two-qubit
depolarizing 1e-3 after every RZZ and amplitude damping 1e-3 on every qubit
after every mixer layer, angles U[0, pi) from seed 3; one step = 10^5 exact
samples drawn in launches of 8192 chains (the sampler's whole hot path: every
layer's Kraus draws, contraction, readout and resampling). Prints one JSON
line: samples/s over the timed steps (device time, inputs resident), the
roofline of the sampler kernel (algorithmic FP32 flops per launch over its
event time against the FP32 FMA rate measured on the device by
pw_device_fma_rate, DRAM bytes per launch from the ncu summary under
profiles/), the FP64 oracle timed on the host cores, the end-to-end rate
through the host-buffer API, the kernel launches of the timed region and the
SM clocks sampled meanwhile. `--impl reference` times the oracle alone: each
of its steps is a bounded sample of the same workload (one chain per host
core), run for real, warm-up steps included.

`--workload grad3reg` measures the QAOA amplitude derivatives instead: the
seeded p=3 random 3-regular instances (n in [20, 48]) whose frontier fits on
chip, K=64 bitstrings per instance drawn by its own sampler, one step = the
exact d amp / d(gamma, beta) of every instance (pw_qaoa_amp_grad); the value
is amplitude gradients (2p-vectors) per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload grid8x8noisy|grid6x6|n12|heavyhex400|grad3reg] [--precision fp32|fp64]
                  [--samples S] [--no-cpu-baseline] [--no-autotune] [--grad-instances N]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "exact samples/s on 1 GB300 (mixed vs plain FP32, same accuracy); TC % of peak"

# arithmetic of each workload's configuration (the 12-qubit one is complex128)
DEFAULT_PRECISION = {"grid6x6": "fp32", "n12": "fp64", "heavyhex400": "fp32", "grid8x8noisy": "fp32",
                     "grad3reg": "fp32"}
# engine of each workload: the 64-qubit noisy grid's 2^16-entry frontiers run
# on the HBM engine (dense passes on the tensor cores), the others on chip
DEFAULT_ENGINE = {"grid8x8noisy": "hbm"}
GEMMS = {"split3": 0, "split2": 1, "bf16": 2, "fp32": 3}   # PW_GEMM_*
ENGINES = {"auto": 0, "onchip": 1, "hbm": 2}                # PW_ENGINE_*


def measured_peaks():
    """HBM GB/s and dense BF16 TFLOP/s measured on the GB300s (the
    driver writes MEASURED_PEAKS.json), else the stated fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "of fallback"
GRAD_K = 64   # bitstrings per instance of the gradient workload


def workload(name):
    import workloads as W
    if name == "grid6x6":
        return W.grid_6x6_p2(), 100000, 4096, "qaoa_p2_grid6x6 (36 qubits, ideal, 10^5 samples, B=4096)"
    if name == "n12":
        return W.maxcut_3reg_n12(), 10000, 256, "qaoa_p1_3reg_n12 (ideal, 10^4 samples, B=256)"
    if name == "heavyhex400":
        return W.heavy_hex_400_p1(), 100000, 16384, "qaoa_p1_heavyhex400 (400 qubits, ideal, 10^5 samples, B=16384)"
    if name == "grad3reg":
        return (None, GRAD_K, 0, "qaoa_p3_3reg_gradients (instances of n in [20, 48] whose frontier fits on chip, "
                                 "K=64 bitstrings each, d amp/d(gamma, beta))")
    if name == "grid8x8noisy":
        return (W.grid_8x8_p2_noisy(), 100000, 8192,
                "qaoa_p2_grid8x8_noisy (64 qubits, depol 1e-3, AD 1e-3, 10^5 samples, B=8192)")
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------ oracle

def _oracle_worker(args):
    name, seed, ids, budget = args
    import workloads as W  # noqa: F401
    from oracle import circuit as OC
    from oracle import sampler as OS
    spec = workload(name)[0]
    ops = OC.qaoa_circuit(spec)
    t0 = time.perf_counter()
    done = 0
    for sid in ids:
        if spec.depol2 > 0 or spec.ad_gamma > 0:
            OS.noisy_sample(spec.n, ops, seed, sid, backend="tn" if spec.n > 16 else "sv")
        elif spec.n <= 16:
            OS.sample_sv(spec.n, ops, seed, [sid])
        else:
            OS.sample_tn(spec.n, ops, seed, sid)
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    return done, time.perf_counter() - t0


def oracle_rate(name, budget_s=20.0, seed=1):
    """Samples/s of the FP64 oracle (naive Alg. 1/2 sampler) on the host cores,
    one chain per worker process (spawned), bounded by budget_s per worker."""
    cores = max(1, min(os.cpu_count() or 1, 16))
    ctx = mp.get_context("spawn")
    jobs = [(name, seed, list(range(w, 10 ** 6, cores)), budget_s) for w in range(cores)]
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    done = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return done / busy, cores, done, wall


def _oracle_chain(args):
    name, seed, sid = args
    from oracle import circuit as OC
    from oracle import sampler as OS
    spec = workload(name)[0]
    ops = OC.qaoa_circuit(spec)
    if spec.depol2 > 0 or spec.ad_gamma > 0:
        OS.noisy_sample(spec.n, ops, seed, sid, backend="tn" if spec.n > 16 else "sv")
    elif spec.n <= 16:
        OS.sample_sv(spec.n, ops, seed, [sid])
    else:
        OS.sample_tn(spec.n, ops, seed, sid)
    return 1


def oracle_steps(name, warmup, steps, seed):
    """The oracle as the reference arm: warmup + steps steps, each a bounded
    sample of the workload (one chain per host core, in a spawned pool); the
    rate is the chains of the timed steps over their wall time."""
    cores = max(1, min(os.cpu_count() or 1, 16))
    ctx = mp.get_context("spawn")
    timed, wall = 0, 0.0
    with ctx.Pool(cores) as pool:
        for k in range(warmup + steps):
            ids = [(name, seed, k * cores + i) for i in range(cores)]
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_chain, ids))
            dt = time.perf_counter() - t0
            if k >= warmup:
                timed += done
                wall += dt
    return timed / wall, cores, timed, wall / max(1, steps) * 1e3


def workload_config(args, world):
    """The `config` of the bench line: the workload alone, identical in both arms."""
    spec, n_samples, B, desc = workload(args.workload)
    if args.samples:
        n_samples = args.samples
    engine = getattr(args, "engine", None) or (DEFAULT_ENGINE.get(args.workload, "onchip")
                                               if args.precision == "fp32" else "onchip")
    return {"workload": desc, "samples_per_step": n_samples, "chains_per_launch": B, "precision": args.precision,
            "engine": engine, "gemm": getattr(args, "gemm", "split3") if engine == "hbm" else None,
            "l2": "flushed (256 MB write) before every timed step",
            "parallelism": f"replicas x{world} (disjoint sample ranges)"}


# ------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)
            self.f.close()

    def summary(self, dev_index):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if not self.proc:
            return out
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != dev_index:
                continue
            rows.append(parts)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        out["sm_mhz"] = statistics.median(sm) if sm else None
        out["sm_max_mhz"] = max(mx) if mx else None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    seen.add(nm)
        out["reasons"] = sorted(seen)
        out["samples"] = len(rows)
        return out


# -------------------------------------------------------------------- ours

def replica_first(rank, n_samples, warmup, steps):
    """First sample id of a replica: every rank draws its own range of sample
    ids (warm-up, timed and end-to-end steps), disjoint from the other
    ranks'; with the counter-based draws each sample is the same as on one
    GPU."""
    return rank * n_samples * (warmup + steps + 1)


def max_over_ranks(value, world, device=None):
    """The largest value over the ranks (the timed region of the slowest)."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    if device is not None and device.type == "cuda":
        t = t.to(device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_2510_24218_gb300 as pw

    spec, n_samples, B, desc = workload(args.workload)
    if args.samples:
        n_samples = args.samples
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prec = pw.PW_PREC_FP64 if args.precision == "fp64" else pw.PW_PREC_FP32
    circ = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas,
                              spec.depol2, spec.ad_gamma)
    eng, gemm = ENGINES[args.engine], GEMMS[args.gemm]
    opts = dict(precision=prec, chains_per_launch=B, engine=eng, gemm=gemm)
    shape = {"tuned": False}
    if args.autotune:
        # the plan shape (readout block size, sweep order, threads per chain)
        # searched on this device before the warm-up; the engine, the
        # arithmetic and the batch stay the workload's
        cache = os.environ.get("PW_AUTOTUNE_CACHE") or os.path.join(tempfile.gettempdir(), "pw_autotune.jsonl")
        opts, trial_rate, hit = pw.pw_autotune(circ, min(n_samples, 16384), cache, torch.cuda.current_stream(dev),
                                               **opts)
        shape = {"tuned": True, "from_cache": hit, "trial_samples_per_s": trial_rate,
                 **{k: opts[k] for k in ("max_block", "order", "threads_per_chain")}}
    plan = pw.pw_plan_build(circ, **opts)
    pst = pw.pw_plan_stats(plan)
    words = (spec.n + 63) // 64
    out = torch.empty((n_samples, words), dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)
    first = replica_first(rank, n_samples, args.warmup, args.steps)

    hbm = pst["engine"] == ENGINES["hbm"]

    def step(i, stats=False, pl=None):
        return pw.pw_sample(pl or plan, args.seed, first + i * n_samples, n_samples, out, None, stream,
                            want_stats=stats)

    launches_per_step = (n_samples + B - 1) // B
    # the roofline's denominator: the FMA rate of this device's CUDA cores,
    # measured by the library's probe kernel (not a nominal figure)
    peak = pw.pw_device_fma_rate(prec, stream)
    near = 0
    for i in range(args.warmup):
        near += step(i, stats=True)["near_boundary"]
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    dense = {"passes": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0}
    clk_path = os.path.join(tempfile.gettempdir(), f"pw_clocks_{os.getpid()}.csv")
    with ClockSampler(clk_path) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            # the HBM engine's dense passes are timed by the library with CUDA
            # events around each GEMM kernel, on this stream (stats requested)
            st = step(args.warmup + i, stats=hbm)
            ev[i][1].record(stream)
            if hbm:
                launches += st["launches"]
                for k in dense:
                    dense[k] += st["dense_" + k]
            else:
                launches += launches_per_step
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms = max_over_ranks(ms, world, dev)
    total = n_samples * args.steps * world
    value = total / (ms / 1e3)

    def rate_of(engine, gemm_kind, steps=2, shape=True):
        """samples/s of the same workload on another engine or arithmetic
        (warm-up call, then `steps` timed steps): the comparison arms (with
        the tuned plan shape, or the plan's default one)."""
        base = opts if shape else dict(precision=prec, chains_per_launch=B)
        p2 = pw.pw_plan_build(circ, **{**base, "engine": engine, "gemm": gemm_kind})
        try:
            step(0, pl=p2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(steps):
                step(1 + i, pl=p2)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return n_samples * steps / (e0.elapsed_time(e1) / 1e3)
        finally:
            pw.pw_plan_destroy(p2)

    arms = {}
    if hbm and rank == 0 and not args.no_arms:
        arms["fp32_simt_same_plan"] = rate_of(ENGINES["hbm"], GEMMS["fp32"])
        arms["onchip_engine"] = rate_of(ENGINES["onchip"], 0, shape=False)
    per_launch_ms = ms / max(1, launches)
    # roofline of the sampler kernel: algorithmic flops of one launch / launch time
    flops_per_launch = pst["flops_per_sample"] * (n_samples / max(1, launches / args.steps))
    achieved = flops_per_launch / (per_launch_ms / 1e3) / 1e12
    clocks = clk.summary(dev.index)

    # e2e: the public host API each step (circuit + plan from host arrays,
    # plan upload, sampling, copy of the samples back to host memory)
    host_out = np.empty((n_samples, words), dtype=np.uint64)
    e2e_times = []
    h2d = 0
    for i in range(max(2, min(args.steps, 5))):
        t0 = time.perf_counter()
        c2 = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, spec.h, spec.p, spec.gammas, spec.betas,
                                spec.depol2, spec.ad_gamma)
        p2 = pw.pw_plan_build(c2, **opts)
        pw.pw_sample_host(p2, args.seed, first + i * n_samples, n_samples, host_out)
        pw.pw_plan_destroy(p2)
        pw.pw_circuit_destroy(c2)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = n_samples * world / statistics.median(e2e_times)
    h2d = _plan_blob_bytes(pw, plan)

    pw.pw_plan_destroy(plan)
    pw.pw_circuit_destroy(circ)
    return dict(value=value, ms=ms, launches=launches, near=near, pst=pst, desc=desc, n_samples=n_samples, B=B,
                achieved=achieved, peak=peak, hbm=hbm, dense=dense, arms=arms, shape=shape, per_launch_ms=per_launch_ms, flops_per_launch=flops_per_launch, clocks=clocks,
                e2e=e2e_value, h2d=h2d, d2h=n_samples * words * 8, wall=t_wall)


# ---------------------------------------------------------- gradient leg

def grad_instances(pw, prec):
    """The seeded p=3 3-regular instances whose frontier fits on chip (the
    parameter-shift gradient runs p(|E| + n) contractions per gradient: the
    wider instances, which the HBM engine can contract, are not timed)."""
    import workloads as W
    out = []
    for spec in W.gradient_instances():
        c = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, None, spec.p, spec.gammas, spec.betas)
        try:
            pw.pw_plan_destroy(pw.pw_plan_build(c, precision=prec, engine=pw.PW_ENGINE_ONCHIP))
            out.append(spec)
        except pw.PwError:
            pass
        finally:
            pw.pw_circuit_destroy(c)
    return out


def _grad_oracle_worker(args):
    names, seed, budget = args
    import workloads as W
    from oracle import gradient as G
    by_name = {s.name: s for s in W.gradient_instances()}
    t0 = time.perf_counter()
    rows = 0
    for j, name in enumerate(names):
        spec = by_name[name]
        G.amp_and_grad_tn(spec, W.random_bitstrings(1, spec.n, seed=seed + j))
        rows += 1
        if time.perf_counter() - t0 > budget:
            break
    return rows, time.perf_counter() - t0


def grad_oracle_rate(names, budget_s=20.0, seed=1):
    """Amplitude gradients/s of the FP64 oracle (generator insertion, each term
    by variable elimination) on the host cores: worker w takes the instances
    names[w], names[w + cores], ... one bitstring each until its budget is
    spent."""
    cores = max(1, min(os.cpu_count() or 1, 16))
    ctx = mp.get_context("spawn")
    jobs = [(names[w::cores] or names[:1], seed + 1000 * w, budget_s) for w in range(cores)]
    with ctx.Pool(cores) as pool:
        res = pool.map(_grad_oracle_worker, jobs)
    done = sum(r[0] for r in res)
    return done / max(r[1] for r in res), cores, done


def run_grad(args, rank, world):
    import numpy as np
    import torch

    import paper_2510_24218_gb300 as pw

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prec = pw.PW_PREC_FP64 if args.precision == "fp64" else pw.PW_PREC_FP32
    specs = grad_instances(pw, prec)
    if args.grad_instances:
        specs = specs[:args.grad_instances]
    stream = torch.cuda.current_stream(dev)
    K = GRAD_K
    bits, grads, amps = [], [], []
    launches_per_step = 0
    flops_per_step = 0.0
    for i, spec in enumerate(specs):
        # the instance's own sampler draws its K bitstrings (inputs of the step)
        c = pw.pw_circuit_qaoa(spec.n, spec.edges, spec.weights, None, spec.p, spec.gammas, spec.betas)
        pl = pw.pw_plan_build(c, precision=prec, engine=pw.PW_ENGINE_ONCHIP)
        amp_flops = pw.pw_plan_stats(pl)["flops_per_amplitude"]
        b = torch.empty((K, (spec.n + 63) // 64), dtype=torch.int64, device=dev)
        pw.pw_sample(pl, args.seed + rank, i * K, K, b, None, stream, want_stats=False)
        pw.pw_plan_destroy(pl)
        pw.pw_circuit_destroy(c)
        bits.append(b)
        grads.append(torch.empty((K, 2 * spec.p, 2), dtype=torch.float64, device=dev))
        amps.append(torch.empty((K, 2), dtype=torch.float64, device=dev))
        terms = spec.p * (len(spec.edges) + spec.n)
        # the amplitudes, one contraction + one accumulation per term, the final sum of the lanes
        launches_per_step += 2 + 2 * terms
        # algorithmic flops: every shifted circuit has the plan structure of the original
        flops_per_step += (1 + terms) * K * amp_flops

    def step(bs, gs, as_):
        for spec, b, g, a in zip(specs, bs, gs, as_):
            pw.pw_qaoa_amp_grad(spec.n, spec.edges, spec.weights, None, spec.p, spec.gammas, spec.betas, b, g,
                                amp_out=a, precision=prec, stream=stream)

    peak = pw.pw_device_fma_rate(prec, stream)
    for _ in range(args.warmup):
        step(bits, grads, amps)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk_path = os.path.join(tempfile.gettempdir(), f"pw_clocks_{os.getpid()}.csv")
    with ClockSampler(clk_path) as clk:
        for i in range(args.steps):
            ev[i][0].record(stream)
            step(bits, grads, amps)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
    value = len(specs) * K * args.steps * world / (ms / 1e3)

    # e2e: bitstrings from pinned host memory, derivatives back to host memory
    h_bits = [b.cpu().pin_memory() for b in bits]
    h_grads = [torch.empty(g.shape, dtype=g.dtype).pin_memory() for g in grads]
    t0 = time.perf_counter()
    d_bits = [hb.to(dev, non_blocking=True) for hb in h_bits]
    step(d_bits, grads, amps)
    for hg, g in zip(h_grads, grads):
        hg.copy_(g, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    h2d = sum(hb.numel() * 8 for hb in h_bits)
    d2h = sum(hg.numel() * 8 for hg in h_grads)
    ns = [s.n for s in specs]
    achieved = flops_per_step * args.steps / (ms / 1e3) / 1e12
    return dict(value=value, ms=ms, launches=launches_per_step * args.steps, clocks=clk.summary(dev.index),
                achieved=achieved, flops_per_step=flops_per_step, peak=peak,
                e2e=len(specs) * K * world / e2e_s, h2d=h2d, d2h=d2h, n_instances=len(specs),
                n_range=[min(ns), max(ns)], finite=bool(all(torch.isfinite(g).all().item() for g in grads)))


KERNEL_SOURCES = ("paper_2510_24218_gb300/csrc/sampler.cu", "paper_2510_24218_gb300/csrc/pw_internal.h",
                  "paper_2510_24218_gb300/csrc/smem_layout.h", "paper_2510_24218_gb300/csrc/planner.cpp")
# the dense GEMM passes of the HBM engine: their kernels, and the planner that
# chooses their tile, row and outer bits
DENSE_SOURCES = ("paper_2510_24218_gb300/csrc/dense.cu", "paper_2510_24218_gb300/csrc/dense.h",
                 "paper_2510_24218_gb300/csrc/pw_internal.h", "paper_2510_24218_gb300/csrc/planner.cpp")
PROFILE_OF = {"grid6x6": "pw_chain_kernel_grid6x6_p2.md", "grid8x8noisy": "pw_chain_kernel_grid8x8_p2_noisy.md",
              "heavyhex400": "pw_chain_kernel_heavyhex400_p1.md",
              "grid8x8noisy_hbm": "dense_tc_kernel_grid8x8_p2_noisy_hbm.md"}


def kernel_sources_sha256(files=KERNEL_SOURCES):
    """sha256 of the kernel's sources with comments and blank space removed:
    it changes with the code, not with its comments."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def profiled_traffic(workload_name, chains_per_launch, algorithmic_bytes=None):
    """DRAM bytes (read + write) of one launch of the profiled kernel, from the
    ncu capture summarised under profiles/, or None when there is none for
    this workload, or the kernel sources have changed since it was taken.
    A summary of the sampler kernel gives the bytes of one launch of the
    captured size (None for another size); a summary of the dense passes
    gives their DRAM bytes per algorithmic byte over all passes of a run,
    scaled here to the algorithmic bytes of the timed launches."""
    name = PROFILE_OF.get(workload_name)
    if name is None:
        return None
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    fields = {}
    for ln in open(path):
        if ":" in ln and ln.startswith("    ") and ln.strip().split(":")[0] in (
                "kernel-sources-sha256", "dram-bytes-per-launch", "chains-per-launch",
                "dram-bytes-per-algorithmic-byte"):
            k, v = ln.strip().split(":", 1)
            fields[k] = v.strip()
    files = DENSE_SOURCES if workload_name.endswith("_hbm") else KERNEL_SOURCES
    if fields.get("kernel-sources-sha256") != kernel_sources_sha256(files):
        return None
    try:
        if "dram-bytes-per-algorithmic-byte" in fields:
            if not algorithmic_bytes:
                return None
            return float(fields["dram-bytes-per-algorithmic-byte"]) * algorithmic_bytes
        if int(fields.get("chains-per-launch", -1)) != chains_per_launch:
            return None
        return float(fields["dram-bytes-per-launch"])
    except (KeyError, ValueError):
        return None


def _plan_blob_bytes(pw, plan):
    # size of the plan tables uploaded to the device (read from the stats:
    # the upload is the only host->device copy of a step)
    return int(pw.pw_plan_stats(plan)["device_bytes"])


def roofline_of(args, r, fma_peak):
    """Roofline of the dominant kernel. HBM engine: the dense GEMM pass
    (dense_tc_kernel / dense_simt_kernel), its algorithmic bytes (every
    frontier entry read and written once) over its event-timed duration
    against the measured HBM copy rate, with its tensor-pipe rate against the
    measured BF16 peak beside it. On-chip engine: the sampler kernel's
    algorithmic FP32 flops over its time against the measured FMA rate."""
    if r["hbm"]:
        hbm_gbs, bf16_tf, note = measured_peaks()
        d = r["dense"]
        gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] else None
        tcf = d["flops"] / (d["ms"] / 1e3) / 1e12 if d["ms"] else None
        tc = args.gemm != "fp32"
        return {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s",
                "frac": gbs / hbm_gbs if gbs else None,
                "traffic": profiled_traffic(args.workload + "_hbm", r["B"], d["bytes"] / max(1, d["passes"])),
                "kernel": "dense_tc_kernel<6,3>" if args.gemm == "split3" else
                          ("dense_simt_kernel<6>" if not tc else f"dense_tc_kernel ({args.gemm})"),
                "launches_timed": d["passes"], "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["passes"]),
                "avg_launch_ms": d["ms"] / max(1, d["passes"]),
                "peak_note": f"{note} HBM copy rate (MEASURED_PEAKS.json)",
                "tensor": ({"achieved": tcf, "peak": bf16_tf, "unit": "TFLOP/s", "frac": tcf / bf16_tf if tcf else None,
                            "note": f"issued BF16 MMA flops of the dense passes (2^W x 2^k complex multiply-adds x "
                                    f"the split's products) over their time, {note} dense BF16 peak"} if tc else None)}
    return {"bound": "alu", "achieved": r["achieved"], "peak": fma_peak, "unit": "TFLOP/s",
            "frac": (r["achieved"] / fma_peak) if fma_peak else None,
            "traffic": profiled_traffic(args.workload, r["B"]) if args.precision == "fp32" else None,
            "kernel": "pw_chain_kernel<float>" if args.precision == "fp32" else "pw_chain_kernel<double>",
            "peak_note": f"of measured: {args.precision.upper()} FMA rate of this device's CUDA cores "
                         "(pw_device_fma_rate probe, best of five ~30 ms launches)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid8x8noisy")
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"],
                    help="default: the workload's own (fp64 for n12, fp32 otherwise)")
    ap.add_argument("--seed", type=int, default=20251203)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--samples", type=int, default=0, help="override samples per step (profiling)")
    ap.add_argument("--grad-instances", type=int, default=0,
                    help="grad3reg: time only the first N fitting instances (profiling)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the plan's default shape (default: search readout block size, sweep order and "
                         "threads per chain with pw_autotune before the warm-up; results cached in "
                         "$PW_AUTOTUNE_CACHE or the temp directory)")
    ap.add_argument("--engine", default=None, choices=list(ENGINES),
                    help="default: the workload's own (hbm for grid8x8noisy, onchip otherwise)")
    ap.add_argument("--gemm", default="split3", choices=list(GEMMS),
                    help="HBM engine: arithmetic of the dense passes (default split3: tensor cores, FP32-equivalent)")
    ap.add_argument("--no-arms", action="store_true", help="skip the comparison arms (FP32 SIMT, on-chip engine)")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = DEFAULT_PRECISION.get(args.workload, "fp32")
    if args.engine is None:
        args.engine = DEFAULT_ENGINE.get(args.workload, "onchip") if args.precision == "fp32" else "onchip"

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    spec, n_samples, B, desc = workload(args.workload)
    if args.workload == "grad3reg":
        return main_grad(args, rank, world, desc)

    if args.impl == "reference":
        # the reference arm of this build is the FP64 CPU oracle, on host cores
        if rank != 0:
            return
        rate, cores, timed, ms_step = oracle_steps(args.workload, args.warmup, args.steps, args.seed)
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "samples/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(args, 1),
                "chains_timed": timed, "extrapolated": False,
                "cpu_baseline": {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
                                 "sample": f"each step is a bounded sample of the workload: {cores} chains, one per "
                                           f"host core (naive Alg. 1/2, FP64); {timed} chains over the "
                                           f"{args.steps} timed steps"},
                "e2e": {"value": rate, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # before the first GPU call (the pool is spawned)
        rate, cores, done, wall = oracle_rate(args.workload, budget_s=args.cpu_budget)
        cpu = {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} chains of the same workload, naive Alg. 1/2 with FP64 "
                         f"{'elimination' if spec.n > 16 else 'state-vector'} amplitudes, ~{args.cpu_budget:.0f} s"}

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    r = run_ours(args, rank, world)
    if rank == 0:
        peak = r["peak"]
        line = {
            "metric": METRIC, "value": r["value"], "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": workload_config(args, world),
            "details": {"amplitudes_per_s": r["value"] * r["pst"]["amps_per_sample"],
                        "engine": args.engine, "gemm": args.gemm if r["hbm"] else None,
                        "plan": {k: r["pst"][k] for k in ("n_slots", "width_bits", "n_blocks", "threads_per_chain",
                                                          "chains_per_cta", "ctas_per_chain", "flops_per_sample",
                                                          "dense_tile_bits", "dense_passes_per_sample",
                                                          "dense_flops_per_sample")},
                        "plan_shape": r["shape"],
                        "near_boundary_draws_in_warmup": int(r["near"]),
                        "comparison_samples_per_s": r["arms"],
                        "mixed_vs_fp32_same_plan": (r["value"] / r["arms"]["fp32_simt_same_plan"]
                                                    if r["arms"].get("fp32_simt_same_plan") else None)},
            "roofline": roofline_of(args, r, peak),
            "cpu_baseline": cpu,
            "e2e": {"value": r["e2e"], "unit": "samples/s", "h2d_bytes_per_step": r["h2d"],
                    "d2h_bytes_per_step": r["d2h"]},
            "gpu_launches": int(r["launches"]),
            "clocks": r["clocks"],
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main_grad(args, rank, world, desc):
    metric = "exact QAOA amplitude gradients/s (d amp/d(gamma, beta), p=3) on 1 GB300"
    import paper_2510_24218_gb300 as pw
    prec = pw.PW_PREC_FP64 if args.precision == "fp64" else pw.PW_PREC_FP32
    # the workload's instance set (host planning only, no device call)
    names = [s.name for s in grad_instances(pw, prec)]
    if args.impl == "reference":
        if rank != 0:
            return
        rate, cores, done = grad_oracle_rate(names, budget_s=max(5.0, args.cpu_budget / 2))
        print(json.dumps({"impl": "reference", "metric": metric, "value": rate, "unit": "gradients/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": desc},
                          "cpu_baseline": {"value": rate, "unit": "gradients/s", "cores": cores, "kind": "oracle",
                                           "sample": f"{done} gradients (one bitstring each) of the same "
                                                     "instances, FP64 generator insertion by elimination"},
                          "e2e": {"value": rate, "unit": "gradients/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, done = grad_oracle_rate(names, budget_s=args.cpu_budget)
        cpu = {"value": rate, "unit": "gradients/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} gradients (one bitstring each) of the same instances, FP64 generator "
                         f"insertion by elimination, ~{args.cpu_budget:.0f} s"}
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    r = run_grad(args, rank, world)
    if rank == 0:
        print(json.dumps({
            "metric": metric, "value": r["value"], "unit": "gradients/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": desc, "instances": r["n_instances"], "n_range": r["n_range"],
                       "bitstrings_per_instance": GRAD_K, "precision": args.precision,
                       "l2": "inputs are a few KB per instance; each contraction re-reads its plan tables",
                       "parallelism": f"replicas x{world}", "all_finite": r["finite"]},
            "roofline": {"bound": "alu", "achieved": r["achieved"], "peak": r["peak"], "unit": "TFLOP/s",
                         "frac": r["achieved"] / r["peak"],
                         "peak_note": f"of measured: {args.precision.upper()} FMA rate of this device's CUDA cores "
                                      "(pw_device_fma_rate probe)",
                         "traffic": None, "kernel": "pw_chain_kernel (amplitude mode)",
                         "flops_per_step": r["flops_per_step"],
                         "note": "step-level: the algorithmic flops of every contraction of the step over the step's "
                                 "time (the contractions of up to 16 lanes overlap, so no per-launch time is taken); "
                                 "host planning and uploads run in parallel with them"},
            "cpu_baseline": cpu,
            "e2e": {"value": r["e2e"], "unit": "gradients/s", "h2d_bytes_per_step": r["h2d"],
                    "d2h_bytes_per_step": r["d2h"]},
            "gpu_launches": int(r["launches"]),
            "clocks": r["clocks"],
        }))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
