#!/usr/bin/env python
"""Benchmark of the cache-blocked state-vector simulator on GB300.

Workload (default): quantum-volume circuit, n = 30 qubits, depth 30 (450 Haar SU(4) gates),
complex64 state (8 GiB), chunk c = 12 gathered with 5 pinned bits, tensor-core register groups,
look-ahead chunk choice (the paper's rule is timed alongside).  One step = build the gate
records, plan the cache blocking (host), reset the state to |0..0>, apply the circuit on the
cache-blocked path, and read the norm back.  Metric: gates per second (higher is better), plus effective HBM bandwidth
= (blocking sweeps + permutation sweeps) x 2 x 2^n x 8 B / time.

Prints ONE JSON line on rank 0.  --impl reference times the CPU oracle on a bounded sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gates/s (cache-blocked path), n=30 complex64 quantum volume"
PEAK_FALLBACK_GBS = 6800.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return PEAK_FALLBACK_GBS, "fallback"


def _workload(name):
    import circuitgen as cg
    w = dict(cg.WORKLOADS[name])
    w["desc"] = cg.build(name)
    return w


# ------------------------------------------------------------------ clock sampling
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ distributed helpers
def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class _Barrier:
    """Rank synchronisation for replica runs: a barrier and a max over ranks (timings only; the
    simulation itself exchanges nothing).  NCCL on GPUs; gloo for host-only use."""

    def __init__(self, world, device, backend: str = "nccl"):
        self.world = world
        self.pg = None
        self.backend = backend
        if world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=device)
            else:
                dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device="cuda" if self.backend == "nccl" else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------ CPU oracle timing
def cpu_oracle_rate(w, budget_s: float = 12.0, max_gates: int = 60):
    """Gates/s of the CPU oracle (complex128, all host cores) on a bounded prefix of the workload:
    gates are applied one by one until `budget_s` seconds of work or `max_gates` gates."""
    from oracle import sim
    n = w["n"]
    state = sim.basis_state(n, 0)
    done = 0
    t0 = time.perf_counter()
    for g in w["desc"][:max_gates]:
        sim.apply(state, n, [g])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    del state
    return done / dt, done, dt, sim.num_threads()


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    w = _workload(args.workload)
    from oracle import sim
    n = w["n"]
    per_step = max(1, args.ref_gates_per_step)
    state = sim.basis_state(n, 0)
    gates = w["desc"]
    pos = 0

    def step():
        nonlocal pos
        for _ in range(per_step):
            sim.apply(state, n, [gates[pos % len(gates)]])
            pos += 1

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    rate = args.steps * per_step / dt
    sample = (f"{per_step} gates per step of the n={n} workload in complex128 (first "
              f"{args.steps * per_step + args.warmup * per_step} gates incl. warm-up), one pass per gate")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "gates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(w),
        "cpu_baseline": {"value": rate, "unit": "gates/s", "cores": sim.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_batch(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import circuitgen as cg
    ns, descs = cg.build_batch(args.workload)
    budget = max(1.0, min(20.0, args.cpu_budget / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_batch_rate(ns, descs, budget)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rate, cores, sample = cpu_oracle_batch_rate(ns, descs, budget)
        rates.append(rate)
    dt = time.perf_counter() - t0
    rate = statistics.median(rates)
    line = {
        "impl": "reference", "metric": BATCH_METRIC, "value": rate, "unit": "state-gates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": rate, "unit": "state-gates/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": "state-gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(w):
    return {"workload": f"{args_workload_name(w)}", "n": w["n"], "gates": len(w["desc"]), "chunk_bits": w["c"],
            "gather_pinned": w.get("pinned"), "state": "complex64", "l2": "state 8 GiB >> 129 MB L2 (no flush needed)"}


def args_workload_name(w):
    kinds = {"quantum_volume": "quantum volume", "random_layers": "random layers", "qft": "QFT"}
    depth = f" depth {w['depth']}" if "depth" in w else ""
    return f"{kinds[w['kind']]} n={w['n']}{depth}, {len(w['desc'])} gates, complex64, chunk c={w['c']}"


# sources a kernel's binary depends on (the kernel file first)
_KERNEL_SOURCES = {
    "k_block.cu": ["k_block.cu", "block_core.cuh", "ptx.cuh", "sv_internal.h"],
    "k_batch.cu": ["k_batch.cu", "block_core.cuh", "ptx.cuh", "sv_internal.h"],
}


def kernel_source_sha(kernel_src: str) -> str:
    csrc = os.path.join(ROOT, os.path.dirname(kernel_src))
    h = hashlib.sha256()
    for name in _KERNEL_SOURCES.get(os.path.basename(kernel_src), [os.path.basename(kernel_src)]):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_for(kernel_src: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    sources of the kernel; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    sha = kernel_source_sha(kernel_src)
    e = d.get(workload, {}).get(os.path.basename(kernel_src))
    if not e or e.get("source_sha") != sha:
        return None
    return e.get("dram_bytes_per_launch")


def _per_gate(sv, st, desc, stream, args, sweep_bytes):
    import torch
    G = len(desc)
    gates = sv.make_gates(desc)
    st.init_basis(0)
    st.apply(gates)
    st.synchronize()
    pg_steps = max(1, min(2, args.steps))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(pg_steps):
        st.init_basis(0)
        st.apply(gates)
        st.norm2()
    e1.record(stream)
    torch.cuda.synchronize()
    pg_ms = e0.elapsed_time(e1) / pg_steps
    s = st.stats()
    per_gate = {"gates_per_s": G / (pg_ms / 1000.0), "ms_per_step": pg_ms,
                "effective_GBs": G * sweep_bytes / (pg_ms / 1000.0) / 1e9,
                "kernel_GBs": G * sweep_bytes / (s.ms_gate / 1000.0) / 1e9 if s.ms_gate else None}
    return per_gate, pg_ms


# ------------------------------------------------------------------ batched workload
BATCH_METRIC = "state-gates/s (batched persistent launch), 512 noisy trajectories n=12..24 + 64 HEA(20) sets, complex64"


def cpu_oracle_batch_rate(ns, descs, budget_s: float):
    """Oracle state-gates/s on the whole batch, extrapolated from a bounded sample: for each
    distinct qubit count, gates of one of its circuits are applied one by one for an equal
    share of `budget_s`; the workload time is sum over states of gates x seconds-per-gate(n)."""
    from oracle import sim
    sizes = sorted(set(ns))
    per_gate_s = {}
    share = budget_s / len(sizes)
    for n in sizes:
        d = descs[ns.index(n)]
        st = sim.basis_state(n, 0)
        done = 0
        t0 = time.perf_counter()
        for g in d:
            sim.apply(st, n, [g])
            done += 1
            if time.perf_counter() - t0 > share:
                break
        per_gate_s[n] = (time.perf_counter() - t0) / max(1, done)
    est = sum(len(d) * per_gate_s[n] for n, d in zip(ns, descs))
    total = sum(len(d) for d in descs)
    sample = (f"per qubit count {sizes[0]}..{sizes[-1]}: the first gates of one circuit in complex128 for "
              f"{share:.2f} s each; whole-batch time extrapolated as sum(gates x s/gate(n)) = {est:.1f} s")
    return total / est, sim.num_threads(), sample


# Algorithmic FP32 FMAs per amplitude of each gate kind (complex64): a dense 2x2 complex matrix
# costs 4 complex multiply-adds per amplitude pair = 8 real FMAs per amplitude, a dense 4x4 16,
# a diagonal one complex multiply = 4, a permutation (X, CX, SWAP) none.
_FMA_PER_AMP = {"u3": 8, "h": 8, "y": 8, "ry": 8, "unitary1": 8, "x": 0, "z": 4, "rz": 4, "cz": 4, "cp": 4,
                "cx": 0, "swap": 0}


def _algorithmic_fma(ns, descs):
    tot = 0.0
    for n, d in zip(ns, descs):
        per = 0
        for kind, qubits, _ in d:
            if kind == "unitary":
                per += 8 if len(qubits) == 1 else 16
            else:
                per += _FMA_PER_AMP[kind]
        tot += float(per) * float(1 << n)
    return tot


def _fp32_peak_tflops():
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def run_batch(args):
    import numpy as np
    import torch
    import circuitgen as cg

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    bar = _Barrier(world, torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    bar.barrier()
    import paper_2102_02957_gb300 as sv

    ns, descs = cg.build_batch(args.workload)
    G = sum(len(d) for d in descs)
    gates = [sv.make_gates(d) for d in descs]
    stream = torch.cuda.Stream()
    states = [sv.StateVector(n, "c64", stream=stream) for n in ns]
    base = {} if not args.chunk_bits else dict(chunk_bits=args.chunk_bits)
    if args.planner == "lookahead":
        base["lookahead"] = 1
    base["use_tc"] = int(args.batch_tc)
    if args.chunk_bits:
        best, tune_ms = dict(base), None
    else:
        best, tune_ms = sv.batch_tune(states, gates, **base)
    b = sv.Batch(states, gates, **best)
    items, sections, nbytes = b.info()

    def step():
        b.run(use_graph=True, from_zero=True)

    for _ in range(args.warmup):
        step()
    b.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    bar.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    b.synchronize()
    torch.cuda.synchronize()
    bar.barrier()
    ck = clocks.stop()
    elapsed_ms = bar.max(e0.elapsed_time(e1))
    ms_step = elapsed_ms / args.steps
    value = world * G * args.steps / (elapsed_ms / 1000.0)
    peak, peak_kind = _peaks()
    achieved = nbytes / (ms_step / 1000.0) / 1e9
    # SIMT sections are bound by FP32 arithmetic (the FMA pipes); with tensor-core sections the
    # arithmetic moves to the tensor pipes and the sweep's bytes are the bound in principle
    flops = 2.0 * _algorithmic_fma(ns, descs)
    alu_peak = _fp32_peak_tflops()
    achieved_tf = flops / (ms_step / 1000.0) / 1e12
    alu = {"achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved_tf / alu_peak,
           "peak_source": "derived: SMs x 128 FP32 FMA lanes x 2 flops x max SM clock (MEASURED_PEAKS.json)",
           "algorithmic_flops_per_launch": flops}
    hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": nbytes}
    main, other = (hbm, alu) if best.get("use_tc") else (alu, hbm)
    roofline = dict(main, bound="hbm" if best.get("use_tc") else "alu", kernel="k_batch",
                    traffic=_traffic_for("paper_2102_02957_gb300/csrc/k_batch.cu", args.workload), launch_ms=ms_step,
                    other={"bound": "alu" if best.get("use_tc") else "hbm", **other})
    norms = [s.norm2() for s in states[:: max(1, len(states) // 16)]]

    # the same circuits one state after another on the single-state blocked path
    seq_ms = None
    if not args.no_per_gate:
        plans = [sv.Plan(n, g, chunk_bits=13, gather_pinned=4) for n, g in zip(ns, gates)]
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for st, g, p in zip(states, gates, plans):
            st.init_basis(0)
            st.apply(g, p)
        s1.record(stream)
        torch.cuda.synchronize()
        seq_ms = s0.elapsed_time(s1)

    # end to end through the public API: gate records on the host in, batch built (plan + program
    # upload), run, every state's norm read back
    e2e = None
    if not args.no_e2e:
        def e2e_step():
            bb = sv.Batch(states, gates, **best)
            bb.run(use_graph=False, from_zero=True)
            out = [s.norm2() for s in states]
            bb.close()
            return out
        e2e_step()
        k2 = max(1, min(3, args.steps))
        torch.cuda.synchronize()
        bar.barrier()
        t0 = time.perf_counter()
        for _ in range(k2):
            e2e_step()
        dt = bar.max(time.perf_counter() - t0)
        e2e = {"value": world * G * k2 / dt, "unit": "state-gates/s",
               "h2d_bytes_per_step": int(sum(g.nbytes for g in gates)), "d2h_bytes_per_step": 8 * len(states),
               "ms_per_step": 1000 * dt / k2}

    b.close()
    for st in states:
        st.close()
    torch.cuda.synchronize()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, cores, sample = cpu_oracle_batch_rate(ns, descs, args.cpu_budget)
        cpu = {"value": rate, "unit": "state-gates/s", "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        line = {
            "metric": BATCH_METRIC, "value": value, "unit": "state-gates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {len(ns)} states, n={min(ns)}..{max(ns)}, {G} gates, "
                                   f"{sum(2 ** n for n in ns) * 8 / 2 ** 30:.1f} GiB complex64",
                       "chunk_bits": best.get("chunk_bits"), "planner": "lookahead" if best.get("lookahead") else "rule",
                       "tensor_cores": bool(best.get("use_tc")),
                       "tuned_ms": tune_ms, "work_items": items,
                       "sections": sections, "graph": True, "from_zero": True,
                       "l2": "10 GiB of states >> 129 MB L2 (no flush needed)"},
            "roofline": roofline, "sequential_blocked_ms": seq_ms,
            "speedup_vs_sequential": (seq_ms / ms_step) if seq_ms else None,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": ck, "gpu_launches": 1, "norms_sampled": norms,
        }
        print(json.dumps(line), flush=True)
    bar.close()
    return 0


# ------------------------------------------------------------------ cost model
def _train_cost_model(sv, st, w, plan_opts):
    """Collect section timings of two circuits of the workload's family (same size, other seeds)
    under the paper's rule and under random candidate choices, and train the network on them."""
    import circuitgen as cg
    t0 = time.perf_counter()
    n = w["n"]
    fam = {"quantum_volume": lambda s: cg.quantum_volume(n, w.get("depth", 30), s),
           "random_layers": lambda s: cg.random_layers(n, w.get("depth", 30), s),
           "qft": lambda s: cg.qft(n)}[w["kind"]]
    cm = sv.CostModel(17)
    opts = [dict(plan_opts)]
    for k, seed in enumerate((1001, 1002)):
        g = sv.make_gates(fam(seed))
        cm.collect(st, g, opts, policy_seed=0)
        cm.collect(st, g, opts, policy_seed=5000 + k)
    mse = cm.train(epochs=400, batch=64, lr=2e-3, seed=3)
    info = {"samples": cm.num_samples(), "train_mse_log_us": mse, "seconds": time.perf_counter() - t0,
            "trained_on": f"{w['kind']} n={n} seeds 1001-1002, rule and random candidate choices"}
    return cm, info


# ------------------------------------------------------------------ main GPU benchmark
def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    bar = _Barrier(world, torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    bar.barrier()
    import paper_2102_02957_gb300 as sv

    w = _workload(args.workload)
    if args.chunk_bits:
        w["c"] = args.chunk_bits
    n, c, desc = w["n"], w["c"], w["desc"]
    G = len(desc)
    pinned = args.gather_pinned if args.gather_pinned >= 0 else w.get("pinned", 4)
    w["pinned"] = pinned
    plan_opts = dict(chunk_bits=c, seg_bits=args.seg_bits, gather_pinned=pinned, use_tc=int(args.tc))
    stream = torch.cuda.Stream()
    st = sv.StateVector(n, "c64", stream=stream)
    sweep_bytes = 2.0 * (1 << n) * 8

    # learned cost model (steered planner): trained before the timed region on section timings of
    # circuits of the same family and size with other seeds
    model, model_info = None, None
    if args.planner == "steered":
        model, model_info = _train_cost_model(sv, st, w, plan_opts)
    if args.planner == "lookahead":
        plan_opts["lookahead"] = 1
    st.set_profiling(True)

    rule_opts = {k: v for k, v in plan_opts.items() if k != "lookahead"}

    def step(use_model=True):
        gates = sv.make_gates(desc)
        plan = (sv.Plan(n, gates, model=model, **plan_opts) if use_model
                else sv.Plan(n, gates, **rule_opts))
        st.init_basis(0)
        st.apply(gates, plan)
        nrm = st.norm2()
        return nrm, plan

    for _ in range(args.warmup):
        step()
    st.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    bar.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    ms_block = ms_perm = 0.0
    n_block = n_perm = launches = 0
    norm_last = None
    for _ in range(args.steps):
        norm_last, plan = step()
        s = st.stats()
        ms_block += s.ms_block
        ms_perm += s.ms_permute
        n_block += s.sweeps_block
        n_perm += s.sweeps_permute
        launches += s.kernel_launches + 2  # + init (set-one kernel) + norm reduction
    t_end.record(stream)
    torch.cuda.synchronize()
    bar.barrier()
    ck = clocks.stop()
    elapsed_ms = bar.max(t_start.elapsed_time(t_end))
    ms_step = elapsed_ms / args.steps
    value = world * G * args.steps / (elapsed_ms / 1000.0)
    info = plan.info()
    sweeps_per_step = info.n_blocks + info.n_swap_rounds + info.n_unpermute_rounds
    eff_gbs = sweeps_per_step * sweep_bytes / (ms_step / 1000.0) / 1e9
    peak, peak_kind = _peaks()

    blk_ms = ms_block / max(1, n_block)
    perm_ms = ms_perm / max(1, n_perm)
    blk_gbs = sweep_bytes / (blk_ms / 1000.0) / 1e9
    perm_gbs = sweep_bytes / (perm_ms / 1000.0) / 1e9 if n_perm else None
    dominant = "k_block" if ms_block >= ms_perm else "k_permute"
    dom_src = "paper_2102_02957_gb300/csrc/k_block.cu" if dominant == "k_block" else \
        "paper_2102_02957_gb300/csrc/k_permute.cu"
    achieved = blk_gbs if dominant == "k_block" else perm_gbs
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                "traffic": _traffic_for(dom_src, args.workload),
                "algorithmic_bytes_per_launch": sweep_bytes,
                "launch_ms": blk_ms if dominant == "k_block" else perm_ms,
                "k_block": {"launches_per_step": info.n_blocks, "ms": blk_ms, "GBs": blk_gbs,
                            "share": ms_block / (ms_block + ms_perm)},
                "k_permute": {"launches_per_step": info.n_swap_rounds + info.n_unpermute_rounds, "ms": perm_ms,
                              "GBs": perm_gbs, "share": ms_perm / (ms_block + ms_perm)}}

    # the paper's rule-based planner on the same workload, for comparison with the steered one
    rule = None
    if args.planner != "rule":
        rule_info = None
        for _ in range(1):
            step(use_model=False)
        torch.cuda.synchronize()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        k_rule = max(1, min(2, args.steps))
        r0.record(stream)
        for _ in range(k_rule):
            _, rplan = step(use_model=False)
        r1.record(stream)
        torch.cuda.synchronize()
        rule_info = rplan.info()
        rule = {"ms_per_step": r0.elapsed_time(r1) / k_rule, "sections": rule_info.n_blocks,
                "gates_per_s": G / (r0.elapsed_time(r1) / k_rule / 1000.0)}

    # plain per-gate GPU path on the same workload (the paper's baseline)
    per_gate = None
    pg_ms = float("nan")
    if not args.no_per_gate:
        per_gate, pg_ms = _per_gate(sv, st, desc, stream, args, sweep_bytes)

    # end to end through the C ABI with host buffers: every step uploads its input state from
    # pinned host memory, builds its gate records and plan on the host, applies the circuit and
    # downloads its output state.  Two states on two streams take the steps in turn, so one step's
    # copies over the host link overlap the other's kernels (a serving pipeline); the time is the
    # wall clock over k2 steps from an idle device to the last output in host memory.
    e2e = None
    st.close()
    if not args.no_e2e:
        h_in = torch.zeros(2 << n, dtype=torch.float32).pin_memory()
        h_in[0] = 1.0
        # three states in rotation: step i's upload (state i % 3) can run while step i - 1's
        # download (another state) is still in flight, the link carrying both directions at once
        n_rot = 3
        h_out = [torch.empty(2 << n, dtype=torch.float32).pin_memory() for _ in range(n_rot)]
        e_streams = [torch.cuda.Stream() for _ in range(n_rot)]
        e_states = [sv.StateVector(n, "c64", stream=s) for s in e_streams]
        # the steps' kernels run one step at a time (each step's apply waits for the previous
        # step's, on another stream), so that the host copies overlap the kernels instead of
        # several states' kernels sharing the GPU while the copies wait
        computed = [torch.cuda.Event() for _ in range(n_rot)]

        def e2e_step(i):
            k, prev = i % n_rot, (i - 1) % n_rot
            g = sv.make_gates(desc)
            p = sv.Plan(n, g, **plan_opts)
            e_states[k].set_state_async(h_in.data_ptr())
            e_streams[k].wait_event(computed[prev])
            e_states[k].apply(g, p)
            computed[k].record(e_streams[k])
            e_states[k].get_state_async(h_out[k].data_ptr())

        for i in range(n_rot):
            e2e_step(i)
        for s in e_states:
            s.synchronize()
        # the host link's rate on this machine, for reading the end-to-end number (untimed)
        link = {}
        for name, fn in (("h2d_GBs", lambda: e_states[0].set_state_async(h_in.data_ptr())),
                         ("d2h_GBs", lambda: e_states[0].get_state_async(h_out[0].data_ptr()))):
            l0 = torch.cuda.Event(enable_timing=True)
            l1 = torch.cuda.Event(enable_timing=True)
            l0.record(e_streams[0])
            fn()
            l1.record(e_streams[0])
            l1.synchronize()
            link[name] = (8 << n) / (l0.elapsed_time(l1) / 1000.0) / 1e9
        k2 = max(2, min(6, 2 * args.steps))
        torch.cuda.synchronize()
        bar.barrier()
        t0 = time.perf_counter()
        for i in range(k2):
            e2e_step(i)
        for s in e_states:
            s.synchronize()
        dt = bar.max(time.perf_counter() - t0)
        e2e = {"value": world * G * k2 / dt, "unit": "gates/s", "h2d_bytes_per_step": int((2 << n) * 4),
               "d2h_bytes_per_step": int((2 << n) * 4), "ms_per_step": 1000 * dt / k2,
               "pipeline": "3 states on 3 streams in rotation, kernels of one step at a time: uploads and downloads of other steps overlap each step's kernels",
               "host_link": link}
        out0 = h_out[(k2 - 1) % n_rot][:2].numpy().copy()
        for s in e_states:
            s.close()
        del h_in, h_out
        _ = out0

    torch.cuda.synchronize()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, done, dt, cores = cpu_oracle_rate(w, budget_s=args.cpu_budget)
        cpu = {"value": rate, "unit": "gates/s", "cores": cores, "kind": "oracle",
               "sample": f"first {done} gates of the same workload applied to an n={n} complex128 state "
                         f"({dt:.1f} s, one pass per gate)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(w),
            "effective_hbm_GBs": eff_gbs, "effective_hbm_frac": eff_gbs / peak,
            "sweeps_per_step": {"blocks": info.n_blocks, "swap_rounds": info.n_swap_rounds,
                                "reorder_rounds": info.n_unpermute_rounds},
            "planner": args.planner, "cost_model": model_info, "rule_planner": rule,
            "per_gate": per_gate, "speedup_vs_per_gate": (pg_ms / ms_step) if per_gate else None,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": ck,
            "gpu_launches": launches, "norm": norm_last,
        }
        print(json.dumps(line), flush=True)
    bar.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="qv30")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-gate", action="store_true")
    ap.add_argument("--seg-bits", type=int, default=4, help="register-group width inside a chunk (4 or 5)")
    ap.add_argument("--chunk-bits", type=int, default=0, help="override the workload's chunk bits")
    ap.add_argument("--tc", type=int, default=1, help="1: fused register groups on the tensor cores (3xTF32)")
    ap.add_argument("--batch-tc", type=int, default=1,
                    help="batched workloads: 1 runs sections of >= 11 chunk bits on the tensor cores (128-thread CTAs)")
    ap.add_argument("--gather-pinned", type=int, default=-1,
                    help="0: chunk_swap passes (the paper's layout moves); p > 0: gathered chunks with p pinned low "
                         "bits; default: the workload's (5 for quantum volume: 256-byte tensor-copy boxes)")
    ap.add_argument("--planner", default="lookahead", choices=["rule", "lookahead", "steered"],
                    help="rule: the paper's chunk choice; lookahead: the chunk that takes the most gates; "
                         "steered: the learned cost model picks among both and smaller chunks (trained before timing)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-gates-per-step", type=int, default=4)
    args = ap.parse_args()
    import circuitgen as cg
    batched = args.workload in cg.BATCH_WORKLOADS
    if args.impl == "reference":
        return run_reference_batch(args) if batched else run_reference(args)
    return run_batch(args) if batched else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
