#!/usr/bin/env python3
"""Throughput benchmark of the GB300 state-vector simulator.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

A step is one pass of the whole hot path over one synthetic input: set the
register to its basis state, apply the circuit (planner path: shared-memory
tile passes), and read the per-qubit expectations <Q_q> (Eq. Shor7).  The
default workload is a seeded random circuit on 30 qubits, depth 40 (1800
gates), in complex128: the configuration the headline metric is quoted on.

Printed (rank 0, one JSON line): gates/s over all ranks (``value``, inputs
resident in device memory, timed with CUDA events), the same through the
C-ABI call with the gate list in host memory (``e2e``), the roofline of the
dominant kernel from event-timed launches, the CPU oracle on a bounded sample
(``cpu_baseline``), SM clocks sampled during the timed region, and the number
of kernel launches.  ``--impl reference`` times the CPU oracle instead.

N > 1 (torchrun): every rank runs its own replica of the workload (the method
needs no exchange between replicas); ``value`` = all ranks' gates / max time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import inputs  # noqa: E402

METRIC = "gates/s and effective HBM GB/s (fraction of peak) at 30-34 qubits; fused FP32 vs FP64"

WORKLOADS = {
    "random30_c128": dict(kind="random", n=30, depth=40, seed=2, dtype="c128",
                          text="seeded random circuit, 30 qubits, depth 40 (1800 gates), complex128"),
    "random30_c64": dict(kind="random", n=30, depth=40, seed=2, dtype="c64",
                         text="seeded random circuit, 30 qubits, depth 40 (1800 gates), complex64"),
    "random34_c64": dict(kind="random", n=34, depth=20, seed=4, dtype="c64",
                         text="seeded random circuit, 34 qubits, depth 20 (1020 gates), complex64 (128 GiB)"),
    "adder30_c64": dict(kind="adder", n=30, m=15, seed=3, dtype="c64",
                        text="QFT register adder of two 15-qubit registers (30 qubits), complex64"),
    # the paper's own adder runs (App. B): same registers, same N_O
    "adder3x11_c128": dict(kind="adder", n=33, m=11, values=(292, 585, 1170), dtype="c128",
                           text="the paper's 3-11QBA adder 292+585+1170 (33 qubits, N_O = 286), complex128 (128 GiB)"),
    "adder2x17_c64": dict(kind="adder", n=34, m=17, values=(26214, 104857), dtype="c64",
                          text="the paper's 2-17QBA adder 26214+104857 (34 qubits, N_O = 493), complex64 (128 GiB)"),
    "adder2x17_c128": dict(kind="adder", n=34, m=17, values=(26214, 104857), dtype="c128",
                           text="the paper's 2-17QBA adder 26214+104857 (34 qubits, N_O = 493), complex128 (256 GiB)"),
    "qft10_c128": dict(kind="qft", n=10, seed=1, dtype="c128",
                       text="10-qubit QFT with reversal swaps on a seeded basis state, complex128"),
    "hadamard30_c128": dict(kind="hadamard", n=30, dtype="c128",
                            text="Hadamard on every qubit of 30 qubits (the paper's scaling test), complex128"),
    "batch512_c64": dict(kind="batch", n=24, dtype="c64",
                         text="batch of 512 seeded random circuits, n ~ U{12..24}, depth ~ U{10..60}, complex64, "
                              "one persistent graph-captured launch"),
}

# Peaks: measured copy bandwidth from MEASURED_PEAKS.json; ALU peaks are the
# nominal GB300 figures (FP64 1.25 TFLOP/s from the vendor figure;
# FP32 152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s).
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP32-pipe issue rate in thread-instructions per second: 152 SMs x 128 lanes
# x 2.07 GHz (the hardware ceiling of the double-float complex128 kernels,
# which run on the FP32 pipes)
FP32_ISSUE_TINST = 152 * 128 * 2.07e9 / 1e12
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# TF32 dense tensor rate = bf16 rate x (1.1 / 2.25), the nominal ratio
TF32_OVER_BF16 = 1.1 / 2.25


def resize_workload(name, n):
    """The workload `name` at n qubits (the random circuit, the Hadamard
    replay, the seeded adder with two registers of n / 2 qubits): its
    description and its new name."""
    w = dict(WORKLOADS[name])
    if not (w["kind"] in ("random", "hadamard") or (w["kind"] == "adder" and "seed" in w)):
        raise ValueError("--n does not apply to %s" % name)
    if w["kind"] == "adder":
        if n % 2:
            raise ValueError("the seeded adder takes an even --n")
        w["m"] = n // 2
        w["text"] = w["text"].replace("two %d-qubit registers" % WORKLOADS[name]["m"], "two %d-qubit registers" % w["m"])
    w["text"] = w["text"].replace("%d qubits" % WORKLOADS[name]["n"], "%d qubits" % n)
    w["n"] = n
    return w, "%s_n%d" % (name, n)


def workload_gates(w):
    if w["kind"] == "random":
        return inputs.random_circuit(w["n"], w["depth"], w["seed"]), inputs.random_basis(w["n"], w["seed"])
    if w["kind"] == "adder":
        if "values" in w:
            return inputs.adder_circuit(list(w["values"]), w["m"]), 0
        rng = np.random.default_rng(w["seed"])
        a, b = (int(v) for v in rng.integers(0, 1 << w["m"], 2))
        return inputs.adder_circuit([a, b], w["m"]), 0
    if w["kind"] == "qft":
        x, g = inputs.qft_circuit(w["n"], seed=w["seed"])
        return g, x
    if w["kind"] == "hadamard":
        return inputs.hadamard_all(w["n"]), 0
    raise ValueError(w["kind"])


def dtype_label(dt, kernel=None):
    """Arithmetic type of the path: complex64 computes in FP32; complex128
    keeps IEEE doubles in memory and computes in double-float (two FP32
    values, ~48 significand bits) in the tile passes and per-gate sweeps, and
    as exact bf16 digit-slice products on the tensor cores (double-float
    accumulation) in the fused 5-qubit blocks."""
    if dt == "c64":
        return "f32"
    if kernel == "dense_cuda_core":
        return "f64"
    if kernel == "fused_tc_digits":
        return "df64 (IEEE f64 storage; exact bf16 digit-slice products on the tensor cores, double-float sums)"
    return "df64 (IEEE f64 storage, double-float arithmetic)"


# The batch's algorithmic bytes count every pass and block as a read and a
# write of its state; states of up to 2^23 complex64 amplitudes (64 MiB) can
# stay in the 129 MB L2 from one pass or block to the next.
BATCH_L2_NOTE = ("algorithmic bytes = every pass or block reads and writes its state; states of <= 2^23 "
                 "amplitudes (64 MiB) can stay in the 129 MB L2 between passes")


def path_label(dt, pst, pergate=False):
    if pergate:
        return "one sweep per gate"
    k = pst["fuse_k"]
    if not k:
        return "planner (tile passes)"
    if dt == "c64" and k in (4, 5):
        return "planner (fused %d-qubit blocks on the tensor cores, 3xTF32)" % k
    if dt == "c64" and k == 6:
        return "planner (fused 6-qubit blocks on the tensor cores, bf16x3)"
    if dt == "c128" and k == 5:
        return "planner (fused 5-qubit blocks on the tensor cores, bf16 digit slices)"
    return "planner (fused %d-qubit blocks on the CUDA cores)" % k


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def tf32_peak():
    """TF32 tensor peak: the measured bf16 burst GEMM rate x the nominal ratio."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]) * TF32_OVER_BF16, "measured bf16 burst x 1.1/2.25"
    return FALLBACK_BF16_TFLOPS * TF32_OVER_BF16, "fallback bf16 x 1.1/2.25"


def _ncu_table(name, kernel, workload):
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for ln in f:
            ln = ln.split("#", 1)[0].split()
            if len(ln) >= 3 and ln[0] == kernel and ln[1] == workload:
                return float(ln[2])
    return None


def ncu_traffic(kernel, workload):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, or None."""
    return _ncu_table("ncu_traffic.txt", kernel, workload)


def ncu_fp32_inst(kernel, workload):
    """Per-launch FP32-pipe thread-instructions of a kernel (ncu instruction
    counters of the current kernel build), or None."""
    return _ncu_table("ncu_fp32_inst.txt", kernel, workload)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        first = vis.split(",")[0].strip() if vis else ""
        if first.isdigit():
            cmd += ["-i", first]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- distributed glue
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(units, seconds, ws, device=None):
    """Total units over ranks and the max elapsed time (for N > 1)."""
    if ws == 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([units, seconds], dtype=torch.float64, device=device)
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------- CPU oracle
ORACLE_MAX_N = 30  # the oracle's state lives in host memory: 16 GiB at 30 qubits


def oracle_sample(w, gates, x0, budget_s=15.0):
    """The oracle, as it stands, on the first gates of the workload until
    about budget_s seconds of work; returns (gates/s, gates done, threads,
    note).  Above ORACLE_MAX_N qubits the state does not fit in host memory:
    the oracle then runs the workload's gates that act on qubits below
    ORACLE_MAX_N at ORACLE_MAX_N qubits, and the per-gate time is scaled by
    2^(n - ORACLE_MAX_N) (an extrapolation, stated in the note)."""
    import oracle
    n = w["n"]
    note = ""
    if n > ORACLE_MAX_N:
        ns = ORACLE_MAX_N
        gates = [g for g in gates if max(tuple(g.targets) + tuple(g.controls)) < ns]
        x0 &= (1 << ns) - 1
        note = " (at %d qubits, per-gate time scaled by 2^%d: extrapolated)" % (ns, n - ns)
        n, scale = ns, float(1 << (w["n"] - ns))
    else:
        scale = 1.0
    a = oracle.basis(n, x0)
    done, t0 = 0, time.perf_counter()
    for g in gates:
        oracle.run(n, [g], state=a)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    del a
    return done / el / scale, done, oracle.num_threads(), note


def oracle_batch_sample(circs, x0s, budget_s=15.0):
    """The oracle on the batch's circuits in order, each run in full, until
    about budget_s seconds; returns (gates/s, circuits done, gates done, threads)."""
    import oracle
    done = gates = 0
    t0 = time.perf_counter()
    for (n, g), x0 in zip(circs, x0s):
        oracle.run(n, g, x0=x0)
        done += 1
        gates += len(g)
        if time.perf_counter() - t0 > budget_s:
            break
    return gates / (time.perf_counter() - t0), done, gates, oracle.num_threads()


# ----------------------------------------------------------------- ours
def run_ours(args, w, ws, rank, local):
    import torch
    import paper_quant_ph_0608239_gb300 as q
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    gates, x0 = workload_gates(w)
    n, ng = w["n"], len(gates)
    st = q.State(n, w["dtype"])
    # the plan picks its tile size / fusion width by timing its candidates
    # (QSIM_MODE_AUTO); --fuse-k pins a fusion width instead
    if args.pergate:  # one sweep of the state per gate (Sec. III.A)
        plan = st.plan(gates, mode=q.MODE_PERGATE)
    elif args.fuse_k or args.tile_bits:
        plan = st.plan(gates, fuse_k=args.fuse_k, tile_bits=args.tile_bits)
    else:
        plan = st.plan(gates, mode=q.MODE_AUTO)
    stream = torch.cuda.current_stream()

    def step():
        st.set_basis(x0)
        plan.run()
        return st.qubit_probs()

    for _ in range(plan.stats()["candidates"]):  # tuning runs (untimed)
        step()
    for _ in range(args.warmup):
        step()
    pst = plan.stats()
    torch.cuda.synchronize()
    c0 = st.counters()
    st.profile(True)
    clocks = ClockSampler()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        qp = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    el = e0.elapsed_time(e1) / 1e3
    prof = st.profile_read()
    st.profile(False)
    c1 = st.counters()
    launches = c1["launches"] - c0["launches"]
    total_gates, max_el = aggregate(float(ng * args.steps), el, ws, dev)
    value = total_gates / max_el
    norm_drift = abs(st.norm() - 1.0)

    # e2e: the gate list in host memory through qsim_run_circuit each step,
    # the expectations read back to host memory.
    arr = q.gate_array(gates)
    e2e_T = 0 if pst["fuse_k"] else pst["tile_bits"]
    e2e_k = pst["fuse_k"]
    e2e_mode = q.MODE_PERGATE if args.pergate else q.MODE_FUSED
    for _ in range(1):
        st.set_basis(x0)
        st.run(None, gate_arr=arr, mode=e2e_mode, tile_bits=e2e_T, fuse_k=e2e_k)
        st.qubit_probs()
    torch.cuda.synchronize()
    c2 = st.counters()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st.set_basis(x0)
        st.run(None, gate_arr=arr, mode=e2e_mode, tile_bits=e2e_T, fuse_k=e2e_k)
        st.qubit_probs()
    torch.cuda.synchronize()
    e2e_el = time.perf_counter() - t0
    c3 = st.counters()
    e2e_gates, e2e_max = aggregate(float(ng * args.steps), e2e_el, ws, dev)

    hbm_peak, peak_src = peaks()
    fam, (nl, ms, by, fl) = max(prof.items(), key=lambda kv: kv[1][1])
    per_launch_s = ms / nl / 1e3
    gbs = by / nl / per_launch_s / 1e9
    tflops = fl / nl / per_launch_s / 1e12
    frac_hbm = gbs / hbm_peak
    tkey = args.workload
    if pst["fuse_k"] and "_fused" not in tkey:  # the autotuner picked dense blocks
        tkey += "_fused%d" % pst["fuse_k"]
    traffic = ncu_traffic(fam, tkey)
    hbm_roof = {"bound": "hbm", "kernel": fam, "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": frac_hbm, "traffic": traffic, "peak_source": peak_src + " copy (MEASURED_PEAKS.json)",
                "alg_bytes_per_launch": by / nl, "launches": nl, "avg_launch_ms": ms / nl}
    if w["dtype"] == "c128" and fam != "dense_cuda_core":
        # double-float arithmetic on the FP32 pipes: FP32 thread-instructions
        # per second (ncu's per-launch count over the live launch time)
        # against the FP32 issue rate; null without a capture of this kernel
        inst = ncu_fp32_inst(fam, tkey)
        ach = inst / (ms / nl / 1e3) / 1e12 if inst else None
        alu_roof = {"bound": "alu", "kernel": fam, "achieved": ach, "peak": FP32_ISSUE_TINST,
                    "unit": "T FP32 thread-instructions/s", "frac": ach / FP32_ISSUE_TINST if ach else None,
                    "traffic": traffic, "peak_source": "FP32 issue: 152 SM x 128 lanes x 2.07 GHz",
                    "fp32_inst_per_launch": inst, "alg_flops_per_launch": fl / nl,
                    "alg_tflops": tflops, "launches": nl, "avg_launch_ms": ms / nl}
    else:
        alu_peak = FP64_PEAK_TFLOPS if fam == "dense_cuda_core" and w["dtype"] == "c128" else FP32_PEAK_TFLOPS
        alu_roof = {"bound": "alu", "kernel": fam, "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": tflops / alu_peak, "traffic": traffic,
                    "peak_source": ("nominal FP64: 1.25 TFLOP/s" if alu_peak == FP64_PEAK_TFLOPS
                                    else "nominal FP32: 152 SM x 128 x 2 x 2.07 GHz"),
                    "alg_flops_per_launch": fl / nl, "launches": nl, "avg_launch_ms": ms / nl}
    frac_alu = alu_roof["frac"] or 0.0
    if fam == "fused_tc_digits":
        # 21 bf16 slice products per algorithmic product (digits.cuh); the
        # tensor pipe executes 21x the algorithmic flops in bf16
        bp = tf32_peak()[0] / TF32_OVER_BF16
        ach = 21.0 * tflops
        alu_roof = {"bound": "tensor", "kernel": fam, "achieved": ach, "peak": bp, "unit": "TFLOP/s (bf16)",
                    "frac": ach / bp, "traffic": traffic,
                    "peak_source": "bf16 dense: measured burst GEMM (MEASURED_PEAKS.json); 21 bf16 slice products "
                                   "per algorithmic product",
                    "alg_flops_per_launch": fl / nl, "alg_tflops": tflops, "launches": nl,
                    "avg_launch_ms": ms / nl}
        frac_alu = ach / bp
    if fam == "fused_tc_bf16x3":
        # six bf16 slice products per algorithmic product
        bp = tf32_peak()[0] / TF32_OVER_BF16
        ach = 6.0 * tflops
        alu_roof = {"bound": "tensor", "kernel": fam, "achieved": ach, "peak": bp, "unit": "TFLOP/s (bf16)",
                    "frac": ach / bp, "traffic": traffic,
                    "peak_source": "bf16 dense: measured burst GEMM (MEASURED_PEAKS.json); 6 bf16 slice products "
                                   "per algorithmic product",
                    "alg_flops_per_launch": fl / nl, "alg_tflops": tflops, "launches": nl,
                    "avg_launch_ms": ms / nl}
        frac_alu = ach / bp
    if fam == "fused_tensor_core":
        # 3xTF32: three TF32 products per algorithmic product; the achieved
        # figure counts algorithmic flops once
        tp, tsrc = tf32_peak()
        alu_roof = {"bound": "tensor", "kernel": fam, "achieved": tflops, "peak": tp, "unit": "TFLOP/s",
                    "frac": tflops / tp, "traffic": traffic,
                    "peak_source": "TF32 dense: " + tsrc + "; 3 TF32 products per algorithmic product",
                    "alg_flops_per_launch": fl / nl, "launches": nl, "avg_launch_ms": ms / nl}
        frac_alu = tflops / tp
    roof, other = (alu_roof, hbm_roof) if frac_alu > frac_hbm else (hbm_roof, alu_roof)

    # effective bandwidth of the whole step (algorithmic bytes / step time)
    step_bytes = sum(v[2] for v in prof.values()) / args.steps
    eff_gbs = step_bytes / (el / args.steps) / 1e9

    out = {
        "metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_label(w["dtype"], fam),
        "data": "synthetic: seeded generator (inputs/circuits.py), no dataset",
        "config": {"workload": w["text"], "name": args.workload, "n": n, "gates": ng, "dtype": w["dtype"],
                   "path": path_label(w["dtype"], pst, args.pergate), "tile_passes": pst["passes"], "tile_bits": pst["tile_bits"],
                   "autotune": [dict(c, chosen=(i == pst["chosen"])) for i, c in enumerate(pst["autotune"])],
                   "state_bytes": st.nbytes, "l2": "inputs larger than L2 (state %d MiB >> 129 MB)" % (st.nbytes >> 20),
                   "parallelism": "replicas x%d" % ws},
        "eff_hbm_gbs": eff_gbs, "eff_hbm_frac": eff_gbs / hbm_peak,
        "norm_drift": norm_drift,
        "roofline": roof, "roofline_other": other,
        "kernels": {k: {"launches": v[0], "ms": v[1], "alg_bytes": v[2], "alg_flops": v[3]} for k, v in prof.items()},
        "e2e": {"value": e2e_gates / e2e_max, "unit": "gates/s",
                "h2d_bytes_per_step": (c3["h2d_bytes"] - c2["h2d_bytes"]) // args.steps,
                "d2h_bytes_per_step": (c3["d2h_bytes"] - c2["d2h_bytes"]) // args.steps},
        "gpu_launches": launches,
        "clocks": clk,
    }
    plan.free()
    st.free()
    del st
    torch.cuda.empty_cache()

    if rank == 0 and ws == 1 and not args.no_companions and w["kind"] == "random":
        main = {"gates_per_s": value, "ms_per_run": max_el / args.steps * 1e3, "runs": args.steps,
                "path": out["config"]["path"]}
        out["configs"] = config_lines(q, main, args)
        out["single_gate_sweeps"] = single_gate_sweeps(q)
        out["qubit_interchange_sweeps"] = qubit_interchange_sweeps(q)
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, done, thr, note = oracle_sample(w, gates, x0, args.cpu_budget)
        out["cpu_baseline"] = {"value": v, "unit": "gates/s", "cores": thr, "kind": "oracle",
                               "sample": "first %d of %d gates of the workload (%d qubits, complex128 "
                                         "oracle), timed on %d host threads%s" % (done, ng, n, thr, note)}
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out if rank == 0 else None


def single_gate_sweeps(q, n=30, targets=(0, 1, 2, 4, 8, 16, 29)):
    """Per-gate sweeps of the whole state (the one-gate-per-sweep execution of
    Sec. III.A), timed with CUDA events: effective GB/s per target bit for H,
    a Haar SU(2), a phase shift and a CNOT, in complex64 and complex128."""
    import torch
    from inputs import Gate
    hbm, _ = peaks()
    out = {}
    v = np.random.default_rng(0).standard_normal(4)
    v /= np.linalg.norm(v)
    for dt in ("c64", "c128"):
        st = q.State(n, dt)
        S = 8 if dt == "c64" else 16
        res = {}
        for name, mk, touched in (
                ("H", lambda t: Gate("H", (t,), (), ()), 1.0),
                ("SU2", lambda t: Gate("SU2", (t,), (), tuple(v)), 1.0),
                ("R", lambda t: Gate("R", (t,), (), (0.3,)), 0.5),
                ("CNOT", lambda t: Gate("NOT", (t,), ((t + 7) % n,), ()), 0.5)):
            row = {}
            for t in targets:
                g = mk(t)
                st.apply_gate(g)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                stream = torch.cuda.current_stream()
                e0.record(stream)
                for _ in range(3):
                    st.apply_gate(g)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 3
                gbs = 2.0 * S * touched * (1 << n) / (ms / 1e3) / 1e9
                row[str(t)] = {"ms": round(ms, 3), "GBs": round(gbs, 1), "frac": round(gbs / hbm, 3)}
            res[name] = row
        out[dt] = res
        st.free()
        torch.cuda.empty_cache()
    return out


def qubit_interchange_sweeps(q, n=30, Ks=(1, 2, 4)):
    """The paper's qubit interchange (Sec. III.B: local bit l_i <-> nonlocal
    bit h_i for i < K, Eqs. onequbitchange and twoqubitchange0-5) as one pass
    over the state (qsim_permute_bits), timed with CUDA events: effective GB/s
    per K.  Algorithmic bytes: 2 S 2^n per pass, 2 S 2^(n-1) for K = 1 (the
    half whose two bits differ).  A failure is reported in place of a figure
    and does not stop the run."""
    import torch
    hbm, _ = peaks()
    out = {}
    for dt in ("c64", "c128"):
        S = 8 if dt == "c64" else 16
        res = {}
        st = None
        try:
            st = q.State(n, dt)
            for K in Ks:
                lo, hi = list(range(K)), [n - 1 - i for i in range(K)]
                try:
                    st.permute_bits(lo, hi)  # warm-up
                    stream = torch.cuda.current_stream()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(4):
                        st.permute_bits(lo, hi)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / 4
                    moved = 0.5 if K == 1 else 1.0
                    gbs = 2.0 * S * moved * (1 << n) / (ms / 1e3) / 1e9
                    res[str(K)] = {"ms": round(ms, 3), "GBs": round(gbs, 1), "frac": round(gbs / hbm, 3)}
                except Exception as e:  # noqa: BLE001 -- reported, not fatal
                    res[str(K)] = {"error": str(e)[:200]}
        except Exception as e:  # noqa: BLE001
            res = {"error": str(e)[:200]}
        finally:
            if st is not None:
                st.free()
            torch.cuda.empty_cache()
        out[dt] = res
    return out


def _event_runs(fn, reps):
    """Per-run milliseconds of fn() over reps runs, CUDA events on the current
    stream around each run (after the caller's warm-up)."""
    import torch
    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for r in range(reps):
        fn()
        evs[r + 1].record(stream)
    torch.cuda.synchronize()
    return [evs[r].elapsed_time(evs[r + 1]) for r in range(reps)]


def _timed_circuit(q, n, dt, gates, x0, reps, **plan_kw):
    """A planned circuit timed as a bench step (set the basis state, run the
    plan, read <Q_q>): tuning runs and one warm-up untimed, then reps runs,
    each bracketed by CUDA events; median ms, gates/s, the plan's path and its
    algorithmic bytes per run as a fraction of the measured HBM copy rate."""
    import torch
    st = q.State(n, dt)
    plan = st.plan(gates, **plan_kw)

    def step():
        st.set_basis(x0)
        plan.run()
        st.qubit_probs()

    for _ in range(plan.stats()["candidates"] + 1):
        step()
    ms = statistics.median(_event_runs(step, reps))
    pst = plan.stats()
    out = {"gates_per_s": len(gates) / (ms / 1e3), "ms_per_run": ms, "runs": reps,
           "path": path_label(dt, pst, plan_kw.get("mode") == q.MODE_PERGATE),
           "passes": pst["passes"] if pst["mode"] != q.MODE_PERGATE else pst["sweeps"],
           # the plan's algorithmic bytes per run over the measured copy rate
           "hbm_frac": pst["alg_bytes"] / (ms / 1e3) / 1e9 / peaks()[0]}
    plan.free()
    st.free()
    del st
    torch.cuda.empty_cache()
    return out


def config_lines(q, main, args):
    """The other configurations of the benchmark and the arms of the fused
    complex64 vs per-gate complex128 comparison, each event-timed over
    repeated runs (median): the 10-qubit QFT, the 30-qubit random circuit on
    every path, the adder of two 15-qubit registers (with its output index
    checked), the 34-qubit circuit (complex64, 128 GiB) and the batch of 512
    circuits."""
    res = {}
    reps = max(3, min(args.steps, 5))
    # 10-qubit QFT, complex128
    x, g = inputs.qft_circuit(10, seed=1)
    res["qft10_c128"] = {"pergate": _timed_circuit(q, 10, "c128", g, x, 20, mode=q.MODE_PERGATE),
                         "planner": _timed_circuit(q, 10, "c128", g, x, 20, mode=q.MODE_AUTO)}
    # 30-qubit random circuit, depth 40: every path
    g = inputs.random_circuit(30, 40, 2)
    x = inputs.random_basis(30, 2)
    c2 = {"c128_autotuned": main,
          "c64_autotuned": _timed_circuit(q, 30, "c64", g, x, reps, mode=q.MODE_AUTO),
          "c64_tile_passes": _timed_circuit(q, 30, "c64", g, x, reps, tile_bits=12),
          "c64_tensor_cores_k5": _timed_circuit(q, 30, "c64", g, x, reps, fuse_k=5),
          "c64_tensor_cores_k6": _timed_circuit(q, 30, "c64", g, x, reps, fuse_k=6),
          "c128_tensor_cores_k5": _timed_circuit(q, 30, "c128", g, x, reps, fuse_k=5),
          "c128_tile_passes": _timed_circuit(q, 30, "c128", g, x, 2, tile_bits=12),
          "c128_pergate": _timed_circuit(q, 30, "c128", g, x, 2, mode=q.MODE_PERGATE)}
    # fused FP32 (the fastest complex64 fused path) over one FP64 sweep per gate
    fused64 = min(c2["c64_tensor_cores_k5"]["ms_per_run"], c2["c64_tensor_cores_k6"]["ms_per_run"])
    c2["fused_c64_over_pergate_c128"] = c2["c128_pergate"]["ms_per_run"] / fused64
    res["random30"] = c2
    # adder of two 15-qubit registers (complex64): first seeded pair, output index checked
    a, b = inputs.adder_pairs(15, 8, seed=3)[0]
    g = inputs.adder_circuit([a, b], 15)
    ad = {"autotuned": _timed_circuit(q, 30, "c64", g, 0, reps, mode=q.MODE_AUTO),
          "tile_passes": _timed_circuit(q, 30, "c64", g, 0, reps),
          "tensor_cores_k5": _timed_circuit(q, 30, "c64", g, 0, reps, fuse_k=5),
          "tensor_cores_k6": _timed_circuit(q, 30, "c64", g, 0, reps, fuse_k=6)}
    st = q.State(30, "c64")
    st.run(g, fuse_k=5)
    qp = st.qubit_probs()
    st.free()
    ad["output_index_exact"] = sum(1 << i for i in range(30) if qp[i] > 0.5) == inputs.adder_expected_index([a, b], 15)
    res["adder2x15_c64"] = ad
    # 34 qubits, depth 20, complex64 (128 GiB): 5- and 6-qubit tensor-core
    # blocks (the tile passes take 2-4x longer there)
    g = inputs.random_circuit(34, 20, 4)
    res["random34_c64"] = {"tensor_cores_k5": _timed_circuit(q, 34, "c64", g, inputs.random_basis(34, 4), 3,
                                                             fuse_k=5),
                           "tensor_cores_k6": _timed_circuit(q, 34, "c64", g, inputs.random_basis(34, 4), 3,
                                                             fuse_k=6)}
    # batch of 512 circuits: one graph replay per run
    import torch
    circs = inputs.batch_circuits()
    states = [q.State(n, "c64") for n, _ in circs]
    x0s = [inputs.random_basis(n, seed=3000 + i) for i, (n, _) in enumerate(circs)]
    bt = q.Batch(states, x0s, [gg for _, gg in circs])
    bt.run()
    bt.sync()
    ms = statistics.median(_event_runs(bt.run, reps))
    bst = bt.stats()
    res["batch512_c64"] = {"gates_per_s": bst["gates"] / (ms / 1e3), "ms_per_run": ms, "runs": reps,
                           "cuda_graph": bst["graph"], "tensor_core_circuits": bst["fused"],
                           "eff_hbm_frac": bst["alg_bytes"] / (ms / 1e3) / 1e9 / peaks()[0], "note": BATCH_L2_NOTE}
    bt.free()
    for st in states:
        st.free()
    del states
    torch.cuda.empty_cache()
    return res


def run_batch_workload(args, w, ws, rank, local):
    """Batch config: one step = one replay of the captured persistent launch."""
    import torch
    import paper_quant_ph_0608239_gb300 as q
    torch.cuda.set_device(local)
    circs = inputs.batch_circuits()
    if args.batch_count:
        circs = circs[:args.batch_count]
    ng = sum(len(g) for _, g in circs)
    states = [q.State(n, "c64") for n, _ in circs]
    x0s = [inputs.random_basis(n, seed=3000 + i) for i, (n, _) in enumerate(circs)]
    b = q.Batch(states, x0s, [g for _, g in circs])
    bst = b.stats()
    for _ in range(args.warmup):
        b.run()
    b.sync()
    c0 = sum(st.counters()["launches"] for st in states)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        b.run()
    e1.record(stream)
    b.sync()
    clk = clocks.stop()
    el = e0.elapsed_time(e1) / 1e3
    launches = args.steps * bst["kernels"]  # the persistent launch and the tensor-core lane, per step
    # baseline of the comparison: one planned run per circuit
    plans = [st.plan(g) for st, (_, g) in zip(states, circs)]
    for st, p, x0 in zip(states, plans, x0s):
        st.set_basis(x0)
        p.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for st, p, x0 in zip(states, plans, x0s):
        st.set_basis(x0)
        p.run()
    torch.cuda.synchronize()
    per_circuit = ng / (time.perf_counter() - t0)
    for p in plans:
        p.free()
    # e2e: planning, upload and the run through qsim_run_batch, gate lists in host memory
    arrs = [q.gate_array(g) for _, g in circs]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q.run_batch(states, x0s, arrs)
    e2e = ng * args.steps / (time.perf_counter() - t0)
    h2d = sum(len(g) for _, g in circs) * 112  # qsim_gate records read by the planner
    hbm_peak, peak_src = peaks()
    per_run = el / args.steps
    gbs, tfl = bst["alg_bytes"] / per_run / 1e9, bst["alg_flops"] / per_run / 1e12
    traffic = ncu_traffic("batch", args.workload)
    hbm_roof = {"bound": "hbm", "kernel": "batch", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak, "traffic": traffic, "peak_source": peak_src + " copy (MEASURED_PEAKS.json)",
                "alg_bytes_per_launch": bst["alg_bytes"], "launches": args.steps, "avg_launch_ms": per_run * 1e3,
                "note": BATCH_L2_NOTE}
    alu_roof = {"bound": "alu", "kernel": "batch", "achieved": tfl, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tfl / FP32_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "nominal FP32: 152 SM x 128 x 2 x 2.07 GHz",
                "alg_flops_per_launch": bst["alg_flops"], "launches": args.steps, "avg_launch_ms": per_run * 1e3}
    if bst["fused"]:
        # the tensor-core lane's dense products are counted in alg_flops but run
        # on the tensor cores, not the FP32 pipes: no FP32 roofline then
        roof, other = hbm_roof, None
    else:
        roof, other = (alu_roof, hbm_roof) if alu_roof["frac"] > hbm_roof["frac"] else (hbm_roof, alu_roof)
    out = {
        "metric": METRIC, "value": ng * args.steps / el, "unit": "gates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded generator (inputs/circuits.py), no dataset",
        "config": {"workload": w["text"], "name": args.workload, "circuits": len(circs), "gates": ng,
                   "tile_passes": bst["passes"], "work_items": bst["items"], "cuda_graph": bst["graph"],
                   "tensor_core_circuits": bst["fused"], "tensor_core_blocks": bst["blocks"],
                   "l2": "inputs larger than L2 (batch states %d MiB)" % (sum(st.nbytes for st in states) >> 20),
                   "parallelism": "replicas x%d" % ws},
        "one_launch_per_circuit_gates_per_s": per_circuit,
        "e2e": {"value": e2e, "unit": "gates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4},
        "gpu_launches": launches, "clocks": clk, "roofline": roof, "roofline_other": other,
    }
    b.free()
    for st in states:
        st.free()
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, nc, ngs, thr = oracle_batch_sample(circs, x0s, args.cpu_budget)
        out["cpu_baseline"] = {"value": v, "unit": "gates/s", "cores": thr, "kind": "oracle",
                               "sample": "the first %d of %d circuits of the batch in full (%d gates, complex128 "
                                         "oracle), timed on %d host threads" % (nc, len(circs), ngs, thr)}
    return out if rank == 0 else None


# -------------------------------------------------------------- reference
def run_reference(args, w, ws, rank):
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    if rank != 0:
        return None
    if w["kind"] == "batch":  # the oracle on the batch's circuits in order
        circs = inputs.batch_circuits()
        x0s = [inputs.random_basis(n, seed=3000 + i) for i, (n, _) in enumerate(circs)]
        budget = max(2.0, min(args.cpu_budget, 120.0 / max(1, args.steps + args.warmup)))
        oracle_batch_sample(circs, x0s, budget / 4)
        vals = []
        for _ in range(args.steps):
            v, nc, ngs, thr = oracle_batch_sample(circs, x0s, budget)
            vals.append(v)
        v = statistics.median(vals)
        sample = "the first %d of %d circuits of the batch in full per step (%d gates), %d host threads" % (
            nc, len(circs), ngs, thr)
        return {
            "metric": METRIC, "value": v, "unit": "gates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * ngs / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic: seeded generator (inputs/circuits.py)",
            "config": {"workload": w["text"], "name": args.workload, "circuits": len(circs)},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "gates/s", "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
    gates, x0 = workload_gates(w)
    budget = max(2.0, min(args.cpu_budget, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(w, gates, x0, budget / 4)
    vals = []
    thr, done, note = 1, 0, ""
    for _ in range(args.steps):
        v, done, thr, note = oracle_sample(w, gates, x0, budget)
        vals.append(v)
    v = statistics.median(vals)
    sample = "first %d of %d gates per step (%d qubits, complex128 oracle), %d host threads%s" % (
        done, len(gates), w["n"], thr, note)
    return {
        "metric": METRIC, "value": v, "unit": "gates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * done / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic: seeded generator (inputs/circuits.py)",
        "config": {"workload": w["text"], "name": args.workload, "n": w["n"], "gates": len(gates)},
        "impl": "reference",
        "cpu_baseline": {"value": v, "unit": "gates/s", "cores": thr, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="random30_c128")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work per sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-companions", action="store_true")
    ap.add_argument("--n", type=int, default=0,
                    help="override the qubit count of the random, Hadamard and seeded adder workloads (smaller cases for profiling)")
    ap.add_argument("--pergate", action="store_true", help="one sweep of the state per gate (no tile passes)")
    ap.add_argument("--dtype", choices=["c64", "c128"], default=None, help="override the workload's precision")
    ap.add_argument("--batch-count", type=int, default=0, help="batch workload: only the first N circuits")
    ap.add_argument("--tile-bits", type=int, default=0,
                    help="pin the tile size T of the tile passes (default: autotuned)")
    ap.add_argument("--fuse-k", type=int, default=0,
                    help="fuse the circuit into dense k-qubit blocks (k = 4, 5 run on the tensor cores for complex64)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    ws, rank, local = dist_env()
    w = dict(WORKLOADS[args.workload])
    if args.n:
        try:
            w, args.workload = resize_workload(args.workload, args.n)
        except ValueError as e:
            ap.error(str(e))
    if args.dtype and args.dtype != w["dtype"] and w["kind"] != "batch":
        w["dtype"] = args.dtype
        w["text"] = w["text"].replace("complex128", args.dtype).replace("complex64", args.dtype)
        args.workload = args.workload + "_" + args.dtype
    if args.pergate:
        args.workload = args.workload + "_pergate"
    if args.batch_count and w["kind"] == "batch":
        w["text"] = w["text"].replace("batch of 512", "batch of the first %d of 512" % args.batch_count)
        args.workload = args.workload + "_first%d" % args.batch_count
    if args.fuse_k:
        args.workload = args.workload + "_fused%d" % args.fuse_k
    if args.tile_bits:
        args.workload = args.workload + "_T%d" % args.tile_bits
    if args.impl == "reference":
        out = run_reference(args, w, ws, rank)
    elif w["kind"] == "batch":
        out = run_batch_workload(args, w, ws, rank, local)
    else:
        out = run_ours(args, w, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
