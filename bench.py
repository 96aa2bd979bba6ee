#!/usr/bin/env python
"""Benchmark: circuit wall time and effective HBM GB/s per state sweep, fused
vs per-gate, on one GB300 (n = 30 random layered circuit; complex128 headline
on the tensor-core plan, complex64 and per-gate numbers alongside).

One step = one execution of the contracted circuit on the resident
2^30-amplitude complex128 state (every 5-qubit block on tensor cores as exact
fp16 digit products) followed by its FP64 norm. The state (16 GiB) is far
larger than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 runs N independent replicas (the path does not shard across GPUs in
this build); the reported value is the job's time per circuit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "circuit wall time & effective HBM GB/s per state sweep (n=30 c128/c64), fused vs per-gate"
# FP64 rate of one GB300: the nominal 1.25 TFLOP/s (the measured-peaks file has no FP64 figure; an FMA
# loop measured 1.19 TFLOP/s)
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--depth", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-c128", action="store_true",
                    help="run only the complex64 line and print it alone (profiler runs of k_tc_bulk / k_tile)")
    ap.add_argument("--no-per-gate", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="skip the nvidia-smi sampler (profiler runs)")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-config side measurements")
    ap.add_argument("--full-configs", action="store_true",
                    help="also run the complex128 n=32 reference for the tensor-core config (64 GiB, ~1 min)")
    ap.add_argument("--qaoa-n", type=int, default=30, help="register size of the qaoa_n30 configuration")
    ap.add_argument("--stream-n", type=int, default=31, help="register size of the host-resident configuration")
    ap.add_argument("--smgp-ns", default="20,24,28,30", help="register sizes of the SMGP ablation (comma list)")
    ap.add_argument("--tune", default="auto", help="auto | k,m,L[,tc_min_gates[,tc_pipeline]]")
    ap.add_argument("--tile-staging", type=int, default=0,
                    help="with --tune k,m,L: 2 = tile passes staged by bulk copies (profiler runs of k_tile_bulk)")
    ap.add_argument("--only-config", default=None,
                    choices=["qft_n30_m2", "qft_n28_c128", "random_n32_cz_tensor", "ucc_batched_n20",
                             "hea_adjoint_n24", "qaoa_n30", "smgp_ablation", "stream_host_state"],
                    help="run one configuration workload alone (no headline) and print its JSON")
    return ap.parse_args()


def workload(args):
    from paper_2509_04955_gb300 import workloads as W
    return W.random_layered(args.n, args.depth, seed=args.seed, entangler="cnot")


def workload_desc(args, ngates):
    return (f"random layered circuit n={args.n}, depth {args.depth} (H/RX/RY/RZ on every qubit + CNOT on a "
            f"random matching per layer, seed {args.seed}, {ngates} gates), |0..0> then repeated application")


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]), "power": float(parts[3]),
                             "hw": parts[5], "hwt": parts[6], "swt": parts[7], "swp": parts[8]})
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["max"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- oracle timing

def oracle_sample(args, gates, threads: int, budget_s: float = 60.0):
    """Times the FP64 oracle on the same circuit at the same n.

    threads = 1: the first gate of each kind the circuit holds (a complete
    gate-kind sample), scaled by the circuit's count of each kind. threads > 1
    (0 = all processors): whole layers (every gate of layer 1, then more
    layers while the budget lasts), scaled by the number of layers.
    Returns (ms per full circuit, description, threads used)."""
    import ctypes as C
    import numpy as np
    import oracle as O
    n = args.n
    L = O.lib()
    used = L.or_set_threads(threads)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1
    packed = O.pack(gates)
    theta = (C.c_double * 1)()
    ptr = psi.ctypes.data_as(C.POINTER(C.c_double))

    def kind(g):
        return (g.kind, len(g.controls))
    try:
        if used == 1:
            first, counts = {}, {}
            for i, g in enumerate(gates):
                counts[kind(g)] = counts.get(kind(g), 0) + 1
                first.setdefault(kind(g), i)
            per = {}
            t_all = 0.0
            for k, i in first.items():
                t0 = time.perf_counter()
                L.or_apply_gate(ptr, n, C.byref(packed[i]), theta)
                per[k] = time.perf_counter() - t0
                t_all += per[k]
            ms = sum(per[k] * counts[k] for k in counts) * 1e3
            kinds = ", ".join(f"{k[0]}{'+c' * k[1]} x{counts[k]}" for k in sorted(counts))
            desc = (f"oracle (plain C, FP64) on 1 thread: one gate of each kind of the circuit at n={n} "
                    f"({len(per)} gates, {t_all:.1f} s), scaled by the circuit's counts ({kinds})")
        else:
            per_layer = len(gates) // args.depth
            t0 = time.perf_counter()
            layers = 0
            while layers < args.depth and (layers == 0 or time.perf_counter() - t0 < budget_s / 2):
                for i in range(layers * per_layer, (layers + 1) * per_layer):
                    L.or_apply_gate(ptr, n, C.byref(packed[i]), theta)
                layers += 1
            dt = time.perf_counter() - t0
            ms = dt / layers * args.depth * 1e3
            desc = (f"oracle (plain C, FP64) on {used} threads: {layers} whole layer(s) of {per_layer} gates "
                    f"at n={n} in {dt:.1f} s, scaled to the {args.depth} layers")
    finally:
        L.or_set_threads(1)
    return ms, desc, used


def oracle_prefix(n, gates, count, threads=0):
    """The FP64 oracle (all host cores unless `threads`) applying the first
    `count` gates of a circuit to |0..0> at n qubits: (seconds, threads used).
    A configuration's CPU baseline: its cost per gate times the circuit's gates."""
    import ctypes as C
    import numpy as np
    import oracle as O
    L = O.lib()
    used = L.or_set_threads(threads)
    try:
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1
        packed = O.pack(gates[:count])
        theta = (C.c_double * 1)()
        ptr = psi.ctypes.data_as(C.POINTER(C.c_double))
        t0 = time.perf_counter()
        for i in range(count):
            L.or_apply_gate(ptr, n, C.byref(packed[i]), theta)
        return time.perf_counter() - t0, used
    finally:
        L.or_set_threads(1)


# ----------------------------------------------------------------- main paths

def max_over_ranks(value: float, dist, device: str) -> float:
    """The largest value over the ranks (the job's step time is the slowest rank's);
    `dist` is torch.distributed with an initialised group, or None for one process."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_circuit(ms_step_max: float, world: int) -> float:
    """Job time per circuit: each of the `world` replicas runs one circuit per step."""
    return ms_step_max / world


def headline_config(args, gates, world):
    """The headline workload's `config` (both arms print the same one; the GPU
    arm's plan is described under its own key)."""
    n = args.n
    return {"workload": workload_desc(args, len(gates)) + ", complex128",
            "n": n, "state": f"complex128, {(1 << n) * 16 / 2**30:g} GiB", "gates": len(gates),
            "l2": (f"inputs larger than L2 ({(1 << n) * 16 / 2**30:g} GiB state vs 129 MB); no flush"
                   if (1 << n) * 16 > 129e6 else "state fits L2: timed passes may hit L2"),
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The oracle (the tier's reference arm), as it stands, on the host's cores:
    each step applies whole layers of the headline circuit on all processors
    and scales to the full circuit; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    gates = workload(args)
    import oracle as O
    O.build()
    cfg = headline_config(args, gates, int(os.environ.get("WORLD_SIZE", "1")))
    vals = []
    desc, cores = "", 1
    for _ in range(max(1, args.steps)):
        ms, desc, cores = oracle_sample(args, gates, 0, budget_s=max(8.0, 120.0 / max(1, args.steps)))
        vals.append(ms)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(Q, torch, plan, state, steps, warmup, with_norm=True, per_launch=False):
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        Q.qs_plan_execute(plan, state)
        if with_norm:
            Q.qs_norm(state)
    torch.cuda.synchronize()
    launches0 = Q.qs_launch_count()
    if per_launch:
        Q.qs_plan_set_timing(plan, True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    norms = []
    for _ in range(steps):
        Q.qs_plan_execute(plan, state)
        if with_norm:
            norms.append(Q.qs_norm(state))
    t1.record(st)
    torch.cuda.synchronize()
    total = t0.elapsed_time(t1)
    kern = None
    if per_launch:
        kern = Q.qs_plan_timing_read_kinds(plan)
        Q.qs_plan_set_timing(plan, False)
    return total / steps, Q.qs_launch_count() - launches0, kern, norms


def mode_name(Q, kw):
    return "tensor" if kw.get("mode") == Q.QS_MODE_TENSOR else "fused"


def spread(vals):
    """median / min / max of repeated timings (ms)."""
    return {"median": statistics.median(vals), "min": min(vals), "max": max(vals), "reps": len(vals)}


def traffic_record(kernel: str, n: int):
    """DRAM bytes per launch at n from profiles/traffic.json, or None when the
    record is absent or the kernel's sources changed since it was taken."""
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(prof):
        return None
    try:
        tp = json.load(open(prof)).get(kernel, {})
        if tp.get("kernel_hash") == kernel_hash(kernel):
            return tp.get("bytes_per_launch_n30") * 2.0 ** (n - 30)
    except (ValueError, OSError, TypeError):
        return None
    return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as GE
    if rank == 0 or world == 1:
        GE.build()
    if dist:
        dist.barrier()
        GE.build()
    import paper_2509_04955_gb300 as Q
    import numpy as np

    if args.only_config:
        print(json.dumps({"only_config": args.only_config, **run_configs(Q, torch, np, args)}))
        return

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    n = args.n
    gates = workload(args)
    stream = torch.cuda.current_stream().cuda_stream
    F, T = Q.QS_MODE_FUSED, Q.QS_MODE_TENSOR
    sb128, sb64 = 2 * (1 << n) * 16, 2 * (1 << n) * 8
    extra = {}

    if args.no_c128:
        line = {"c64_tensor": c64_line(Q, torch, np, args, gates, stream, hbm_peak, bf16_peak, peak_src, None)}
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ------------------------------------------------------------ headline: complex128
    # every contracted 5-qubit block applied on tensor cores as exact fp16 digit
    # products (the complex128 tensor-core pass), one step = one circuit + FP64 norm
    state = Q.qs_state_alloc(n, Q.QS_C128, stream)
    kw = dict(mode=T)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(**kw))
    info = Q.qs_plan_info_get(plan)
    Q.qs_state_set_basis(state, 0)
    clocks = ClockSampler(local) if not args.no_clocks else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    ms_step, launches, kern, norms = time_steps(Q, torch, plan, state, args.steps, args.warmup, per_launch=True)
    clk = clocks.stop() if clocks else None
    ms_step = max_over_ranks(ms_step, dist, "cuda")
    kms = kern["tc_ms"] / max(1, kern["tc_launches"])
    achieved = sb128 / (kms * 1e-3) / 1e9
    eff_gbps = info["sweeps"] * sb128 / (ms_step * 1e-3) / 1e9
    pg_equiv_gbps = info["per_gate_sweeps"] * sb128 / (ms_step * 1e-3) / 1e9
    kern_share = {"tc_ms_per_step": kern["tc_ms"] / args.steps, "tc_launches_per_step": kern["tc_launches"] / args.steps,
                  "other_ms_per_step": kern["tile_ms"] / args.steps,
                  "other_launches_per_step": kern["tile_launches"] / args.steps}
    alg = 8.0 * 32 * (1 << n) / (kms * 1e-3) / 1e12          # 8 * 2^5 real flops per amplitude
    extra["tensor_pipe"] = {
        "algorithmic_tflops": alg, "executed_f16_tflops": alg * 21, "f16_peak_tflops": bf16_peak,
        "executed_frac": alg * 21 / bf16_peak,
        "note": "a 32x32 complex block is a real 64x64 GEMM per 32-amplitude row (the algorithmic 256 flops per "
                "amplitude); the exact digit scheme executes 21 such products in fp16 (fp16 and bf16 share the "
                "MMA rate; the peak is the measured bf16 GEMM)"}

    # per-gate complex128 (FP64, one launch per gate): the comparator and the FP64 reference state
    s_ref = Q.qs_state_alloc(n, Q.QS_C128, stream)
    if not args.no_per_gate:
        pplan = Q.qs_plan_create(n, Q.QS_C128, gates, None)
        Q.qs_state_set_basis(s_ref, 0)
        pg_ms, _, pk128, _ = time_steps(Q, torch, pplan, s_ref, 1, 1, per_launch=True, with_norm=False)
        pinfo = Q.qs_plan_info_get(pplan)
        Q.qs_state_set_basis(s_ref, 0)
        Q.qs_plan_execute(pplan, s_ref)
        Q.qs_plan_free(pplan)
        extra["per_gate_c128"] = {"ms": pg_ms, "sweeps": pinfo["per_gate_sweeps"], "launches": pinfo["launches"],
                                  "effective_gbps": pinfo["per_gate_sweeps"] * sb128 / (pk128["ms"] * 1e-3) / 1e9}
        extra["speedup_vs_per_gate_c128"] = pg_ms / ms_step
        Q.qs_state_set_basis(state, 0)
        Q.qs_plan_execute(plan, state)
        m, l2 = Q.qs_state_diff(state, s_ref)
        extra["precision_vs_fp64_per_gate"] = {"max_abs": m, "l2": l2}
    # the same circuit on CUDA cores: tile passes in FP32 pairs (and FP64 with --full-configs)
    for name, okw in (("c128_fused_fp32_pairs", dict(mode=F, fuse_k=2, tile_qubits=11, low_qubits=3, c128_pairs=1)),
                      ("c128_fused_fp64", dict(mode=F, fuse_k=1, tile_qubits=12, low_qubits=4, c128_pairs=2))):
        if name == "c128_fused_fp64" and not args.full_configs:
            continue
        s2 = Q.qs_state_alloc(n, Q.QS_C128, stream)
        p2 = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(**okw))
        i2 = Q.qs_plan_info_get(p2)
        Q.qs_state_set_basis(s2, 0)
        f_ms, _, fk, _ = time_steps(Q, torch, p2, s2, 1, 1, per_launch=True, with_norm=False)
        Q.qs_state_set_basis(s2, 0)
        Q.qs_plan_execute(p2, s2)
        extra[name] = dict(okw, ms=f_ms, passes=i2["passes"],
                           pass_gbps=i2["passes"] * sb128 / (fk["ms"] * 1e-3) / 1e9,
                           **dict(zip(("max_abs_vs_fp64_per_gate", "l2_vs_fp64_per_gate"),
                                      Q.qs_state_diff(s2, s_ref) if not args.no_per_gate else (None, None))))
        Q.qs_plan_free(p2)
        Q.qs_state_free(s2)

    # -- end to end through the C ABI with host buffers (pinned): every step copies its
    #    input state in, runs the circuit and its norm, and copies the state out;
    #    qs_plan_execute_host overlaps a step's circuit with the copies of its neighbours
    #    (three device work states); the one-call-at-a-time sequence is reported beside it.
    amp128 = 16
    host_in = torch.zeros(1 << n, dtype=torch.complex128, pin_memory=True)
    host_in[0] = 1
    host_out = torch.empty(1 << n, dtype=torch.complex128, pin_memory=True)
    e2e_steps = max(8, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2):
        Q.lib().qs_state_copy_from_host(state, host_in.data_ptr(), host_in.numel() * amp128)
        Q.qs_plan_execute(plan, state)
        Q.qs_norm(state)
        Q.lib().qs_state_copy_to_host(state, host_out.data_ptr(), host_out.numel() * amp128)
    torch.cuda.synchronize()
    e2e_seq_ms = (time.perf_counter() - t0) * 1e3 / 2
    # the host link as this run sees it: one copy each way alone (it varies with the
    # host's other traffic, and bounds the end-to-end step together with the circuit)
    copy_ms = {}
    for name, fn in (("h2d", lambda: Q.lib().qs_state_copy_from_host(state, host_in.data_ptr(), host_in.numel() * amp128)),
                     ("d2h", lambda: Q.lib().qs_state_copy_to_host(state, host_out.data_ptr(), host_out.numel() * amp128))):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        copy_ms[name] = (time.perf_counter() - t1) * 1e3
    work = [state] + [Q.qs_state_alloc(n, Q.QS_C128, stream) for _ in range(2)]
    Q.qs_plan_execute_host(plan, work, [host_in], [host_out])     # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_norms = Q.qs_plan_execute_host(plan, work, [host_in] * e2e_steps, [host_out] * e2e_steps)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    for w in work[1:]:
        Q.qs_state_free(w)
    e2e_norm = float(np.sum(np.abs(host_out.numpy()) ** 2))
    del host_in, host_out
    Q.qs_plan_free(plan)
    Q.qs_state_free(state)
    torch.cuda.empty_cache()

    # ------------------------------------------------------------ complex64 line
    extra["c64_tensor"] = c64_line(Q, torch, np, args, gates, stream, hbm_peak, bf16_peak, peak_src, s_ref)
    Q.qs_state_free(s_ref)
    torch.cuda.empty_cache()

    if not args.no_configs:
        extra["configs"] = run_configs(Q, torch, np, args, hbm_peak)

    cpu = None
    if rank == 0 and not args.no_cpu:
        ms1, d1, _ = oracle_sample(args, gates, 1)
        msa, da, cores = oracle_sample(args, gates, 0)
        cpu = {"value": msa, "unit": "ms", "cores": cores, "kind": "oracle", "sample": da,
               "one_thread": {"value": ms1, "unit": "ms", "cores": 1, "sample": d1}}

    total_ms = job_ms_per_circuit(ms_step, world)
    cfg = headline_config(args, gates, world)
    line = {
        "metric": METRIC, "value": total_ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128: fp16 digit products, exact FP32 level sums, FP32-pair combine",
        "data": "synthetic", "config": cfg,
        "plan": {"mode": "tensor", "description": "every contracted 5-qubit block on tcgen05 as exact fp16 digit "
                                                  "products", "tc_min_gates": 1, "passes": info["passes"],
                 "blocks": info["blocks"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic_record("k_tc128", n),
                     "kernel": "k_tc128 (complex128 tensor-core 5-qubit block pass)",
                     "peak_source": f"{peak_src} (hbm_gbs, burst copy)",
                     "algorithmic_bytes_per_launch": sb128, "avg_launch_ms": kms},
        "kernel_time": kern_share,
        "effective_gbps": eff_gbps, "per_gate_equivalent_gbps": pg_equiv_gbps,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": (1 << n) * amp128,
                "d2h_bytes_per_step": (1 << n) * amp128 + 8, "steps": e2e_steps,
                "api": "qs_plan_execute_host (3 device work states, copies overlapped with the circuit)",
                "sequential_ms": e2e_seq_ms, "device_norm_last": float(e2e_norms[-1]), "norm_after": e2e_norm,
                "copy_alone_ms": copy_ms,
                "copy_alone_gbs": {k: (1 << n) * amp128 / (v * 1e-3) / 1e9 for k, v in copy_ms.items()}},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
        "norm_drift": (max(abs(x - 1) for x in norms) if norms else None),
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def c64_line(Q, torch, np, args, gates, stream, hbm_peak, bf16_peak, peak_src, s_ref):
    """The same circuit in complex64: the autotuned plan (tensor-core 6-qubit
    blocks, fp16 hi/lo split) with its roofline, the per-gate comparator, and
    each result's error against the complex128 per-gate run."""
    n = args.n
    F, T = Q.QS_MODE_FUSED, Q.QS_MODE_TENSOR
    sb = 2 * (1 << n) * 8
    state = Q.qs_state_alloc(n, Q.QS_C64, stream)
    if args.tune == "auto":
        t0 = time.perf_counter()
        bopts, bms = Q.qs_plan_autotune(state, gates)
        kw = {k: v for k, v in Q.opts_dict(bopts).items() if v or k == "mode"}
        trials = {"chosen": Q.opts_dict(bopts), "ms": bms, "search_s": time.perf_counter() - t0}
    else:
        parts = [int(x) for x in args.tune.split(",")]
        kw = dict(mode=F, fuse_k=parts[0], tile_qubits=parts[1], low_qubits=parts[2], tile_staging=args.tile_staging)
        if len(parts) > 3 and parts[3] > 0:
            kw.update(mode=T, tc_min_gates=parts[3])
            if len(parts) > 4:
                kw.update(tc_pipeline=parts[4])
        trials = None
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(**kw))
    info = Q.qs_plan_info_get(plan)
    Q.qs_state_set_basis(state, 0)
    ms, launches, kern, _ = time_steps(Q, torch, plan, state, args.steps, args.warmup, per_launch=True)
    tc_dom = kern["tc_ms"] > kern["tile_ms"]
    tc_kernel = "k_tc_block" if kw.get("tc_pipeline", 0) == 1 else "k_tc_bulk"
    tile_kernel = "k_tile_bulk" if kw.get("tile_staging", 0) == 2 else "k_tile"
    kms = (kern["tc_ms"] / max(1, kern["tc_launches"])) if tc_dom else (kern["tile_ms"] / max(1, kern["tile_launches"]))
    out = {"ms": ms, "plan": {k: v for k, v in kw.items()}, "mode": mode_name(Q, kw), "passes": info["passes"],
           "gpu_launches": launches, "effective_gbps": info["sweeps"] * sb / (ms * 1e-3) / 1e9,
           "roofline": {"bound": "hbm", "achieved": sb / (kms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": sb / (kms * 1e-3) / 1e9 / hbm_peak,
                        "traffic": traffic_record(tc_kernel if tc_dom else tile_kernel, n),
                        "kernel": f"{tc_kernel} (tensor-core 6-qubit block pass)" if tc_dom else f"{tile_kernel} (tile pass)",
                        "peak_source": f"{peak_src} (hbm_gbs, burst copy)", "avg_launch_ms": kms},
           "autotune": trials}
    if tc_dom:
        alg = 512.0 * (1 << n) / (kms * 1e-3) / 1e12     # 8 * 2^6 real flops per amplitude
        mult = 3 if kw.get("tc_precision", 4) in (0, 3, 4) else 1
        out["tensor_pipe"] = {"algorithmic_tflops": alg, "executed_f16_tflops": alg * mult,
                              "f16_peak_tflops": bf16_peak, "executed_frac": alg * mult / bf16_peak,
                              "note": "a 64x64 complex block is a real 128x128 GEMM per 64-amplitude row (the "
                                      "algorithmic 512 flops per amplitude, no extra factor); the fp16 hi/lo split "
                                      "runs 3 such products"}
    Q.qs_state_set_basis(state, 0)
    Q.qs_plan_execute(plan, state)
    if not args.no_per_gate and s_ref is not None:
        out["max_abs_vs_c128_per_gate"], out["l2_vs_c128_per_gate"] = Q.qs_state_diff(state, s_ref)
        pplan = Q.qs_plan_create(n, Q.QS_C64, gates, None)
        pg_ms, _, pk, _ = time_steps(Q, torch, pplan, state, 1, 1, per_launch=True, with_norm=False)
        pinfo = Q.qs_plan_info_get(pplan)
        Q.qs_state_set_basis(state, 0)
        Q.qs_plan_execute(pplan, state)
        out["per_gate"] = {"ms": pg_ms, "effective_gbps": pinfo["per_gate_sweeps"] * sb / (pk["ms"] * 1e-3) / 1e9,
                           "max_abs_vs_c128_per_gate": Q.qs_state_diff(state, s_ref)[0]}
        out["speedup_vs_per_gate"] = pg_ms / ms
        Q.qs_plan_free(pplan)
    Q.qs_plan_free(plan)
    Q.qs_state_free(state)
    return out


def device_ms(torch, fn, reps=1):
    st = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(st)
    for _ in range(reps):
        fn()
    t1.record(st)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / reps


def device_reps(torch, fn, reps, setup=None):
    """Device times (ms) of `reps` calls of fn, each bracketed by CUDA events
    (setup, e.g. resetting the state, runs outside the bracket)."""
    st = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        if setup:
            setup()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(st)
        fn()
        t1.record(st)
        torch.cuda.synchronize()
        out.append(t0.elapsed_time(t1))
    return out


def run_configs(Q, torch, np, args, hbm_peak=6800.0):
    """Side measurements, one per benchmark configuration (timings on the
    device with CUDA events, repeated; errors against closed forms, the oracle
    or a complex128 run). The SMGP ablation and the host-resident state run
    with --full-configs or --only-config."""
    out = {}
    st = torch.cuda.current_stream().cuda_stream

    def want(name, default=True):
        return args.only_config == name or (args.only_config is None and (default or args.full_configs))

    if want("qft_n30_m2"):
        out["qft_n30_m2"] = config_qft30(Q, torch, np, st, args)
    if want("qft_n28_c128"):
        out["qft_n28_c128"] = config_qft(Q, torch, np, st, args)
    if want("random_n32_cz_tensor"):
        out["random_n32_cz_tensor"] = config_n32(Q, torch, np, st, args)
    if want("ucc_batched_n20"):
        out["ucc_batched_n20"] = config_ucc(Q, torch, np, st, args, hbm_peak)
    if want("hea_adjoint_n24"):
        out["hea_adjoint_n24"] = config_hea(Q, torch, np, st, args)
    if want("qaoa_n30"):
        out["qaoa_n30"] = config_qaoa30(Q, torch, np, st, args)
    if want("smgp_ablation", False):
        out["smgp_ablation"] = config_smgp(Q, torch, np, st, args)
    if want("stream_host_state", False):
        out["stream_host_state"] = config_stream(Q, torch, np, st, args)
    return out


def config_stream(Q, torch, np, st, args):
    """Section 3.2's batched processing on one GB300: a complex64 state kept in
    pinned host memory, streamed through three device buffers of 2^(l + 2)
    amplitudes (batches of 2^l, the 4 high qubits as batch index, at most 2 of
    them per pass). Reported against the host link's own duplex copy rate (the
    roofline of a streamed pass: the state crosses the link once each way) and
    against the same circuit run with the state resident in HBM."""
    from paper_2509_04955_gb300 import workloads as W
    n = args.stream_n
    l, h = n - 4, 2
    gates = W.random_layered(n, 4, seed=0)
    nb = (1 << n) * 8
    out = {"workload": f"random layered n={n} depth 4, complex64 state in pinned host memory "
                       f"({nb / 2**30:.0f} GiB), batches of 2^{l}, 2 batch qubits per pass", "gates": len(gates)}
    host = torch.zeros(1 << n, dtype=torch.complex64, pin_memory=True)
    host[0] = 1
    # duplex copy rate of the link: the whole state in batch-sized chunks each way at once
    dev = torch.empty(2 << l, dtype=torch.complex64, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    chunk = 1 << l
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(1 << (n - l)):
        with torch.cuda.stream(s1):
            dev[:chunk].copy_(host[c * chunk:(c + 1) * chunk], non_blocking=True)
        with torch.cuda.stream(s2):
            host[c * chunk:(c + 1) * chunk].copy_(dev[chunk:], non_blocking=True)
    torch.cuda.synchronize()
    dt_copy = time.perf_counter() - t0
    del dev
    host.zero_()
    host[0] = 1
    out["link_duplex_gbps_each_way"] = nb / dt_copy / 1e9
    opts = Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2)
    Q.qs_stream_apply(host, n, Q.QS_C64, gates[:2], None, opts, batch_qubits=l, pass_qubits=h)   # warm-up
    host.zero_()
    host[0] = 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = Q.qs_stream_apply(host, n, Q.QS_C64, gates, None, opts, batch_qubits=l, pass_qubits=h)
    ms = (time.perf_counter() - t0) * 1e3
    out.update(info)
    out["ms"] = ms
    out["link_gbps_each_way"] = info["passes"] * nb / (ms * 1e-3) / 1e9
    out["frac_of_link_duplex"] = out["link_gbps_each_way"] / out["link_duplex_gbps_each_way"]
    # the same circuit with the state resident in HBM, and the two results compared
    s = Q.qs_state_alloc(n, Q.QS_C64, st)
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
    Q.qs_state_set_basis(s, 0)
    out["in_hbm_ms"] = device_ms(torch, lambda: Q.qs_plan_execute(plan, s))
    Q.qs_state_set_basis(s, 0)
    Q.qs_plan_execute(plan, s)
    s2 = Q.qs_state_alloc(n, Q.QS_C64, st)
    Q.lib().qs_state_copy_from_host(s2, host.data_ptr(), nb)
    out["max_abs_diff_vs_in_hbm"], out["l2_diff_vs_in_hbm"] = Q.qs_state_diff(s2, s)
    Q.qs_plan_free(plan)
    Q.qs_state_free(s)
    Q.qs_state_free(s2)
    del host
    return out


def config_smgp(Q, torch, np, st, args):
    """The ablation of Fig. 14 / 15 on GB300: QAOA (3-regular, p = 4) and VQE-HEA
    (5 layers of RX, RY, RZ + staggered CNOTs) at 20-30 qubits, one gate per launch
    (Algorithms 1-4) vs staggered multi-gate groups (Section 3.3) vs tile passes
    (several gates per HBM sweep); time per circuit and average memory throughput
    (the bytes each variant moves / its time)."""
    from paper_2509_04955_gb300 import workloads as W
    out = {"note": "throughput = sweeps x 2 x 2^n x amplitude bytes / time, the bytes each variant moves"}
    for circ in ("qaoa", "hea"):
        res = {}
        for n in (int(x) for x in args.smgp_ns.split(",")):
            if circ == "qaoa":
                g, npar = W.qaoa(n, 4, W.random_regular_graph(n, 3, seed=0))
            else:
                g, npar = W.hea_staggered(n, 5)
            th = W.thetas_uniform(npar, 2)
            row = {"gates": len(g)}
            for dname, dt in (("c128", Q.QS_C128), ("c64", Q.QS_C64)):
                s = Q.qs_state_alloc(n, dt, st)
                amp = 8 if dt == Q.QS_C64 else 16
                r = {}
                for name, opts in (("per_gate", None), ("smgp", Q.make_opts(mode=Q.QS_MODE_SMGP)),
                                   ("tile_passes", Q.make_opts(mode=Q.QS_MODE_FUSED, phase_min_gates=-1))):
                    plan = Q.qs_plan_create(n, dt, g, opts)
                    Q.qs_state_set_basis(s, 0)
                    Q.qs_plan_execute(plan, s, th)
                    reps = 3 if n <= 24 else 1
                    ms = device_ms(torch, lambda: Q.qs_plan_execute(plan, s, th), reps=reps)
                    info = Q.qs_plan_info_get(plan)
                    r[name] = {"ms": ms, "launches": info["launches"],
                               "gbps": info["sweeps"] * 2 * (1 << n) * amp / (ms * 1e-3) / 1e9}
                    Q.qs_plan_free(plan)
                r["speedup_smgp_vs_per_gate"] = r["per_gate"]["ms"] / r["smgp"]["ms"]
                r["speedup_tile_vs_per_gate"] = r["per_gate"]["ms"] / r["tile_passes"]["ms"]
                row[dname] = r
                Q.qs_state_free(s)
            res[f"n{n}"] = row
        out[circ] = res
    return out


def config_qaoa30(Q, torch, np, st, args):
    """QAOA for MaxCut (Section 4.1's third circuit class) at n=30 on a seeded
    random 3-regular graph, depth p=4 (690 gates): per-gate vs contraction with
    and without diagonal phase passes (one sweep per cost layer); <C> of every
    variant against the complex128 contraction; the phase kernel timed alone on
    one cost layer; depth 1 against the published p=1 closed form; the paper-mode
    contraction's gate-count compression (Fig. 16's ratio)."""
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests"))
    from closed_forms import qaoa_p1_maxcut
    from paper_2509_04955_gb300 import workloads as W
    F, T = Q.QS_MODE_FUSED, Q.QS_MODE_TENSOR
    n, p = args.qaoa_n, 4
    edges = W.random_regular_graph(n, 3, seed=0)
    g, npar = W.qaoa(n, p, edges)
    H = W.maxcut_hamiltonian(edges)
    th = W.thetas_uniform(npar, 1)
    out = {"workload": f"QAOA MaxCut n={n}, random 3-regular graph ({len(edges)} edges), p={p}, seeded angles",
           "gates": len(g)}
    pl = Q.qs_plan_create(n, Q.QS_C128, g, Q.make_opts(paper_mode=1))
    info = Q.qs_plan_info_get(pl)
    out["paper_mode_compression"] = (info["gates"] - info["blocks"]) / info["gates"]
    Q.qs_plan_free(pl)
    variants = {"c64": [("per_gate", None), ("fused_no_phase", Q.make_opts(mode=F, phase_min_gates=-1)),
                        ("fused", Q.make_opts(mode=F)),
                        ("tensor", Q.make_opts(mode=T, tc_min_gates=4, fuse_parametric=1))],
                "c128": [("per_gate", None), ("fused_fp64", Q.make_opts(mode=F, c128_pairs=2)),
                         ("fused_fp32_pairs", Q.make_opts(mode=F, tile_qubits=12, low_qubits=4, c128_pairs=1)),
                         ("tensor", Q.make_opts(mode=T, fuse_parametric=1, c128_pairs=1))]}
    ref_e = None
    for dname, dt in (("c128", Q.QS_C128), ("c64", Q.QS_C64)):
        s = Q.qs_state_alloc(n, dt, st)
        amp = 8 if dt == Q.QS_C64 else 16
        res = {}
        for name, opts in variants[dname]:
            plan = Q.qs_plan_create(n, dt, g, opts)
            Q.qs_state_set_basis(s, 0)
            Q.qs_plan_execute(plan, s, th)
            t = device_reps(torch, lambda: Q.qs_plan_execute(plan, s, th), 1 if name == "per_gate" else 3,
                            lambda: Q.qs_state_set_basis(s, 0))
            ms = statistics.median(t)
            e = Q.qs_expval_pauli_sum(s, *H)
            if ref_e is None:
                ref_e = e
            info = Q.qs_plan_info_get(plan)
            ops = Q.qs_plan_ops(plan)
            res[name] = {"ms": spread(t), "passes": info["passes"],
                         "phase_passes": sum(op["type"] == 4 for op in ops),
                         "effective_gbps": info["sweeps"] * 2 * (1 << n) * amp / (ms * 1e-3) / 1e9,
                         "expected_cut": e, "abs_diff_vs_c128_per_gate": abs(e - ref_e)}
            Q.qs_plan_free(plan)
        # one cost layer alone: a single phase pass
        layer = g[n:n + 3 * len(edges)]
        plan = Q.qs_plan_create(n, dt, layer, Q.make_opts(mode=F))
        assert [op["type"] for op in Q.qs_plan_ops(plan)] == [4]
        Q.qs_plan_execute(plan, s, th)
        ms = device_ms(torch, lambda: Q.qs_plan_execute(plan, s, th), reps=5)
        res["phase_pass_alone"] = {"ms": ms, "gbps": 2 * (1 << n) * amp / (ms * 1e-3) / 1e9,
                                   "terms": len(Q.qs_plan_ops(plan)[0]["terms"])}
        Q.qs_plan_free(plan)
        # depth 1 against the closed form
        g1, _ = W.qaoa(n, 1, edges)
        plan = Q.qs_plan_create(n, dt, g1, Q.make_opts(mode=F))
        Q.qs_state_set_basis(s, 0)
        Q.qs_plan_execute(plan, s, th[:2])
        res["p1_abs_err_vs_closed_form"] = abs(Q.qs_expval_pauli_sum(s, *H) - qaoa_p1_maxcut(n, edges, *th[:2]))
        Q.qs_plan_free(plan)
        out[dname] = res
        Q.qs_state_free(s)
    return out


def config_qft30(Q, torch, np, st, args):
    """Second n=30 workload of the headline metric: QFT from a seeded basis state,
    complex64 and complex128, per-gate vs contracted plans (tensor-core and
    CUDA-core); sampled amplitudes against the closed form
    psi_y = 2^{-n/2} exp(2 pi i x y / 2^n)."""
    from paper_2509_04955_gb300 import workloads as W
    F, T = Q.QS_MODE_FUSED, Q.QS_MODE_TENSOR
    n = 30
    g = W.qft(n)
    x = W.random_basis_index(n, 30)
    idx = np.unique(np.random.default_rng(0).integers(0, 1 << n, size=4096)).astype(np.uint64)
    want = np.exp(2j * np.pi * ((x * idx.astype(object)) % (1 << n)).astype(np.float64) / (1 << n)) / np.sqrt(1 << n)
    out = {"workload": "QFT n=30, seeded basis input (H, controlled phases, final swaps)", "gates": len(g)}
    variants = {"c64": [("per_gate", None, 3), ("tensor", Q.make_opts(mode=T, tc_min_gates=2), 5)],
                "c128": [("per_gate", None, 2), ("tensor", Q.make_opts(mode=T), 5),
                         ("fused_fp32_pairs", Q.make_opts(mode=F, fuse_k=2, c128_pairs=1), 2)]}
    for dname, dt in (("c64", Q.QS_C64), ("c128", Q.QS_C128)):
        s = Q.qs_state_alloc(n, dt, st)
        res = {}
        amp = 8 if dt == Q.QS_C64 else 16
        for name, opts, reps in variants[dname]:
            plan = Q.qs_plan_create(n, dt, g, opts)
            Q.qs_state_set_basis(s, x)
            Q.qs_plan_execute(plan, s)
            t = device_reps(torch, lambda: Q.qs_plan_execute(plan, s), reps, lambda: Q.qs_state_set_basis(s, x))
            info = Q.qs_plan_info_get(plan)
            got = Q.qs_state_get_amplitudes(s, idx, dt)
            ms = statistics.median(t)
            res[name] = {"ms": spread(t), "passes": info["passes"],
                         "effective_gbps": info["sweeps"] * 2 * (1 << n) * amp / (ms * 1e-3) / 1e9,
                         "max_abs_err_vs_closed_form": float(np.abs(got - want).max())}
            Q.qs_plan_free(plan)
        res["speedup_tensor_vs_per_gate"] = res["per_gate"]["ms"]["median"] / res["tensor"]["ms"]["median"]
        out[dname] = res
        Q.qs_state_free(s)
    return out


def config_qft(Q, torch, np, st, args):
    """QFT n=28 complex128 from a seeded basis state: per-gate vs contraction at
    k = 4, 5 on CUDA cores (FP32 pairs) and k = 5 on tensor cores (the widest
    complex128 block; 6-qubit blocks exist for complex64 only); every amplitude
    against the closed form."""
    from paper_2509_04955_gb300 import workloads as W
    F, T = Q.QS_MODE_FUSED, Q.QS_MODE_TENSOR
    n = 28
    g = W.qft(n)
    x = W.random_basis_index(n, 28)
    s = Q.qs_state_alloc(n, Q.QS_C128, st)
    idx = np.unique(np.random.default_rng(0).integers(0, 1 << n, size=4096))
    want = np.exp(2j * np.pi * ((x * idx) % (1 << n)) / (1 << n)) / np.sqrt(1 << n)
    c1 = {"workload": "QFT n=28 complex128, seeded basis input", "gates": len(g),
          "note": "complex128 tensor-core passes take 5-qubit blocks (k = 6 would need twice the tensor-memory "
                  "columns); tensor_k4 contracts to 4 qubits and pads the blocks to 5"}
    for name, opts, reps in (("per_gate", None, 3),
                             ("fused_k4_fp32_pairs", Q.make_opts(mode=F, fuse_k=4, c128_pairs=1), 3),
                             ("fused_k5_fp32_pairs", Q.make_opts(mode=F, fuse_k=5, tile_qubits=11, low_qubits=3,
                                                                 c128_pairs=1), 3),
                             ("fused_k5_fp64", Q.make_opts(mode=F, fuse_k=5, c128_pairs=2), 2),
                             ("tensor_k5", Q.make_opts(mode=T), 5),
                             ("tensor_k4", Q.make_opts(mode=T, fuse_k=4), 3)):
        plan = Q.qs_plan_create(n, Q.QS_C128, g, opts)
        Q.qs_state_set_basis(s, x)
        Q.qs_plan_execute(plan, s)
        t = device_reps(torch, lambda: Q.qs_plan_execute(plan, s), reps, lambda: Q.qs_state_set_basis(s, x))
        full = np.empty(1 << n, dtype=np.complex128)
        Q.qs_state_copy_to_host(s, full)
        c1[name] = {"ms": spread(t), "passes": Q.qs_plan_info_get(plan)["passes"],
                    "max_abs_err_vs_closed_form": float(np.abs(full[idx] - want).max())}
        Q.qs_plan_free(plan)
        del full
    c1["speedup_tensor_vs_per_gate"] = c1["per_gate"]["ms"]["median"] / c1["tensor_k5"]["ms"]["median"]
    sec, used = oracle_prefix(n, g, 60)
    c1["cpu_oracle"] = {"ms_scaled": sec / 60 * len(g) * 1e3, "threads": used,
                        "sample": f"oracle (plain C, FP64) on {used} threads: the first 60 of the {len(g)} gates "
                                  f"at n={n} in {sec:.2f} s, scaled by the gate count"}
    Q.qs_state_free(s)
    return c1


def config_n32(Q, torch, np, st, args):
    """Random n=32 depth 40 with CZ entanglers (1920 gates), complex64 on tensor
    cores (6-qubit blocks, three split precisions) and on CUDA cores; each
    complex64 result against the complex128 GPU run of the same seed (the
    complex128 tensor-core plan, 64 GiB); one layer per gate timed for the
    per-gate comparator (all 40 layers have the same gate counts)."""
    from paper_2509_04955_gb300 import workloads as W
    F, T = Q.QS_MODE_FUSED, Q.QS_MODE_TENSOR
    n = 32
    g = W.random_layered(n, 40, seed=0, entangler="cz")
    per_layer = len(g) // 40
    s = Q.qs_state_alloc(n, Q.QS_C64, st)
    ref = Q.qs_state_alloc(n, Q.QS_C128, st)
    c2 = {"workload": "random layered n=32 depth 40, CZ entanglers, complex64 (32 GiB)", "gates": len(g)}
    pr = Q.qs_plan_create(n, Q.QS_C128, g, Q.make_opts(mode=T))
    t = device_reps(torch, lambda: Q.qs_plan_execute(pr, ref), 5, lambda: Q.qs_state_set_basis(ref, 0))
    c2["c128_tensor"] = {"ms": spread(t), "passes": Q.qs_plan_info_get(pr)["passes"], "norm": Q.qs_norm(ref)}
    Q.qs_plan_free(pr)
    for name, opts, reps in (("tensor_fp16x3", Q.make_opts(mode=T, tc_min_gates=2, tc_precision=4), 5),
                             ("tensor_fp16x3_k5", Q.make_opts(mode=T, fuse_k=5, tc_min_gates=2, tc_precision=4), 5),
                             ("tensor_bf16x3", Q.make_opts(mode=T, tc_min_gates=2, tc_precision=3), 5),
                             ("tensor_bf16", Q.make_opts(mode=T, tc_min_gates=2, tc_precision=1), 5),
                             ("fused_cuda_cores_k2", Q.make_opts(mode=F, fuse_k=2, tile_qubits=13, low_qubits=4), 5)):
        plan = Q.qs_plan_create(n, Q.QS_C64, g, opts)
        t = device_reps(torch, lambda: Q.qs_plan_execute(plan, s), reps, lambda: Q.qs_state_set_basis(s, 0))
        m, l2 = Q.qs_state_diff(s, ref)
        c2[name] = {"ms": spread(t), "passes": Q.qs_plan_info_get(plan)["passes"], "norm": Q.qs_norm(s),
                    "max_abs_err_vs_c128_gpu": m, "l2_err_vs_c128_gpu": l2}
        Q.qs_plan_free(plan)
    pplan = Q.qs_plan_create(n, Q.QS_C64, g[:per_layer], None)
    t = device_reps(torch, lambda: Q.qs_plan_execute(pplan, s), 5, lambda: Q.qs_state_set_basis(s, 0))
    c2["per_gate_c64"] = {"ms_one_layer": spread(t), "ms_scaled_to_40_layers": 40 * statistics.median(t),
                          "gates_per_layer": per_layer}
    c2["speedup_tensor_vs_per_gate"] = c2["per_gate_c64"]["ms_scaled_to_40_layers"] / c2["tensor_fp16x3"]["ms"]["median"]
    # CPU oracle on the same structure at 26 qubits (the size the oracle checks): one layer, scaled
    g26 = W.random_layered(26, 40, seed=0, entangler="cz")
    sec, used = oracle_prefix(26, g26, len(g26) // 40)
    c2["cpu_oracle_n26"] = {"ms_scaled_to_40_layers": sec * 40 * 1e3, "threads": used,
                            "sample": f"oracle (plain C, FP64) on {used} threads: layer 1 ({len(g26) // 40} gates) "
                                      f"at n=26 in {sec:.2f} s, x 40 layers"}
    Q.qs_plan_free(pplan)
    Q.qs_state_free(ref)
    Q.qs_state_free(s)
    return c2


def config_ucc(Q, torch, np, st, args, hbm_peak=6800.0):
    """UCC-style n=20 complex64, 400 Pauli exponentials, B=64 theta ~ N(0, 0.1):
    one CUDA graph per batch (device-resolved angles, device-built blocks) and
    <H> for a 300-term Pauli sum per state; several replays each. The roofline
    fraction counts one read and one write of every state per pass plus one
    read per distinct x mask of H (the expectation sweeps, served mostly from
    L2) over the measured copy bandwidth."""
    from paper_2509_04955_gb300 import workloads as W
    F, T = Q.QS_MODE_FUSED, Q.QS_MODE_TENSOR
    n, B = 20, 64
    g, _ = W.ucc(n, 400, seed=0)
    th = W.thetas_normal(400, 1, sigma=0.1, batch=B)
    H = W.random_pauli_sum(n, 300, seed=3)
    nx = len(set(int(x) for x in H[1]))
    states = [Q.qs_state_alloc(n, Q.QS_C64, st) for _ in range(B)]
    c3 = {"workload": "UCC-style n=20 complex64, 400 terms, B=64, 300-term <H>", "gates": len(g),
          "x_mask_groups": nx}
    for name, opts, reps in (("fused_k1", Q.make_opts(mode=F, fuse_k=1), 5),
                             ("fused_k4_device_blocks", Q.make_opts(mode=F, fuse_k=4, fuse_parametric=1), 5),
                             ("tensor", Q.make_opts(mode=T, tc_min_gates=2), 5),
                             ("tensor_device_blocks", Q.make_opts(mode=T, tc_min_gates=4, fuse_parametric=1), 5)):
        plan = Q.qs_plan_create(n, Q.QS_C64, g, opts)
        passes = Q.qs_plan_info_get(plan)["passes"]

        def reset():
            for sv in states:
                Q.qs_state_set_basis(sv, 0)
        ex = []
        reset()
        Q.qs_plan_execute_batched(plan, states, th, H)     # captures the graph
        t = device_reps(torch, lambda: ex.append(Q.qs_plan_execute_batched(plan, states, th, H)), reps, reset)
        ms = statistics.median(t)
        nbytes = B * (passes * 2 + nx) * (1 << n) * 8
        c3[name] = {"ms_per_batch": spread(t), "circuits_per_s": B / (ms * 1e-3), "passes_per_circuit": passes,
                    "algorithmic_bytes_per_batch": nbytes, "gbps": nbytes / (ms * 1e-3) / 1e9,
                    "frac_of_hbm": nbytes / (ms * 1e-3) / 1e9 / hbm_peak, "expval_b0": float(ex[-1][0])}
        Q.qs_plan_free(plan)
    for sv in states:
        Q.qs_state_free(sv)
    return c3


def config_hea(Q, torch, np, st, args):
    """HEA n=24, 12 layers (576 parameters): adjoint gradient of a 150-term <H>,
    complex128 (FP64 tile passes; FP32 pairs; tensor-core forward) and
    complex64 (CUDA-core and tensor-core forward); several calls each."""
    from paper_2509_04955_gb300 import workloads as W
    n = 24
    g, p = W.hea(n, 12)
    th = W.thetas_uniform(p, 4)
    H = W.random_pauli_sum(n, 150, seed=4)
    c4 = {"workload": "HEA n=24, 576 parameters, 150-term H, adjoint gradient"}
    grads = {}
    T = Q.QS_MODE_TENSOR
    for dname, dt, variants in (("c128", Q.QS_C128, (("fused_fp64", Q.make_opts(mode=Q.QS_MODE_FUSED, c128_pairs=2)), ("default_fp32_pairs", None),
                                                      ("tensor_forward", Q.make_opts(mode=T, c128_pairs=1)))),
                                ("c64", Q.QS_C64, (("default", None),
                                                   ("tensor_forward", Q.make_opts(mode=T, tc_min_gates=2,
                                                                                  fuse_parametric=1))))):
        s = Q.qs_state_alloc(n, dt, st)
        for vname, o in variants:
            Q.qs_adjoint_grad(s, g, th, *H, opts=o)
            walls = []
            for _ in range(5):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                e, gr = Q.qs_adjoint_grad(s, g, th, *H, opts=o)
                walls.append((time.perf_counter() - t0) * 1e3)
            grads[(dname, vname)] = gr
            c4[f"{dname}_{vname}"] = {"ms": spread(walls), "expval": e}
        Q.qs_state_free(s)
    ref = grads[("c128", "fused_fp64")]
    for k, gr in grads.items():
        c4[f"{k[0]}_{k[1]}"]["max_abs_grad_diff_vs_c128_fp64"] = float(np.abs(gr - ref).max())
    return c4


# The sources each kernel is compiled from (its traffic record is void once they change).
KERNEL_SOURCES = {"k_tc_bulk": ("kernels_tc.cu", "tcgen05.cuh", "cplx.cuh"),
                  "k_tc_block": ("kernels_tc.cu", "tcgen05.cuh", "cplx.cuh"),
                  "k_tc128": ("kernels_tc128.cu", "tcgen05.cuh"),
                  "k_tile": ("kernels_tile.cuh", "cplx.cuh", "dfloat.cuh", "qs_internal.h", "tcgen05.cuh"),
                  "k_tile_bulk": ("kernels_tile.cuh", "cplx.cuh", "dfloat.cuh", "qs_internal.h", "tcgen05.cuh")}


def kernel_hash(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2509_04955_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
