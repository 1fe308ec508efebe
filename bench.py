#!/usr/bin/env python
"""Benchmark of GPU Subdomain Lower Bounding (interval Mean Value Form) on GB300.

One step = Steps 1-3 (Section 3.1) for one B&B iteration of the full-scale
workload: n = 8, objective + 10 inequality constraints, each a seeded
1000-entry tape with + - * / sqr sqrt exp log on guarded domains, box
[-10,10]^8; 64 B&B nodes of a bisection frontier, each split into
8^2 * 4^6 = 2^18 subdomains (2^24 subdomains per step, 11 outputs each), in
one persistent launch replayed as a CUDA graph, adjoint gradients, the
library's choice of bounding kernel (segmented tape-specialised for these
tapes). Metric: subdomain bounds per second = subdomains x outputs enclosed
per second.

Also printed: the roofline of the bounding kernel (algorithmic endpoint
operations per second against the FP64 pipe's peak from unit counts and the
sampled clock, and the issue-slot view beside it), the oracle on the host
cores on a bounded sample of the same workload (cpu_baseline), the same metric
end to end through host buffers (e2e), GPU clocks sampled during the timed
region, the plain-path configuration-2 step of earlier measurements, B&B
wall clock to each configuration's gap (configurations 1, 2, 3 and 5; adjoint
+ batched against the plain forward-mode one-node-per-launch path,
time-capped, final gap reported at the cap) with the oracle-backed B&B on the
host cores beside configurations 1 and 2, and the two training-system
patterns (adjoint vs forward tangents, batched vs per-node launches).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 runs under torchrun, one process per GPU, each rank bounding its own
batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import platform
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MVF subdomain bounds/s and B&B time-to-gap vs plain GPU path; FP64-pipe %"
UNIT = "subdomain-bounds/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nodes", type=int, default=64, help="B&B nodes per step per GPU (2^18 subdomains each)")
    ap.add_argument("--specialize", type=int, default=-1,
                    help="bounding kernel: -1 the library's choice (segmented for these tapes), 0 interpreter, "
                         "1 compact, 3 segmented")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end measurement")
    ap.add_argument("--block-threads", type=int, default=0,
                    help="fixed launch of the headline problem (threads per block; 0: autotuned)")
    ap.add_argument("--blocks-per-sm", type=int, default=0, help="fixed blocks per SM (0: autotuned)")
    ap.add_argument("--seg-sync", type=int, default=-1,
                    help="segmented kernel's chunk synchronisation (-1: autotuned, 0 or 1 fixed)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target oracle sample time")
    ap.add_argument("--bnb", type=int, default=1, help="B&B time-to-gap comparisons (rank 0)")
    ap.add_argument("--bnb-configs", type=str, default="1,2,3,5", help="configurations of the B&B comparison")
    ap.add_argument("--bnb-cap", type=float, default=15.0, help="time cap per B&B run, seconds")
    ap.add_argument("--bnb-cap5", type=float, default=20.0, help="time cap per B&B run on configuration 5")
    ap.add_argument("--oracle-bnb", type=float, default=15.0,
                    help="time cap of the oracle-backed B&B on configurations 1 and 2 (0: skip)")
    ap.add_argument("--secondary", type=int, default=1, help="also time the configuration-2 step")
    ap.add_argument("--patterns", type=int, default=1,
                    help="also time adjoint vs forward (configuration 4) and batched vs per-node (configuration 3)")
    return ap.parse_args()


def workload(rank: int, world: int, nodes: int):
    """full-scale step: `nodes` frontier nodes per rank, 2^18 subdomains each"""
    from paper_2507_20769_gb300 import shard
    from paper_2507_20769_gb300 import workloads as W
    wl = W.config_workload(5)
    t = wl.tape
    boxes_all = W.bisection_frontier(t.root_box, nodes * world, seed=2026)
    b, e = shard.shard_range(nodes * world, rank, world)
    boxes = np.ascontiguousarray(boxes_all[b:e])
    splits = np.ascontiguousarray(np.array([W.full_scale_splits(x, t.root_box) for x in boxes], np.int32))
    return wl, t, boxes, splits


def workload_desc(nodes, world):
    return {"workload": "configuration 5 (full scale): n=8, objective + 10 inequality constraints, seeded "
                        "1000-entry tapes (+ - * / sqr sqrt exp log on guarded domains), box [-10,10]^8; one B&B "
                        "iteration = 64 nodes of a bisection frontier x 2^18 subdomains (8^2 * 4^6 per node) "
                        "= 2^24 subdomains x 11 outputs",
            "nodes_per_step_per_gpu": nodes, "subdomains_per_node": 1 << 18, "outputs": 11,
            "gradients": "adjoint (reverse-mode interval)", "launch": "one persistent launch per step, CUDA graph",
            "l2": "flushed between timed steps (256 MiB write); the kernel's state area (~0.3-0.9 GB) exceeds L2",
            "parallelism": f"nodes sharded over {world} GPU(s)"}


# --------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, device_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"]
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
        except Exception:
            pass
        if uuid:
            cmd += ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------- CPU oracle leg
def cpu_model() -> str:
    """the host CPU's model line from /proc/cpuinfo (AArch64 lists the part number)"""
    try:
        with open("/proc/cpuinfo") as fh:
            lines = fh.read().splitlines()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model name"):
        for ln in lines:
            if ln.startswith(key):
                return ln.split(":", 1)[1].strip()
    parts = sorted({ln.split(":", 1)[1].strip() for ln in lines if ln.startswith("CPU part")})
    known = {"0xd4f": "Neoverse V2", "0xd40": "Neoverse V1", "0xd0c": "Neoverse N1", "0xd49": "Neoverse N2"}
    names = [known.get(x.lower(), f"CPU part {x}") for x in parts]
    return f"{platform.machine()} {', '.join(names)}" if names else platform.machine()


def oracle_rate(t, boxes, splits, seconds: float):
    """The oracle as it stands (fast exp/log mode, adjoint gradients, all host
    cores) runs Steps 1-2 on the first subdomains of the workload's first
    node, as many as fit in about `seconds`; then one core on a tenth of that.
    Returns (subdomain-bounds/s, subdomains, cores, seconds, subdomain-bounds/s
    on one core)."""
    import oracle
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    probe = 64 * cores
    oracle.enclose(t, boxes[0], splits[0], first=0, count=probe, grad_mode="adjoint", tight=False)
    d1 = max(time.perf_counter() - t0, 1e-4)
    S = int(np.prod(splits[0].astype(np.int64)))
    count = int(min(S, max(probe, probe * seconds / d1)))
    t0 = time.perf_counter()
    oracle.enclose(t, boxes[0], splits[0], first=0, count=count, grad_mode="adjoint", tight=False)
    dt = time.perf_counter() - t0
    one = max(16, count // (10 * cores))
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.enclose(t, boxes[0], splits[0], first=0, count=one, grad_mode="adjoint", tight=False)
        d_one = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return count * t.n_out / dt, count, cores, dt, one * t.n_out / d_one


def run_reference(args, rank, world):
    """--impl reference: the oracle on the host cores, same metric and
    workload; each step encloses a bounded sample of the step's subdomains
    (the first ones of the first node), sized so that the whole run stays
    within a few minutes"""
    if rank != 0:
        return 0
    wl, t, boxes, splits = workload(0, 1, args.nodes)
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    import oracle
    _, count, cores, _, _ = oracle_rate(t, boxes, splits, per_step)
    times = []
    S = int(np.prod(splits[0].astype(np.int64)))
    for step in range(args.warmup + args.steps):
        first = (step * count) % max(1, S - count + 1)
        t0 = time.perf_counter()
        oracle.enclose(t, boxes[0], splits[0], first=first, count=count, grad_mode="adjoint", tight=False)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = count * t.n_out * len(times) / total
    sample = (f"{count} subdomains per step (Steps 1-2 on consecutive subdomains of the first node, adjoint "
              f"gradients, fast exp/log mode); CPU: {cpu_model()}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_desc(args.nodes, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ main
def main():
    args = parse()
    from paper_2507_20769_gb300 import shard
    rank, world, local = shard.rank_world()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_2507_20769_gb300 import build as B
    if not os.path.exists(B.LIB):
        if local == 0:
            B.build()
        if world > 1:
            dist.barrier()
    from paper_2507_20769_gb300 import ivb

    wl, t, boxes, splits = workload(rank, world, args.nodes)
    n_nodes = boxes.shape[0]
    subs_step = int(np.prod(splits.astype(np.int64), axis=1).sum())
    units_step = subs_step * t.n_out
    t0 = time.perf_counter()
    p = ivb.Problem(t, grad_mode="adjoint", batched=1, use_graph=1, autotune=1, specialize=args.specialize,
                    max_nodes=max(64, n_nodes), block_threads=args.block_threads, blocks_per_sm=args.blocks_per_sm,
                    seg_sync=args.seg_sync)
    create_s = time.perf_counter() - t0
    boxes_d = torch.from_numpy(boxes).to(dev)
    splits_d = torch.from_numpy(splits).to(dev)
    out = {"lb": torch.empty(n_nodes, dtype=torch.float64, device=dev),
           "infeasible": torch.empty(n_nodes, dtype=torch.uint8, device=dev),
           "ub": torch.empty(n_nodes, dtype=torch.float64, device=dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    warmup = max(3, args.warmup)
    for _ in range(warmup):
        p.bound_nodes_ex(boxes_d, splits_d, out=out)
    torch.cuda.synchronize(dev)

    # ------------------------------------------------ timed region (device-resident)
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = p.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        p.bound_nodes_ex(boxes_d, splits_d, out=out)
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    launches = p.launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_local = sum(step_ms) / 1e3
    t_max = shard.max_over_ranks(t_local, dev)
    units_all = shard.sum_over_ranks(units_step * args.steps, dev)
    value = units_all / t_max

    # ------------------------------------------------ e2e through host buffers
    r = p.bound_nodes_ex(boxes, splits)
    e2e_times = []
    for k in range(max(1, args.e2e_steps)):
        t0 = time.perf_counter()
        r = p.bound_nodes_ex(boxes, splits)
        e2e_times.append(time.perf_counter() - t0)
    e2e_local = sum(e2e_times)
    e2e_max = shard.max_over_ranks(e2e_local, dev)
    e2e_value = shard.sum_over_ranks(units_step * len(e2e_times), dev) / e2e_max
    h2d = boxes.nbytes + splits.nbytes
    d2h = r["lb"].nbytes + r["infeasible"].nbytes + r["ub"].nbytes

    step_s = t_local / args.steps
    roofline = roofline_block(p, subs_step, step_s, clk, dev, probes=True)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(args.nodes, world), "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "steps": len(e2e_times)},
            "gpu_launches": int(launches), "clocks": clk,
            "subdomains_per_s": value / t.n_out, "tuning": p.get_tuning(),
            "kernel": kernel_desc(p, create_s)}

    if rank == 0 and world == 1:
        rate, count, cores, secs, rate1 = oracle_rate(t, boxes, splits, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"Steps 1-2 on the first {count} subdomains of the first node "
                                          f"({secs:.1f} s; adjoint gradients, fast exp/log mode); the reduction "
                                          "of Step 3 is a min over them",
                                "value_1core": rate1, "cpu": cpu_model()}
        line["kernels"] = kernel_compare(t, boxes_d, splits_d, out, flush, stream, subs_step, step_s, dev)
    p.destroy()
    if rank == 0 and world == 1 and args.secondary:
        line["config2"] = config2_step(dev, flush, stream)
    if rank == 0 and world == 1 and args.bnb:
        line["bnb"] = [bnb_compare(int(c), args.bnb_cap5 if c.strip() == "5" else args.bnb_cap)
                       for c in args.bnb_configs.split(",") if c.strip()]
    if rank == 0 and world == 1 and args.oracle_bnb > 0:
        line["oracle_bnb"] = oracle_bnb_study(args.oracle_bnb)
    if rank == 0 and world == 1 and args.patterns:
        line["differentiation"] = differentiation_compare()
        line["batching"] = batching_compare()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def roofline_block(p, subs_step, step_s, clk, dev, probes=False):
    """FP64-pipe roofline of the bounding kernel. `achieved` counts the
    algorithmic work: the static count of outward-rounded endpoint operations
    per subdomain (ivb_op_counts: the value, adjoint and Mean Value Form rules,
    decode) times the subdomains of a step, over the step time (the bounding
    kernel is > 99.9 % of a step: profiles/ has the launch list). `peak` is the
    FP64 pipe from unit counts and the SM clock sampled during the steps:
    2 FP64 lanes per clock per SM x SMs x clock. Beside it, the issue-slot view
    (`pipe_busy_frac`): each category priced in DFMA issue slots at the
    measured rates of the primitives the kernel runs."""
    import torch
    from paper_2507_20769_gb300 import ivb
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = clk.get("sm_mhz") or 2070.0
    peak = 2.0 * sms * clock_mhz * 1e6
    counts = p.op_counts()
    ops_per_sub = sum(counts.values())
    achieved = ops_per_sub * subs_step / step_s
    seg = p.get_segmentation()
    which = {0: "interpreter", 1: "specialised", 2: "segmented"}[p.get_tuning()["kernel"]]
    rf = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "G FP64 endpoint-op/s",
          "frac": achieved / peak, "traffic": traffic_for(subs_step, which),
          "peak_source": f"derived: {sms} SMs x 2 FP64 lanes/clock x {clock_mhz:.0f} MHz (SM clock sampled during "
                         f"the steps) = {2 * peak / 1e12:.3f} FP64 TFLOP/s; MEASURED_PEAKS.json has no FP64 figure",
          "work_per_subdomain": {"endpoint_ops": ops_per_sub, "counts": counts,
                                 "recomputed_operations": seg["recomputed"]},
          "kernel": which}
    if probes:
        names = ("dfma", "dadd", "dmul", "own_rcp", "own_div", "own_sqrt", "own_exp", "own_log")
        rates = {k: ivb.ivb_fp64_probe(k) for k in names}
        probe = rates["dfma"]
        for k, extra in (("own_log", "dadd"), ("own_sqrt", "dmul")):
            # these probes carry one extra round-to-nearest add / multiply per operation
            rates[k] = 1.0 / max(1.0 / rates[k] - 1.0 / rates[extra], 1e-30)
        cost = {"addsub": probe / rates["dadd"], "mul": probe / rates["dmul"], "div": probe / rates["own_div"],
                "rcp": probe / rates["own_rcp"], "sqrt": probe / rates["own_sqrt"], "exp": probe / rates["own_exp"],
                "log": probe / rates["own_log"], "rn": probe / rates["dadd"]}
        slots = sum(counts[k] * cost[k] for k in counts)
        rf["pipe_busy_frac"] = slots * subs_step / step_s / peak
        rf["issue_slot_view"] = {"dfma_slots_per_subdomain": slots, "measured_dfma_probe_glanes": probe / 1e9,
                                 "frac_of_measured_probe": slots * subs_step / step_s / probe,
                                 "primitive_rates_glanes": {k: v / 1e9 for k, v in rates.items()}}
    return rf


def kernel_desc(p, create_s=None):
    s = p.get_specialization()
    d = {"problem_create_seconds": round(create_s, 2)} if create_s is not None else {}
    if not s["active"] or p.get_tuning()["kernel"] == 0:
        d["bounding_kernel"] = "tape interpreter (ivb::k_bound)" + (
            " (the autotuner timed it faster than the compiled kernel)" if s["active"] else "")
        return d
    seg = p.get_segmentation()
    d.update({"bounding_kernel": ("segmented " if seg["chunks"] else "") +
              "tape-specialised (ivb_jit_bound, NVRTC sm_103a at problem creation)",
              "registers": s["registers"], "local_bytes": s["local_bytes"],
              "compile_seconds": round(s["compile_seconds"], 2)})
    if seg["chunks"]:
        d["segmentation"] = seg
    return d


def kernel_compare(t, boxes_d, splits_d, out, flush, stream, subs_step, step_s, dev):
    """the same step through each kernel on its own (bit-identical bounds):
    the tape interpreter, and the segmented tape-specialised kernel with the
    library's segmentation defaults -- the two the library's autotuner
    chooses between for these tapes"""
    import torch
    from paper_2507_20769_gb300 import ivb
    res = {}
    for name, spec in (("interpreter", 0), ("segmented", 3)):
        p = ivb.Problem(t, grad_mode="adjoint", batched=1, use_graph=1, autotune=1, specialize=spec,
                        max_nodes=max(64, int(boxes_d.shape[0])))
        for _ in range(2):
            p.bound_nodes_ex(boxes_d, splits_d, out=out)
        ms = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p.bound_nodes_ex(boxes_d, splits_d, out=out)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        m = float(np.median(ms))
        rf = roofline_block(p, subs_step, m / 1e3, {"sm_mhz": None}, dev)
        res[name] = {"ms_per_step": m, "subdomain_bounds_per_s": subs_step * t.n_out / (m / 1e3),
                     "frac": rf["frac"], "traffic": rf["traffic"], "tuning": p.get_tuning(),
                     "kernel": kernel_desc(p), "vs_headline": (1e3 * step_s) / m}
        p.destroy()
    return res


def config2_step(dev, flush, stream, steps=5):
    """configuration 2 (n=4, objective + 3 constraints of 60 entries, 64 nodes
    x 16^4 subdomains per step), the workload of earlier measurements, with the
    library's choice of kernel (one compact tape-specialised program here)"""
    import torch
    from paper_2507_20769_gb300 import ivb
    from paper_2507_20769_gb300 import workloads as W
    wl = W.config_workload(2)
    t = wl.tape
    boxes = W.bisection_frontier(t.root_box, 64, seed=2026)
    splits = np.tile(wl.splits, (64, 1)).astype(np.int32)
    subs = 64 * int(np.prod(wl.splits))
    bd, sd = torch.from_numpy(boxes).to(dev), torch.from_numpy(splits).to(dev)
    with ivb.Problem(t, grad_mode="adjoint", specialize=-1) as p:
        for _ in range(3):
            p.bound_nodes_ex(bd, sd)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p.bound_nodes_ex(bd, sd)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        step_s = sum(ms) / len(ms) / 1e3
        clk = {"sm_mhz": None}
        rf = roofline_block(p, subs, step_s, clk, dev)
        kd = kernel_desc(p)
    return {"workload": "configuration 2: n=4, 1+3 outputs x 60-entry tapes, 64 nodes x 16^4 subdomains",
            "value": subs * t.n_out / step_s, "unit": UNIT, "ms_per_step": 1e3 * step_s, "steps": steps,
            "roofline": {k: rf[k] for k in ("achieved", "peak", "unit", "frac", "kernel", "traffic")},
            "kernel": kd}


# source files each bounding kernel is built from (the traffic record is valid
# only while they are unchanged)
KERNEL_SOURCES = {
    "interpreter": ("ivb_kernels.cu", "ivb_bound_common.cuh", "ivb_iv.cuh", "ivb_fp64x.cuh", "ivb_emu.cuh"),
    "specialised": ("ivb_jit.cpp", "ivb_bound_common.cuh", "ivb_iv.cuh", "ivb_fp64x.cuh", "ivb_emu.cuh"),
    "segmented": ("ivb_jit_seg.cpp", "ivb_jit.h", "ivb_bound_common.cuh", "ivb_iv.cuh", "ivb_fp64x.cuh", "ivb_emu.cuh"),
}


def kernel_sha(which):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[which]:
        with open(os.path.join(ROOT, "paper_2507_20769_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_for(subs_step, which):
    """DRAM bytes per launch of the bounding kernel from the committed ncu
    summary, scaled by subdomains, while the kernel's sources are the ones
    that were profiled; None otherwise"""
    path = os.path.join(ROOT, "profiles", "bound_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh).get(which)
    if not rec or rec.get("kernel_sha256") != kernel_sha(which):
        return None
    return rec["dram_bytes_per_subdomain"] * subs_step


def _timed(fn, reps=2):
    import torch
    fn()                                   # warm-up (includes autotuning on first use)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def differentiation_compare():
    """configuration 4: n = 16, one 400-entry objective, one node of 2^20
    subdomains per launch: reverse-mode interval adjoints vs forward tangents"""
    from paper_2507_20769_gb300 import ivb
    from paper_2507_20769_gb300 import workloads as W
    wl = W.config_workload(4)
    t = wl.tape
    boxes = t.root_box[None].copy()
    splits = wl.splits[None].astype(np.int32)
    res = {"subdomains": int(np.prod(wl.splits.astype(np.int64))), "n_vars": t.n_vars, "tape_entries": t.n_ops}
    for gm in ("adjoint", "forward"):
        with ivb.Problem(t, grad_mode=gm) as p:
            sec = _timed(lambda: p.bound_nodes(boxes, splits))
            res[gm] = {"seconds": sec, "subdomains_per_s": res["subdomains"] / sec,
                       "endpoint_ops_per_subdomain": sum(p.op_counts().values())}
    res["adjoint_speedup"] = res["forward"]["seconds"] / res["adjoint"]["seconds"]
    return res


def batching_compare():
    """configuration 3: 256 nodes of uneven widths (n = 6, objective + 5
    constraints of 150 entries), per-node subdomain counts 2^10..2^20 from the
    adaptive picker: one persistent launch (CUDA graph) vs one launch per node"""
    from paper_2507_20769_gb300 import ivb
    from paper_2507_20769_gb300 import workloads as W
    t = W.config_tape(3)
    boxes, targets = W.uneven_nodes(t.n_vars, 256, t.root_box, seed=W.config_seed(3) + 5)
    ref_w = t.root_box[:, 1] - t.root_box[:, 0]
    splits = np.stack([ivb.ivb_pick_splits(b, int(tg), "adaptive", ref_w) for b, tg in zip(boxes, targets)])
    S = int(np.prod(splits.astype(np.int64), axis=1).sum())
    res = {"nodes": 256, "subdomains": S}
    for name, opts in (("batched_adjoint", dict(grad_mode="adjoint", batched=1)),
                       ("batched_forward", dict(grad_mode="forward", batched=1)),
                       ("per_node_forward", dict(grad_mode="forward", batched=0))):
        with ivb.Problem(t, max_nodes=256, **opts) as p:
            sec = _timed(lambda: p.bound_nodes(boxes, splits), reps=1)
            res[name] = {"seconds": sec, "subdomain_bounds_per_s": S * t.n_out / sec}
    res["speedup_vs_per_node_forward"] = res["per_node_forward"]["seconds"] / res["batched_adjoint"]["seconds"]
    return res


def bnb_compare(cfg, cap):
    """B&B wall clock to the configuration's gap (Section 3 B&B with this
    library's Subdomain Lower Bounding), time-capped, final bounds at the cap:
      adjoint_batched: the paper's MVF, adjoint gradients, 32 parents per
        iteration bounded in one persistent launch (CUDA graph), the library's
        kernel choice;
      plain_forward_one_node_per_launch: MVF with forward tangents, one node
        per launch;
      host_additions: adjoint + batched with MVF meet NIE, the filtered
        objective, constraint propagation on the host (3 rounds) and CPU/GPU
        overlap.
    The clock covers the solve; problem creation (NVRTC) and the launch
    tuning on one batch of about 2^19 subdomains come first and are reported
    as setup_seconds."""
    from paper_2507_20769_gb300 import ivb
    from paper_2507_20769_gb300 import workloads as W
    wl = W.config_workload(cfg)
    t = wl.tape
    split = (dict(splits=wl.splits) if wl.splits is not None
             else dict(target=1 << (18 if cfg == 5 else 15), strategy="adaptive"))
    res = {"config": cfg, "gap_abs": wl.gap_abs, "gap_rel": wl.gap_rel, "time_cap_s": cap,
           "split": {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in split.items()}}
    arms = (("adjoint_batched", dict(grad_mode="adjoint", batched=1, specialize=-1), dict(batch=32)),
            ("plain_forward_one_node_per_launch", dict(grad_mode="forward", batched=0, specialize=0), dict(batch=1)),
            ("host_additions", dict(grad_mode="adjoint", batched=1, specialize=-1, form="mvf_nie", filter=1),
             dict(batch=32, propagate=3, overlap=1)))
    for name, opts, bopts in arms:
        t0 = time.perf_counter()
        with ivb.Problem(t, **opts) as p:
            # one-time setup outside the clock: compile at creation, and the launch
            # tuned on a batch of the root's bisection frontier with about 2^19
            # subdomains (2 to 64 nodes, the size of one batched iteration)
            if opts.get("batched", 1):
                per = (int(np.prod(split["splits"])) if "splits" in split else int(split["target"]))
                nodes = W.bisection_frontier(t.root_box, int(np.clip(-(-(1 << 19) // per), 2, 64)), seed=1)
                sp = (np.tile(np.asarray(split["splits"], np.int32), (len(nodes), 1)) if "splits" in split else
                      np.stack([ivb.ivb_pick_splits(b, split["target"], split["strategy"],
                                                    t.root_box[:, 1] - t.root_box[:, 0]) for b in nodes]))
                p.bound_nodes(nodes, sp.astype(np.int32))
            setup = time.perf_counter() - t0
            r = p.bnb_solve(t.root_box, eps_abs=wl.gap_abs, eps_rel=wl.gap_rel, time_limit=cap, **split, **bopts)
            kind = kernel_desc(p).get("bounding_kernel")
        gap = r["ub"] - r["lb"]
        res[name] = {"seconds": r["seconds"], "setup_seconds": setup, "converged": r["converged"], "nodes": r["nodes"],
                     "subdomains": r["subdomains"], "lb": r["lb"], "ub": r["ub"],
                     "gap": gap if np.isfinite(gap) else None,
                     "rel_gap": gap / abs(r["ub"]) if np.isfinite(gap) and r["ub"] != 0 else None,
                     "kernel": kind}
    a, b = res["adjoint_batched"], res["plain_forward_one_node_per_launch"]
    c = res["host_additions"]
    if a["converged"] and b["converged"]:
        res["speedup_time_to_gap"] = b["seconds"] / a["seconds"]
    if c["converged"] and b["converged"]:
        res["speedup_time_to_gap_with_host_additions"] = b["seconds"] / c["seconds"]
    return res


def oracle_bnb_study(cap):
    """the oracle as the lower-bounding solver of the same B&B (one node per
    iteration, fast exp/log mode, adjoint gradients), host cores, time-capped"""
    import oracle
    from paper_2507_20769_gb300 import workloads as W
    out = []
    for cfg in (1, 2):
        wl = W.config_workload(cfg)
        r = oracle.bnb(wl.tape, splits=wl.splits, eps_abs=wl.gap_abs, eps_rel=wl.gap_rel, grad_mode="adjoint",
                       tight=False, time_limit=cap)
        gap = r["ub"] - r["lb"]
        out.append({"config": cfg, "seconds": r["seconds"], "converged": r["converged"], "nodes": r["nodes"],
                    "lb": r["lb"], "ub": r["ub"],
                    "rel_gap": gap / abs(r["ub"]) if np.isfinite(gap) and r["ub"] != 0 else None,
                    "cores": oracle.max_threads(), "cpu": cpu_model()})
    return out


if __name__ == "__main__":
    sys.exit(main())
