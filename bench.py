#!/usr/bin/env python
"""Benchmark of GPU Subdomain Lower Bounding (interval Mean Value Form) on GB300.

One step = Steps 1-3 (Section 3.1) for one batch of B&B nodes of the
configuration-2 workload (n = 4, objective + 3 inequality constraints, seeded
60-entry tapes with all eight intrinsics, box [-5,5]^4, 16^4 = 65536 subdomains
per node), in one persistent launch replayed as a CUDA graph, adjoint gradients.
Metric: subdomain bounds per second = subdomains x outputs enclosed per second.

Also printed: the roofline of the bounding kernel against the FP64 pipe peak
measured live, the oracle on the host cores (cpu_baseline), the same metric end
to end through host buffers (e2e), GPU clocks sampled during the timed region,
and B&B wall clock to relative gap 1e-3 for the adjoint+batched path and the
plain forward-mode one-node-per-launch path (time-capped).

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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nodes", type=int, default=64, help="nodes per step per GPU")
    ap.add_argument("--bnb", type=int, default=1, help="run the B&B time-to-gap comparison (rank 0)")
    ap.add_argument("--bnb-time", type=float, default=45.0, help="time cap per B&B run, seconds")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target oracle sample time")
    ap.add_argument("--bnb-configs", type=str, default="",
                    help="comma list of configurations (2, 3, 5) for a B&B time-to-gap study with the host "
                         "additions switched on one by one (minutes; off by default)")
    ap.add_argument("--bnb-config-cap", type=float, default=90.0, help="time cap per run of that study, seconds")
    ap.add_argument("--oracle-bnb", type=float, default=0.0,
                    help="> 0: also run the oracle-backed B&B (host cores) on configurations 1 and 2 with this "
                         "time cap in seconds (off by default)")
    ap.add_argument("--specialize", type=int, default=1,
                    help="1: tape-specialised bounding kernel (NVRTC at problem creation); 0: tape interpreter")
    ap.add_argument("--patterns", type=int, default=1,
                    help="also time adjoint vs forward (configuration 4) and batched vs per-node (configuration 3)")
    return ap.parse_args()


def workload(rank: int, world: int, nodes: int):
    from paper_2507_20769_gb300 import shard
    from paper_2507_20769_gb300 import workloads as W
    wl = W.config_workload(2)
    t = wl.tape
    boxes_all = W.bisection_frontier(t.root_box, nodes * world, seed=2026)
    b, e = shard.shard_range(nodes * world, rank, world)
    boxes = np.ascontiguousarray(boxes_all[b:e])
    splits = np.ascontiguousarray(np.tile(wl.splits, (boxes.shape[0], 1)).astype(np.int32))
    return wl, t, boxes, splits


def workload_desc(nodes, world):
    return {"workload": "configuration 2: n=4, objective + 3 inequality constraints, seeded 60-entry tapes "
                        "(+ - * / sqr sqrt exp log on guarded domains), box [-5,5]^4, 16^4 = 65536 subdomains "
                        "per node, batch of B&B nodes from a bisection frontier",
            "nodes_per_step_per_gpu": nodes, "subdomains_per_node": 65536, "outputs": 4,
            "gradients": "adjoint (reverse-mode interval)", "launch": "one persistent launch per step, CUDA graph",
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"nodes sharded over {world} GPU(s)"}


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
    cores) runs Steps 1-3 on whole workload nodes, as many as fit in about
    `seconds`; then one core on 8192 subdomains of the first node. Returns
    (subdomain-bounds/s, nodes, subdomains per node, cores, seconds,
    subdomain-bounds/s on one core)."""
    import oracle
    cores = oracle.max_threads()
    S = int(np.prod(splits[0].astype(np.int64)))
    t0 = time.perf_counter()
    oracle.bound_nodes(t, boxes[:1], splits[:1], grad_mode="adjoint", tight=False)
    d1 = max(time.perf_counter() - t0, 1e-4)
    k = int(min(len(boxes), max(1, round(seconds / d1))))
    t0 = time.perf_counter()
    oracle.bound_nodes(t, boxes[:k], splits[:k], grad_mode="adjoint", tight=False)
    dt = time.perf_counter() - t0
    one = min(8192, S)
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.enclose(t, boxes[0], splits[0], first=0, count=one, grad_mode="adjoint", tight=False)
        d_one = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return k * S * t.n_out / dt, k, S, cores, dt, one * t.n_out / d_one


def run_reference(args, rank, world):
    """--impl reference: the oracle on the host cores, same metric and workload;
    each step bounds whole nodes (Steps 1-3), as many as fit its time share"""
    if rank != 0:
        return 0
    wl, t, boxes, splits = workload(0, 1, args.nodes)
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    import oracle
    _, k, S, cores, _, _ = oracle_rate(t, boxes, splits, per_step)
    times = []
    for step in range(args.warmup + args.steps):
        first = (step * k) % max(1, len(boxes) - k + 1)
        t0 = time.perf_counter()
        oracle.bound_nodes(t, boxes[first:first + k], splits[first:first + k], grad_mode="adjoint", tight=False)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = k * S * t.n_out * len(times) / total
    sample = (f"{k} whole nodes of {S} subdomains per step (Steps 1-3, adjoint gradients, fast exp/log mode); "
              f"CPU: {cpu_model()}")
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
    p = ivb.Problem(t, grad_mode="adjoint", batched=1, use_graph=1, autotune=1, specialize=args.specialize)
    boxes_d = torch.from_numpy(boxes).to(dev)
    splits_d = torch.from_numpy(splits).to(dev)
    out = {"lb": torch.empty(n_nodes, dtype=torch.float64, device=dev),
           "infeasible": torch.empty(n_nodes, dtype=torch.uint8, device=dev),
           "ub": torch.empty(n_nodes, dtype=torch.float64, device=dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(3, args.warmup)):
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
    e2e_times = []
    for k in range(args.steps + 1):
        t0 = time.perf_counter()
        r = p.bound_nodes_ex(boxes, splits)
        if k > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e_local = sum(e2e_times)
    e2e_max = shard.max_over_ranks(e2e_local, dev)
    e2e_value = shard.sum_over_ranks(units_step * len(e2e_times), dev) / e2e_max
    h2d = boxes.nbytes + splits.nbytes
    d2h = r["lb"].nbytes + r["infeasible"].nbytes + r["ub"].nbytes

    # ------------------------------------------------ roofline (FP64 pipe, ALU bound)
    names = ("dfma", "dadd", "dmul", "ddiv", "drcp", "dsqrt", "exp", "log",
             "own_rcp", "own_div", "own_sqrt", "own_exp", "own_log", "emu_mul", "mixed_mul", "emu_add", "mixed_add")
    rates = {k: ivb.ivb_fp64_probe(k) for k in names}
    probe = rates["dfma"]   # measured DFMA lane-op/s: the unit of the per-primitive costs
    # peak of the FP64 pipe from unit counts and clocks: 2 DFMA lanes per clock per SM on
    # GB300 (ncu's dfma peak_sustained), times the SMs and the SM clock sampled during the steps
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = clk.get("sm_mhz") or 2070.0
    peak = 2.0 * sms * clock_mhz * 1e6
    for k, extra in (("log", "dadd"), ("own_log", "dadd"), ("dsqrt", "dmul"), ("own_sqrt", "dmul")):
        # these probes carry one extra round-to-nearest add / multiply per operation
        rates[k] = 1.0 / max(1.0 / rates[k] - 1.0 / rates[extra], 1e-30)
    # cost of each category in DFMA issue slots: the primitives the kernel runs
    cost = {"addsub": probe / rates["dadd"], "mul": probe / rates["dmul"], "div": probe / rates["own_div"],
            "rcp": probe / rates["own_rcp"], "sqrt": probe / rates["own_sqrt"], "exp": probe / rates["own_exp"],
            "log": probe / rates["own_log"], "rn": probe / rates["dadd"]}
    vendor = {"addsub": probe / rates["dadd"], "mul": probe / rates["dmul"], "div": probe / rates["ddiv"],
              "rcp": probe / rates["drcp"], "sqrt": probe / rates["dsqrt"], "exp": probe / rates["exp"],
              "log": probe / rates["log"], "rn": probe / rates["dadd"]}
    counts = p.op_counts()
    slots_per_sub = sum(counts[k] * cost[k] for k in counts)
    vendor_slots = sum(counts[k] * vendor[k] for k in counts)
    ops_per_sub = sum(counts.values())
    step_s = t_local / args.steps
    achieved = slots_per_sub * subs_step / step_s
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                "unit": "G FP64 DFMA-slot/s", "frac": achieved / peak,
                "traffic": traffic_for(subs_step, "specialised" if args.specialize else "interpreter"),
                "peak_source": f"derived: {sms} SMs x 2 FP64 lanes/clock x {clock_mhz:.0f} MHz (SM clock sampled "
                               f"during the steps) = {2 * peak / 1e12:.3f} FP64 TFLOP/s",
                "measured_probe_peak": probe / 1e9, "frac_of_measured_probe": achieved / probe,
                "probe_note": "ivb_fp64_probe: 8 independent DFMA chains per thread, 32 warps per SM; "
                              "primitive costs are in units of this rate",
                "work_per_subdomain": {"endpoint_ops": ops_per_sub, "dfma_slots": slots_per_sub,
                                       "counts": counts,
                                       "dfma_slots_with_cuda_intrinsics": vendor_slots},
                "primitive_rates_glanes": {k: v / 1e9 for k, v in rates.items()},
                "kernel_share_note": "step time includes the two tiny key/finalize kernels and the queue copy; "
                                     "the bounding kernel's share is in profiles/"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(args.nodes, world), "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches), "clocks": clk,
            "subdomains_per_s": value / t.n_out, "tuning": p.get_tuning(),
            "kernel": kernel_desc(p)}

    if rank == 0 and world == 1:
        rate, k, S, cores, secs, rate1 = oracle_rate(t, boxes, splits, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"Steps 1-3 on {k} whole nodes of {S} subdomains ({secs:.1f} s; "
                                          "adjoint gradients, fast exp/log mode)",
                                "value_1core": rate1, "cpu": cpu_model()}
    if rank == 0 and world == 1 and args.specialize:
        line["interpreter"] = interpreter_compare(t, boxes_d, splits_d, out, flush, stream, subs_step, step_s)
    if rank == 0 and world == 1 and args.bnb:
        line["bnb"] = bnb_compare(t, wl, args.bnb_time)
    if rank == 0 and world == 1 and args.oracle_bnb > 0:
        line["oracle_bnb"] = oracle_bnb_study(args.oracle_bnb)
    if rank == 0 and world == 1 and args.bnb_configs:
        line["bnb_configs"] = bnb_config_study([int(c) for c in args.bnb_configs.split(",")], args.bnb_config_cap)
    if rank == 0 and world == 1 and args.patterns:
        line["differentiation"] = differentiation_compare()
        line["batching"] = batching_compare()
    p.destroy()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def kernel_desc(p):
    s = p.get_specialization()
    if not s["active"]:
        return {"bounding_kernel": "tape interpreter (ivb::k_bound)"}
    return {"bounding_kernel": "tape-specialised (ivb_jit_bound, NVRTC sm_103a at problem creation)",
            "registers": s["registers"], "local_bytes": s["local_bytes"],
            "compile_seconds": round(s["compile_seconds"], 2)}


def interpreter_compare(t, boxes_d, splits_d, out, flush, stream, subs_step, step_s):
    """the same step through the tape interpreter (bit-identical bounds), for context"""
    import torch
    from paper_2507_20769_gb300 import ivb
    p = ivb.Problem(t, grad_mode="adjoint", batched=1, use_graph=1, autotune=1, specialize=0)
    for _ in range(3):
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
    p.destroy()
    m = float(np.median(ms))
    return {"ms_per_step": m, "subdomains_per_s": subs_step / (m / 1e3),
            "specialised_speedup": m / (1e3 * step_s)}


# source files each bounding kernel is built from (the traffic record is valid
# only while they are unchanged)
KERNEL_SOURCES = {
    "interpreter": ("ivb_kernels.cu", "ivb_bound_common.cuh", "ivb_iv.cuh", "ivb_fp64x.cuh", "ivb_emu.cuh"),
    "specialised": ("ivb_jit.cpp", "ivb_bound_common.cuh", "ivb_iv.cuh", "ivb_fp64x.cuh", "ivb_emu.cuh"),
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


def bnb_compare(t, wl, cap):
    """B&B wall clock to relative gap 1e-3: adjoint + batched vs plain"""
    from paper_2507_20769_gb300 import ivb
    res = {"gap_rel": wl.gap_rel, "time_cap_s": cap}
    arms = (
        # the paper's method on this path: adjoint gradients, batched nodes, CUDA graph
        ("adjoint_batched", dict(grad_mode="adjoint", batched=1), dict(batch=32)),
        # plus the host-side additions: constraint propagation of every child and
        # the host overlapping the GPU (next batch enqueued before the last is absorbed),
        # with the tape-specialised kernel
        ("adjoint_batched_propagate_overlap_specialised", dict(grad_mode="adjoint", batched=1, specialize=1),
         dict(batch=32, propagate=3, overlap=1)),
        ("plain_forward_one_node_per_launch", dict(grad_mode="forward", batched=0), dict(batch=1)),
    )
    for name, opts, bopts in arms:
        with ivb.Problem(t, **opts) as p:
            r = p.bnb_solve(t.root_box, splits=wl.splits, eps_abs=0.0, eps_rel=wl.gap_rel, time_limit=cap, **bopts)
        gap = r["ub"] - r["lb"]
        res[name] = {"seconds": r["seconds"], "converged": r["converged"], "nodes": r["nodes"],
                     "lb": r["lb"], "ub": r["ub"], "gap": gap,
                     "rel_gap": gap / max(abs(r["ub"]), 1e-300) if np.isfinite(gap) else None}
    a, b = res["adjoint_batched"], res["plain_forward_one_node_per_launch"]
    c = res["adjoint_batched_propagate_overlap_specialised"]
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
        out.append({"config": cfg, "seconds": r["seconds"], "converged": r["converged"], "nodes": r["nodes"],
                    "lb": r["lb"], "ub": r["ub"], "cores": oracle.max_threads(), "cpu": cpu_model()})
    return out


def bnb_config_study(configs, cap):
    """B&B to each configuration's gap: adjoint + batched (32 parents per
    iteration), then + constraint propagation, + CPU/GPU overlap, + the
    tape-specialised kernel (not for configuration 5, whose tapes are too
    large to compile quickly), and with MVF meet NIE and the filtered
    objective. Configurations 3 and 5 split each node by the
    adaptive picker (2^15 and 2^18 subdomains per node)."""
    from paper_2507_20769_gb300 import ivb
    from paper_2507_20769_gb300 import workloads as W
    out = []
    for cfg in configs:
        wl = W.config_workload(cfg)
        t = wl.tape
        split = (dict(splits=wl.splits) if wl.splits is not None
                 else dict(target=1 << (18 if cfg == 5 else 15), strategy="adaptive"))
        arms = [("adjoint_batched", {}, {}), ("+propagate", {}, dict(propagate=3)),
                ("+propagate+overlap", {}, dict(propagate=3, overlap=1))]
        if cfg != 5:
            arms.append(("+propagate+overlap+specialised", dict(specialize=1), dict(propagate=3, overlap=1)))
        # the bound form: MVF intersected with the natural interval extension, filtered objective
        arms.append(("+propagate+overlap+mvf_nie+filter", dict(form="mvf_nie", filter=1),
                     dict(propagate=3, overlap=1)))
        for name, popts, bopts in arms:
            with ivb.Problem(t, grad_mode="adjoint", batched=1, **popts) as p:
                r = p.bnb_solve(t.root_box, batch=32, eps_abs=wl.gap_abs, eps_rel=wl.gap_rel, time_limit=cap,
                                **split, **bopts)
            gap = r["ub"] - r["lb"]
            out.append({"config": cfg, "arm": name, "seconds": r["seconds"], "converged": r["converged"],
                        "nodes": r["nodes"], "lb": r["lb"], "ub": r["ub"],
                        "rel_gap": gap / abs(r["ub"]) if np.isfinite(gap) and r["ub"] != 0 else None})
    return out


if __name__ == "__main__":
    sys.exit(main())
