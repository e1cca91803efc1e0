#!/usr/bin/env python
"""Benchmark of the extended-stabilizer propagation hot path (qx_propagate).

Headline workload (the n=100 configuration at its quoted size, ~1e8 terms /
~5 GB): fan_in_deep_n100.  100 qubits (two words per string), 100,000 gates:
H on every qubit, CX fan-in from the 80 other qubits onto the 20 fan-out
qubits, then 20 rounds of [a random H/S/CX block of ~4,760 gates on the 80
other qubits; RZ(theta ~ U[0, 2 pi)) on fan-out qubit r], and a last block.
Generators Z_0..Z_99, FP64 weights, pruning eps = 1e-14; 80 x 2^20 + 40 =
83,886,120 final terms (3.7 GB of terms).  A step is one qx_propagate of the
whole circuit (initial generators, 20 fan-out steps, the Clifford passes) with
the plan resident on the device.  The terms are larger than L2 and L2 is also
flushed (a 512 MB write) between timed steps, outside the per-step CUDA events.

Metric: Pauli-term updates per second = sum over the K + K' grouped operators
of the terms each was applied to, divided by the step time; beside it,
children per second and the step's algorithmic bytes per second (the
accounting: (parents + children) x (16W + 8) per fan-out step, plus 2N x
(16W + 8) per Clifford pass not fused into an expansion).

Secondary legs: fan_in_heavy_n50 (2.2M terms, L2-resident merge wires, its
FP64-bound kernel against the measured FP64 FMA rate), FP32 weights on both
workloads, serving, gradients, grouping variants and the XYZ + chain sweep.

--gpus N under torchrun: every rank propagates its own seeded instance
(independent problems, no data-path collective): weak scaling.  With
--split generators the ranks share one circuit instead, each propagating the
generators of its range (balanced by the term counts of an untimed run):
strong scaling, with a host gather of per-generator counts and norms.
--impl reference: the CPU oracle (std::map per generator, gate by gate) on
the host cores, each step advancing one heavy generator through a bounded
slice of the same circuit.
"""
import argparse
import json
import os
import platform
import statistics
import select
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "fan_in_deep_n100"
EPS = 1e-14
CONFIG = {
    "workload": WORKLOAD,
    "description": "n=100 (W=2), 100,000 gates: H on all, CX fan-in onto 20 fan-out qubits, "
                   "20 x [random H/S/CX block on the other 80 qubits; RZ(theta ~ U[0,2pi)) on one "
                   "fan-out qubit], last block; generators Z_0..Z_99; 80 x 2^20 + 40 = "
                   "83,886,120 final terms (3.7 GB of terms), FP64 weights, eps=1e-14",
    "n_qubits": 100,
    "gates": 100000,
    "eps": EPS,
    "final_terms": 83886120,
    "l2": "terms larger than L2 (3.7 GB); L2 also flushed between timed steps (512 MB write)",
}
METRIC = "Pauli-term updates/sec"
UNIT = "term-updates/s"
FLUSH_BYTES = 512 << 20
RESERVE_BYTES = 12 << 30  # 83,886,120 + 41,943,080 terms x 44 B = 5.5 GB at the last step, x 2
NON_CLIFFORD = ("T", "TDG", "RX", "RY", "RZ")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def measure_fma_peaks():
    """FP64 and FP32 FMA throughput of this GPU (libqxpeak: independent FMA
    chains, CUDA events, best of 3 launches after an untimed one)."""
    import ctypes

    from paper_2505_03307_gb300 import build as B
    lib = ctypes.CDLL(B.PEAK_LIB)
    lib.qx_peak_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    out = {}
    for bits, iters in ((64, 8192), (32, 131072)):
        best, ms_best = 0.0, 0.0
        for _ in range(3):
            tf, ms = ctypes.c_double(), ctypes.c_double()
            rc = lib.qx_peak_fma(bits, 8, iters, ctypes.byref(tf), ctypes.byref(ms))
            if rc == 0 and tf.value > best:
                best, ms_best = tf.value, ms.value
        out[f"fp{bits}_tflops"] = best
        out[f"fp{bits}_launch_ms"] = ms_best
    out["how"] = ("k_fma_chains: 8 independent FMA chains per thread, 8 blocks of 256 threads "
                  "per SM, 2 flops per FMA, CUDA events, best of 3 launches (qx_peak.cu)")
    return out


def fp64_view(kernel, d, terms_per_launch, fp64_peak):
    """A merge-wire class against the measured FP64 FMA rate: each member of
    a two-member group takes two fused multiply-adds per wire (4 flops)."""
    if kernel != "merge_blocks" or d["ms"] <= 0 or not fp64_peak:
        return None
    flops = 4.0 * terms_per_launch
    t = d["ms"] / max(1, d["launches"]) / 1e3
    tf = flops / t / 1e12
    return {"flops_per_launch": flops, "achieved_tflops": tf, "peak_tflops": fp64_peak,
            "peak_source": "measured FP64 FMA rate (qx_peak.cu)", "frac": tf / fp64_peak}


def ncu_traffic(kernel, workload):
    """Per-launch DRAM bytes of kernel class `kernel` from the committed ncu
    summary of `workload`, if the capture was taken on the current source of
    that kernel (the file and its sha256 are recorded on the kernel's line)."""
    import hashlib
    summ = os.path.join(ROOT, "profiles", f"ncu_traffic_{workload}.txt")
    try:
        for ln in open(summ):
            parts = ln.split()
            if len(parts) == 5 and parts[0] == "traffic_per_launch" and parts[1] == kernel:
                src = os.path.join(ROOT, "paper_2505_03307_gb300", "csrc", parts[3])
                sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
                return float(parts[2]) if sha == parts[4] else None
    except (OSError, ValueError):
        pass
    return None


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.window = None  # host times of the timed region

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __enter__(self):
        # the sampler's start-up (driver and NVML initialisation) stalls kernel
        # launches for several milliseconds: wait for its first sample, so
        # that the start-up happens before the timed region, not inside it
        self.first = ""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        if self.proc:
            ready, _, _ = select.select([self.proc.stdout], [], [], 10.0)
            if ready:
                self.first = self.proc.stdout.readline()
            time.sleep(0.1)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                # the first sample predates the timed region: not counted
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        """Median SM clock and the throttle reasons of the samples taken in
        the timed region (widened by one sampling interval on each side when
        the region is shorter than the interval)."""
        if not self.proc:
            return None
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for ln in getattr(self, "out", "").splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        if self.window:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if not inside:
                inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
            rows = inside
        if not rows:
            return None
        reasons = {nm for r in rows for nm, v in zip(names, r[3]) if v.lower() == "active"}
        return {"sm_mhz": statistics.median(r[1] for r in rows),
                "sm_max_mhz": max(r[2] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "window": "timed region"}


def timed_steps(fn, steps, flush, stream=None):
    """Device time (CUDA events on the launch stream) of `steps` calls of fn,
    L2 flushed before each outside the events; returns (ms list, [the last
    result]).  Earlier results are freed after their step, as a caller that
    propagates in a loop would (holding them all would make every step grow
    the memory pool instead of reusing it)."""
    import torch
    s = stream or torch.cuda.current_stream()
    out, last = [], None
    for _ in range(steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        r = fn()
        e1.record(s)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
        if last is not None:
            last.free()
        last = r
    return out, [last]


def kernel_classes(stats_list):
    kc = {}
    for s in stats_list:
        for name, d in s["kernels"].items():
            a = kc.setdefault(name, {"launches": 0, "alg_bytes": 0, "ms": 0.0})
            a["launches"] += d["launches"]
            a["alg_bytes"] += d["alg_bytes"]
            a["ms"] += d["ms"]
    return kc


# --------------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2505_03307_gb300 import dist as qdist
    from paper_2505_03307_gb300 import qx
    from paper_2505_03307_gb300 import workloads as W

    qx.load_library()
    split = args.split == "generators" and world > 1
    # weak scaling: every rank its own seeded instance; strong: one circuit
    n, instrs = W.fan_in_deep(1 if split else 1 + rank)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    gens = cost = None
    if split:  # ranges balanced by the term counts of an untimed run
        r = qx.propagate(plan, eps=EPS)
        cost = [r.info(g)["nterms"] for g in range(n)]
        r.free()
        gens = qdist.shard_generators(n, rank, world, cost)
    kw = {"eps": EPS} if gens is None else {"eps": EPS, "gens": gens}
    stream = torch.cuda.current_stream()
    # the memory pool reserves the run's peak up front (the last step holds
    # its 42M parents and 84M children, 44 B each, plus scratch), as a server
    # reserves its budget at start-up; growing it inside the first runs maps
    # memory in the middle of them
    qx.reserve_device_memory(RESERVE_BYTES, stream.cuda_stream)
    flush_buf = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    flush = flush_buf.zero_

    # the clock sampler starts before the warm-up steps, so that neither its
    # start-up nor an idle GPU's clock ramp falls into the timed region; only
    # its samples inside the timed region are summarised
    step_ms, stats = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            flush()
            qx.propagate(plan, **kw).free()
        torch.cuda.synchronize()

        # ---- device-resident timed region
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        t_host0 = time.time()
        for _ in range(args.steps):
            flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = qx.propagate(plan, **kw)
            e1.record(stream)
            stats.append(r.stats())
            r.free()
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        clk.mark(t_host0, time.time())
    if world > 1:
        dist.barrier()
    total_ms = sum(step_ms)
    updates = sum(s["term_updates"] for s in stats)
    children = sum(s["children"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    clocks = clk.summary()
    # ---- the same steps again with a CUDA event pair around every launch
    # (kernel shares and the roofline's per-launch times); the events and
    # their readout add host work, so these steps are not the timed ones
    kstats = []
    for _ in range(args.steps):
        flush()
        r = qx.propagate(plan, kernel_timing=True, **kw)
        kstats.append(r.stats())
        r.free()
    torch.cuda.synchronize()
    # ---- a new plan every step: the first run of a plan, with no record of
    # earlier runs (plan building outside the device events)
    cold_ms = []
    for _ in range(max(3, args.steps // 4)):
        p2 = qx.group_ops(qx.load_circuit(n, instrs))
        ms, res = timed_steps(lambda: qx.propagate(p2, **kw), 1, flush, stream)
        cold_ms += ms
        cold_syncs = res[0].stats()["host_syncs"]
        res[0].free()
        del p2

    # ---- end to end through the C ABI: host circuit in, host result out.
    # The circuit is held as qx_instr records (24 B per gate, the C ABI's
    # host input); turning Python tuples into them is binding convenience
    # outside the ABI and happens once, here.
    e2e_ms = []
    e2e_plan_ms = []  # host time of qx_load_circuit + qx_group_ops within each step
    h2d = d2h = 0
    e2e_updates = 0
    pinned = None
    recs = qx.instr_records([g for g, _, _, _ in instrs], [a for _, a, _, _ in instrs],
                            [b for _, _, b, _ in instrs], [th for _, _, _, th in instrs])
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = qx.group_ops(qx.load_circuit_records(n, recs))
        t_plan = time.perf_counter()
        r = qx.propagate(p2, **kw)
        k = r.nterms
        if pinned is None or pinned[2].numel() < k:
            pinned = [torch.empty((k, r.W), dtype=torch.int64, pin_memory=True),
                      torch.empty((k, r.W), dtype=torch.int64, pin_memory=True),
                      torch.empty(k, dtype=torch.float64, pin_memory=True),
                      torch.empty(k, dtype=torch.int32, pin_memory=True)]
        # the export kernel writes the terms into the pinned host buffers
        r.raw_into(*pinned)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
            e2e_plan_ms.append((t_plan - t0) * 1e3)
            e2e_updates += r.stats()["term_updates"]
            h2d = len(instrs) * 24
            d2h = k * (2 * 8 * r.W + 8 + 4)
        r.free()
        del p2
    del pinned

    # ---- strong scaling: the per-generator counts and norms of every rank
    # gathered on the host (the full term arrays stay on their devices)
    gathered = None
    if split:
        def run_range(b, e):
            r = qx.propagate(plan, eps=EPS, gens=(b, e))
            out = [(r.info(g)["nterms"], r.info(g)["sumsq"]) for g in range(e - b)]
            r.free()
            return out
        rows, _ = qdist.run_generator_split(n, rank, world, cost, run_range)
        gathered = {"generators": len(rows), "terms": int(sum(c for c, _ in rows)),
                    "max_norm_error": float(max(abs(s2 - 1.0) for _, s2 in rows))}

    # ---- max of the time over ranks, sum of the work
    total_ms_max, updates_all = qdist.reduce_step_times(total_ms, updates, device="cuda")
    _, children_all = qdist.reduce_step_times(total_ms, children, device="cuda")
    e2e_ms_max, e2e_updates_all = qdist.reduce_step_times(sum(e2e_ms), e2e_updates,
                                                          device="cuda")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    value = updates_all / (total_ms_max / 1e3)
    peak, peak_kind = peaks()
    kc = kernel_classes(kstats)
    dom = max(kc, key=lambda k: kc[k]["ms"])
    d = kc[dom]
    achieved = d["alg_bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] > 0 else 0.0
    share = {k: round(v["ms"] / max(1e-9, sum(x["ms"] for x in kc.values())), 4)
             for k, v in kc.items() if v["launches"]}
    s0 = stats[0]
    ms_step = total_ms_max / args.steps
    step_gbs = s0["alg_bytes"] / (statistics.median(step_ms) / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step,
        "step_ms": [round(t, 4) for t in step_ms],
        "step_host_syncs": [s["host_syncs"] for s in stats],
        "higher_is_better": True, "scaling": "strong" if split else "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded circuits; no dataset)",
        "config": dict(CONFIG, parallelism=(f"generator ranges x{world}" if split else
                                            f"independent circuits x{world}" if world > 1
                                            else "single")),
        "children_per_s": children_all / (total_ms_max / 1e3),
        "step_alg_gbs": step_gbs,
        "step_alg_frac": step_gbs / peak,
        "e2e": {"value": e2e_updates_all / (e2e_ms_max / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms_max / args.steps,
                "plan_ms_median": statistics.median(e2e_plan_ms),
                "path": "qx_load_circuit (host qx_instr records) -> qx_group_ops (new plan) -> "
                        "qx_propagate -> qx_result_raw into pinned host memory"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic(dom, WORKLOAD),
                     "alg_bytes_per_launch": d["alg_bytes"] / max(1, d["launches"]),
                     "avg_launch_ms": d["ms"] / max(1, d["launches"])},
        "kernel_share": share,
        # per-step device time of each kernel class (CUDA events around its
        # launches); the rest of ms_per_step is time between classes
        "kernel_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in kc.items()
                               if v["launches"]},
        "per_step": {"term_updates": s0["term_updates"], "children": s0["children"],
                     "alg_bytes": s0["alg_bytes"], "kernel_launches": s0["kernel_launches"],
                     "host_syncs": s0["host_syncs"], "K": s0["K"], "Kp": s0["Kp"],
                     "final_terms": s0["final_terms"], "fan_steps": s0["fan_steps"],
                     "clifford_passes": s0["clifford_passes"],
                     "guesses_held": s0["guesses_held"]},
        "cold_plan": {"propagate_ms": statistics.median(cold_ms), "host_syncs": cold_syncs,
                      "note": "a new plan for every step (first run of a plan, no record of "
                              "earlier runs); plan building outside the device events"},
        "clocks": clocks,
        "wall_s": t_wall,
    }
    if gathered is not None:
        line["gather"] = gathered
    del plan
    if world == 1:
        fma = measure_fma_peaks()
        line["fma_peaks"] = fma
        if args.mix_steps > 0:
            line["final_mix"] = final_mix_bench(
                qx, W, flush, args.mix_steps, peak,
                line["kernel_ms_per_step"].get("clifford_pass", 0.0))
        if args.heavy_steps > 0:
            line["heavy50"] = heavy50_bench(qx, W, flush, args.heavy_steps, peak,
                                            fma["fp64_tflops"])
        if args.fp32_steps > 0:
            line["fp32"] = fp32_bench(qx, W, flush, args.fp32_steps, statistics.median(step_ms))
        if args.serve_requests > 0:
            line["serving"] = serving_bench(qx, W, args.serve_requests, args.serve_rate)
        if args.adjoint_steps > 0:
            line["adjoint"] = adjoint_bench(qx, W, args.adjoint_steps)
        if args.grouping_steps > 0:
            line["grouping"] = grouping_bench(qx, W, flush, args.grouping_steps)
        if args.xyz_repeats:
            line["xyz_chain"] = xyz_chain_bench(qx, W, [int(r) for r in args.xyz_repeats.split(",")],
                                                flush, oracle_sample=not args.no_cpu_baseline)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _serve_once(qx, reqs, arrays, rate_hz, slots, budget, warm):
    """One pass of the stream at `rate_hz` (0: every request at once):
    circuits/s over the wall clock and latency percentiles."""
    srv = qx.Server(slots=slots, hbm_budget=budget, precision=32)
    for k in range(warm):  # warm-up: planners, engines, allocator pools
        res, _ = srv.wait(srv.submit(reqs[k][1], arrays[k]))
        res.free()
    tickets = [None] * len(reqs)
    scale = 0.0 if rate_hz <= 0 else 1.0
    t0 = time.perf_counter()
    arrival0 = reqs[0][0]

    def submitter():
        for k, (at, n, _) in enumerate(reqs):
            delay = scale * (at - arrival0) * (2000.0 / rate_hz if rate_hz > 0 else 0.0) \
                - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets[k] = srv.submit(n, arrays[k])

    th = threading.Thread(target=submitter)
    th.start()
    lat = []
    for k in range(len(reqs)):
        while tickets[k] is None:
            time.sleep(0.0002)
        res, ms = srv.wait(tickets[k])
        lat.append(ms)
        res.free()
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat.sort()
    return {"rate_hz": rate_hz if rate_hz > 0 else "all at once",
            "circuits_per_s": len(reqs) / wall, "wall_s": wall,
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "batches": st["batches"],
            "mean_batch": st["mean_batch"], "failed": st["failed"], "alone": st["alone"],
            "peak_reserved_bytes": st["peak_reserved"]}


def serving_bench(qx, W, count, rate_hz, slots=2, baseline_count=300):
    """The serving stream (n in [10, 60], 200-5000 Clifford gates, 0-14 T/RZ,
    10k seeded requests): circuits/s and p50/p99 latency of the request loop
    (FP32 weights, batches admitted by the HBM ledger) at Poisson arrival
    rates up to saturation (every request submitted at once), next to the
    same circuits propagated one at a time in FP64 on the same GPU (list-order
    plans, one qx_propagate each)."""
    import torch

    reqs = W.serving_stream(7, count=count, rate_hz=2000.0)
    # the client's marshalling is done before the clock starts
    arrays = [qx.instr_array(instrs) for _, _, instrs in reqs]
    budget = 64 << 30
    rates = [rate_hz] if rate_hz > 0 else [2000.0, 8000.0, 32000.0, 0.0]
    sweep = [_serve_once(qx, reqs, arrays, r, slots, budget, warm=16) for r in rates]
    # one at a time, FP64, no overlap: the first baseline_count circuits
    torch.cuda.synchronize()
    b0 = time.perf_counter()
    for _, n, instrs in reqs[:baseline_count]:
        plan = qx.group_ops(qx.load_circuit(n, instrs))
        r = qx.propagate(plan)
        r.free()
    torch.cuda.synchronize()
    base = baseline_count / (time.perf_counter() - b0)
    # host planning alone, as one planner thread does it (load + push-through
    # plan); the records are marshalled before the clock starts
    recs = [(n, qx.instr_records([g for g, _, _, _ in ins], [a for _, a, _, _ in ins],
                                 [b for _, _, b, _ in ins], [th for _, _, _, th in ins]))
            for _, n, ins in reqs[:baseline_count]]
    p0 = time.perf_counter()
    for n, rec in recs:
        qx.group_ops(qx.load_circuit_records(n, rec), pushthrough=True)
    plan_rate = len(recs) / (time.perf_counter() - p0)
    sat = max(x["circuits_per_s"] for x in sweep)
    return {"requests": count, "slots": slots, "precision": 32, "hbm_budget_bytes": budget,
            "arrivals": "Poisson (seeded), the stream's gaps scaled to each rate",
            "sweep": sweep, "saturated_circuits_per_s": sat,
            "one_at_a_time_fp64_circuits_per_s": base,
            "planning_circuits_per_s_per_thread": plan_rate, "host_cores": os.cpu_count(),
            "one_at_a_time_sample": f"first {baseline_count} requests of the same stream"}


def adjoint_bench(qx, W, steps, warmup=3):
    """Full gradient of a linear functional of output weights with respect to
    all 64 rotation angles of the n = 16, two-layer hardware-efficient ansatz
    (all 16 generators, 5.6M output terms; 4 queried strings per generator,
    a ~ N(0, 1)): forward pass with checkpoints plus reverse pass, next to one
    plain forward propagation of the same circuit."""
    import torch

    n, instrs = W.hea(1, n=16, layers=2)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    r = qx.propagate(plan)
    qg, qp = [], []
    for g in range(n):  # the four heaviest strings of each generator
        strings, w = r.export_strings(g)
        for k in np.argsort(-np.abs(w), kind="stable")[:4]:
            qg.append(g)
            qp.append(strings[int(k)])
    nterms = r.nterms
    r.free()
    a = np.random.default_rng(12).normal(size=len(qg))

    def timed(fn):
        out = []
        for k in range(warmup + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            if k >= warmup:
                out.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(out)

    fwd_ms = timed(lambda: qx.propagate(plan).free())
    tapes = []

    def make_tape():
        if tapes:
            tapes.pop().free()
        tapes.append(qx.Tape(plan, qg, qp))

    tape_ms = timed(make_tape)
    tape = tapes[-1]
    bwd_ms = timed(lambda: tape.backward(a))
    info = tape.info()
    tape.free()
    grad_ms = tape_ms + bwd_ms
    return {"workload": "hea_n16_2layers_all_generators", "rotations": info["rotations"],
            "checkpointed_ops": info["ops"], "checkpoint_bytes": info["held_bytes"],
            "output_terms": nterms, "queries": len(qg), "steps": steps, "warmup": warmup,
            "forward_ms": fwd_ms, "tape_forward_ms": tape_ms, "backward_ms": bwd_ms,
            "gradient_ms": grad_ms, "gradient_over_forward": grad_ms / fwd_ms,
            "angle_gradients_per_s": info["rotations"] / (grad_ms / 1e3),
            "parameter_shift_equivalent_ms": 2 * info["rotations"] * fwd_ms,
            "timing": "host clock around synchronised calls, median of steps"}


def fp32_bench(qx, W, flush, steps, fp64_step_ms, warmup=3):
    """FP32 weights with compensated arithmetic on the headline workload (and
    fan_in_heavy_n50): device time per step (CUDA events, L2 flushed), speed
    against FP64, and the largest relative error against the FP64 oracle's
    closed form (headline: every coefficient is a product of per-qubit cos /
    sin factors times the sign of a Clifford-only propagation) and against
    the FP64 path (fan_in_heavy_n50)."""
    import torch

    out = {"precision": 32, "l2": "flushed between timed steps"}
    n, instrs = W.fan_in_deep(1)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    for _ in range(warmup):
        qx.propagate(plan, precision=32, eps=EPS).free()
    ms, res = timed_steps(lambda: qx.propagate(plan, precision=32, eps=EPS), steps, flush)
    r32 = res[-1]
    st = r32.stats()
    # error against the exact coefficients on sampled strings of 4 generators
    thetas = [th for g, _, _, th in instrs if g == "RZ"]
    rng = np.random.default_rng(3)
    worst = 0.0
    ref64 = qx.propagate(plan, eps=EPS)
    for g in (20, 41, 77, 99):
        strings, w = ref64.export_strings(g)
        pick = rng.choice(len(strings), size=256, replace=False)
        qs = [strings[int(k)] for k in pick]
        got = r32.coeff_batch([g] * len(qs), qs)
        for s_, v in zip(qs, got):
            exact = np.prod([np.cos(thetas[q]) if s_[q] == "X" else np.sin(thetas[q])
                             for q in range(20)])
            sign = np.sign(ref64.coeff(g, s_))
            want = sign * abs(exact)
            worst = max(worst, abs(v - want) / abs(want))
    ref64.free()
    kt = None
    flush()
    rk = qx.propagate(plan, precision=32, eps=EPS, kernel_timing=True)
    kt = {k: round(d["ms"], 4) for k, d in rk.stats()["kernels"].items() if d["launches"]}
    rk.free()
    r32.free()
    m = statistics.median(ms)
    out["fan_in_deep_n100"] = {
        "ms_per_step": m, "term_updates_per_s": st["term_updates"] / (m / 1e3),
        "children_per_s": st["children"] / (m / 1e3),
        "speedup_vs_fp64": fp64_step_ms / m, "max_rel_error_vs_exact": worst,
        "error_sample": "256 sampled strings of generators 20, 41, 77, 99 against "
                        "sign x prod(|cos|, |sin|) in FP64",
        "kernel_ms": kt}
    del plan
    # the merge-heavy secondary workload
    n, instrs = W.fan_in_heavy(1)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    for _ in range(warmup):
        qx.propagate(plan, precision=32).free()
        qx.propagate(plan).free()
    ms32, res = timed_steps(lambda: qx.propagate(plan, precision=32), steps, flush)
    r32 = res[-1]
    ms64, res64 = timed_steps(lambda: qx.propagate(plan), steps, flush)
    ref = res64[-1]
    worst = 0.0
    for g in (16, 33, 49):
        a, b = r32.export_dict(g), ref.export_dict(g)
        assert a.keys() == b.keys()
        for key, w in b.items():
            if abs(w) > 1e-6:
                worst = max(worst, abs(a[key] - w) / abs(w))
    m32, m64 = statistics.median(ms32), statistics.median(ms64)
    out["fan_in_heavy_n50"] = {"ms_per_step": m32, "fp64_ms_per_step": m64,
                               "speedup_vs_fp64": m64 / m32, "max_rel_error_vs_fp64": worst,
                               "error_sample": "generators 16, 33, 49, |w| > 1e-6"}
    r32.free()
    ref.free()
    return out


def heavy50_bench(qx, W, flush, steps, peak, fp64_peak, warmup=3):
    """fan_in_heavy_n50 (n = 50, 2000 gates, 16 T and 16 RZ on 16 fan-out
    qubits, 34 x 65,536 + 16 x 2 = 2,228,256 final terms, 62 MB): the
    merge-heavy case.  Its 16 merge wires run in place over 53 MB of weights
    that stay in L2 between wires, so their algorithmic bytes are not DRAM bytes;
    the wire kernel is bound by the FP64 unit and is reported against the
    measured FP64 FMA rate as well."""
    n, instrs = W.fan_in_heavy(1)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    for _ in range(warmup):
        qx.propagate(plan).free()
    ms, res = timed_steps(lambda: qx.propagate(plan), steps, flush)
    st = res[0].stats()
    for r in res:
        r.free()
    kst = []
    for _ in range(steps):
        flush()
        r = qx.propagate(plan, kernel_timing=True)
        kst.append(r.stats())
        r.free()
    kc = kernel_classes(kst)
    dom = max(kc, key=lambda k: kc[k]["ms"])
    d = kc[dom]
    achieved = d["alg_bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] > 0 else 0.0
    m = statistics.median(ms)
    return {"workload": "fan_in_heavy_n50", "final_terms": st["final_terms"],
            "ms_per_step": m, "term_updates_per_s": st["term_updates"] / (m / 1e3),
            "children_per_s": st["children"] / (m / 1e3),
            "step_alg_gbs": st["alg_bytes"] / (m / 1e3) / 1e9,
            "dominant_kernel": dom, "dominant_share": d["ms"] / sum(v["ms"] for v in kc.values()),
            "dominant_alg_gbs": achieved, "dominant_alg_frac": achieved / peak,
            "dominant_note": "L2-resident: the wires' weights stay in L2 between wires, so "
                             "these algorithmic bytes exceed the DRAM bytes (ncu traffic below)",
            "traffic": ncu_traffic(dom, "fan_in_heavy_n50"),
            "fp64": fp64_view(dom, d, st["final_terms"], fp64_peak),
            "kernel_ms_per_step": {k: round(v["ms"] / steps, 4) for k, v in kc.items()
                                   if v["launches"]},
            "l2": "flushed between timed steps"}


def final_mix_bench(qx, W, flush, steps, peak, base_cliff_ms, warmup=3):
    """The headline circuit with 1000 random H/S/CX gates on all 100 qubits
    appended: the Clifford pass (A4) at HBM scale.  Those gates touch the
    fan-out qubits, so no expansion can absorb them: they run as one in-place
    table-form pass over all 83,886,120 terms (2N x 40 B of algorithmic bytes,
    6.7 GB), timed by CUDA events around the launch.  The class time of the
    headline circuit's own passes (base_cliff_ms: the small steps' passes) is
    taken off to give the all-qubit pass alone."""
    n, instrs = W.fan_in_deep(1, final_mix=1000)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    for _ in range(warmup):
        qx.propagate(plan, eps=EPS).free()
    ms, res = timed_steps(lambda: qx.propagate(plan, eps=EPS), steps, flush)
    st = res[0].stats()
    res[0].free()
    kst = []
    for _ in range(steps):
        flush()
        r = qx.propagate(plan, eps=EPS, kernel_timing=True)
        kst.append(r.stats())
        r.free()
    kc = kernel_classes(kst)
    cp = kc.get("clifford_pass", {"ms": 0.0, "launches": 0, "alg_bytes": 0})
    class_ms = cp["ms"] / steps
    pass_ms = max(1e-6, class_ms - base_cliff_ms)
    pass_bytes = 2 * st["final_terms"] * 40  # 2N x (16W + 8) B at W = 2
    achieved = pass_bytes / (pass_ms / 1e3) / 1e9
    m = statistics.median(ms)
    return {"workload": "fan_in_deep_n100 + 1000 random Clifford gates on all qubits",
            "final_terms": st["final_terms"], "ms_per_step": m,
            "term_updates_per_s": st["term_updates"] / (m / 1e3),
            "clifford_pass_ms_per_step": pass_ms,
            "clifford_pass_alg_bytes": pass_bytes,
            "clifford_class_ms_per_step": class_ms,
            "clifford_pass_note": "the all-qubit pass alone: the Clifford class time minus that "
                                  "of the headline circuit's own (small-step) passes",
            "clifford_pass_alg_gbs": achieved, "clifford_pass_frac": achieved / peak,
            "kernel_ms_per_step": {k: round(v["ms"] / steps, 4) for k, v in kc.items()
                                   if v["launches"]},
            "l2": "terms larger than L2; L2 also flushed between timed steps"}


def grouping_bench(qx, W, flush, steps, warmup=3):
    """List-order grouping (Sec. III.A) against qubit-wise grouping
    (qx_group_ops_dag) and Clifford push-through (qx_group_ops_pushthrough) on
    the paper-sized workloads and a QAOA circuit of RZZ gates: operator
    counts, host planning time and device propagation time (CUDA events, L2
    flushed)."""
    import torch

    cases = [("random_layers_n8", W.random_layers(1), 0.0),
             ("brickwork_n50", W.brickwork(1), 0.0),
             ("fan_in_heavy_n50", W.fan_in_heavy(1), 0.0),
             ("random_pairs_n100", W.random_pairs(1), 1e-14),
             ("qaoa_n20_2layers_rzz", W.qaoa(1, n=20, layers=2), 0.0)]
    out = []
    for name, (n, instrs), eps in cases:
        row = {"workload": name, "gates": len(instrs), "eps": eps}
        circ = qx.load_circuit(n, instrs)
        for mode in ("list", "dag", "push"):
            t0 = time.perf_counter()
            plan = qx.group_ops(circ, dag=(mode == "dag"), pushthrough=(mode == "push"))
            plan_ms = (time.perf_counter() - t0) * 1e3
            times = []
            for k in range(warmup + steps):
                flush()
                s = torch.cuda.current_stream()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(s)
                r = qx.propagate(plan, eps=eps)
                e1.record(s)
                torch.cuda.synchronize()
                if k >= warmup:
                    times.append(e0.elapsed_time(e1))
                st = r.stats()
                nterms = r.nterms
                r.free()
            K, Kp = plan.info()
            row[mode] = {"K": K, "Kp": Kp, "plan_ms": plan_ms,
                         "propagate_ms": statistics.median(times), "final_terms": nterms,
                         "fan_steps": st["fan_steps"], "merge_passes": st["merge_passes"],
                         "clifford_passes": st["clifford_passes"]}
        out.append(row)
    return {"steps": steps, "warmup": warmup, "l2": "flushed between timed steps", "cases": out}


def xyz_chain_bench(qx, W, repeats_list, flush, steps=5, warmup=3, n=12, layers=2,
                    oracle_sample=True):
    """The |XYZ + chain> sweep of the paper's scalability experiment: n = 12,
    2 layers, #Repeats of the RX RY RZ block per layer from 100 up.  Device
    time (generator initialisation to final generators, CUDA events, L2
    flushed between steps) and host planning time per #Repeats; the oracle's
    time at the smallest #Repeats on the host cores."""
    import torch

    out = []
    for reps in repeats_list:
        _, cols = W.xyz_chain_columns(1, n=n, layers=layers, repeats=reps)
        rec = qx.instr_records(*cols)
        t0 = time.perf_counter()
        plan = qx.group_ops(qx.load_circuit_records(n, rec))
        plan_ms = (time.perf_counter() - t0) * 1e3
        times = []
        for k in range(warmup + steps):
            flush()
            s = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s)
            r = qx.propagate(plan)
            e1.record(s)
            torch.cuda.synchronize()
            if k >= warmup:
                times.append(e0.elapsed_time(e1))
            st = r.stats()
            nterms = r.nterms
            r.free()
        ms = statistics.median(times)
        out.append({"repeats": reps, "gates": len(rec), "K": st["K"], "Kp": st["Kp"],
                    "final_terms": nterms, "propagate_ms": ms, "plan_ms": plan_ms,
                    "term_updates_per_s": st["term_updates"] / (ms / 1e3)})
        del plan
    res = {"workload": f"xyz_chain_n{n}_{layers}layers (reconstructed topology)",
           "steps": steps, "warmup": warmup, "l2": "flushed between timed steps",
           "sweep": out}
    if oracle_sample:
        sys.path.insert(0, ROOT)
        from oracle import oracle as O
        _, instrs = W.xyz_chain(1, n=n, layers=layers, repeats=repeats_list[0])
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        O.propagate(n, instrs, mode="plan", threads=cores)
        res["oracle"] = {"repeats": repeats_list[0], "ms": (time.perf_counter() - t0) * 1e3,
                         "cores": cores, "kind": "oracle",
                         "sample": "the whole circuit, one thread per generator"}
    return res


# --------------------------------------------------------------------------- oracle

def operator_bounds(instrs):
    """[begin, end) of every maximal run of one- or two-qubit gates (Sec. III.A)."""
    out = []
    for i, g in enumerate(instrs):
        two = g[0] in ("CX", "CZ")
        if not out or out[-1][2] != two:
            out.append([i, i, two])
        out[-1][1] = i + 1
    return [(b, e) for b, e, _ in out]


class OracleStepper:
    """Advances the oracle (gate mode) through the workload circuit for one
    heavy generator, operator by operator, counting term updates per operator
    like the library does (terms present when the operator starts)."""

    def __init__(self, n, instrs, gen):
        from oracle import oracle as O
        self.O = O
        self.n, self.instrs = n, instrs
        self.ops = operator_bounds(instrs)
        self.gen = gen
        self.reset()

    def reset(self):
        self.k = 0
        z = "".join("Z" if q == self.gen else "I" for q in range(self.n))
        self.strings, self.weights = [z], [1.0]

    def step(self, budget_updates):
        """Apply whole operators until budget_updates term updates; returns
        (updates, seconds)."""
        done = 0
        t0 = time.perf_counter()
        while done < budget_updates:
            if self.k == len(self.ops):
                self.reset()
            b = self.ops[self.k][0]
            e = b
            upd = 0
            while self.k < len(self.ops) and done + upd < budget_updates:
                upd += len(self.strings)
                ob, oe = self.ops[self.k]
                e = oe
                self.k += 1
                # the term count changes only after an operator with a
                # non-Clifford gate: end the slice there so that every
                # operator is counted with the terms present at its start
                if any(g[0] in NON_CLIFFORD for g in self.instrs[ob:oe]):
                    break
            r = self.O.propagate_sum(self.n, self.instrs[b:e], self.strings, self.weights,
                                     mode="gate")
            self.strings, self.weights = r["strings"], r["re"]
            done += upd
        return done, time.perf_counter() - t0


def _oracle_run(gen, budget_s, out, k):
    from paper_2505_03307_gb300 import workloads as W
    n, instrs = W.fan_in_deep(1)
    st = OracleStepper(n, instrs, gen)
    done, secs = 0, 0.0
    while secs < budget_s:
        u, s = st.step(2_000_000)
        done += u
        secs += s
    out[k] = (done, secs)


def cpu_baseline(budget_s):
    """The oracle on the host cores: one thread advancing heavy generator
    Z_20 of the headline circuit gate by gate (through whole operators, term
    updates counted per operator like the library), and one thread per core,
    each on its own heavy generator (generators are independent), for about
    budget_s seconds each."""
    cores = os.cpu_count() or 1
    one = [None]
    _oracle_run(20, budget_s, one, 0)
    single = one[0][0] / one[0][1]
    res = [None] * cores
    ths = [threading.Thread(target=_oracle_run, args=(20 + (k % 80), budget_s, res, k))
           for k in range(cores)]
    t0 = time.perf_counter()
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    wall = time.perf_counter() - t0
    allc = sum(r[0] for r in res) / wall
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": cores,
            "single_thread": {"value": single, "cores": 1,
                              "sample": f"generator Z_20, {one[0][1]:.1f} s ({one[0][0]} term "
                                        f"updates)"},
            "sample": f"one thread per core, thread k advancing generator Z_(20 + k mod 80) of "
                      f"the same circuit gate by gate through whole operators for ~{budget_s:.0f} "
                      f"s ({wall:.1f} s wall); term updates counted per operator"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2505_03307_gb300 import workloads as W

    O.build()
    n, instrs = W.fan_in_deep(1)
    st = OracleStepper(n, instrs, 20)
    budget = 3_000_000
    for _ in range(args.warmup):
        st.step(budget)
    times, done = [], 0
    for _ in range(args.steps):
        u, s = st.step(budget)
        done += u
        times.append(s)
    value = done / sum(times)
    sample = ("each step: about 3M term updates of generator Z_20, gate by gate through whole "
              "operators of the same circuit; single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded circuits; no dataset)",
        "config": dict(CONFIG, parallelism="single"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile(args):
    """--warmup then --profile-steps propagations of the headline workload on
    cuda:0 with nothing else on the device: the command the committed ncu
    summaries name.  The profiled propagations sit in the NVTX range
    "qx_profile"."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_03307_gb300 import qx
    from paper_2505_03307_gb300 import workloads as W
    torch.cuda.set_device(0)
    # --profile-nfan < 20: the same construction with fewer fan-out qubits
    # (80 generators of 2^k terms), a small case for multi-pass captures
    n, instrs = W.fan_in_deep(1, n_s=args.profile_nfan, final_mix=args.profile_mix)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    launches = 0
    for k in range(args.warmup + args.profile_steps):
        if k == args.warmup:  # ncu --nvtx --nvtx-include "qx_profile/" captures from here
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("qx_profile")
        r = qx.propagate(plan, eps=EPS)
        launches = r.stats()["kernel_launches"]
        r.free()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_steps": args.profile_steps, "warmup": args.warmup,
                      "kernel_launches_per_propagation": launches}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--split", default="circuits", choices=["circuits", "generators"],
                    help="N > 1: independent circuits per rank (weak) or one circuit split "
                         "by generator range (strong)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="seconds of oracle work per CPU-baseline leg")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the serving stream (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="Poisson arrival rate (Hz) of the serving leg; 0: a sweep up to saturation")
    ap.add_argument("--adjoint-steps", type=int, default=5,
                    help="timed steps of the gradient leg (0: skip)")
    ap.add_argument("--fp32-steps", type=int, default=5,
                    help="timed steps of the FP32 legs (0: skip)")
    ap.add_argument("--mix-steps", type=int, default=5,
                    help="steps of the headline circuit with an all-qubit Clifford block appended "
                         "(0: skip)")
    ap.add_argument("--heavy-steps", type=int, default=10,
                    help="timed steps of the fan_in_heavy_n50 leg (0: skip)")
    ap.add_argument("--grouping-steps", type=int, default=5,
                    help="timed steps per case of the grouping comparison (0: skip)")
    ap.add_argument("--xyz-repeats", default="100,1000,10000,100000",
                    help="#Repeats of the XYZ + chain sweep, comma-separated ('' skips it)")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only --warmup then this many propagations of the headline workload, "
                         "no timing and no other legs (for ncu launch lists)")
    ap.add_argument("--profile-mix", type=int, default=0,
                    help="random Clifford gates on all qubits appended to the --profile-steps "
                         "workload (an all-qubit table-form pass over every term)")
    ap.add_argument("--profile-nfan", type=int, default=20,
                    help="fan-out qubits of the --profile-steps workload (20: the headline)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_steps > 0:
        run_profile(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
