#!/usr/bin/env python
"""Benchmark of the extended-stabilizer propagation hot path (qx_propagate).

Workload (the n=50 Clifford+T configuration at its quoted size): 50 qubits,
2000 gates, 16 T and 16 RZ gates on 16 fan-out qubits, generators Z_0..Z_49;
34 generators reach 65,536 terms each (2,228,256 terms in all).  A step is one
qx_propagate of the whole circuit: initial generators (create_Z_j), fused
Clifford passes, the 2^16 expansion, 16 index-accumulation passes and the
Clifford tail, with inputs resident on the device.  L2 is flushed (a 512 MB
write) between timed steps, outside the per-step CUDA events.

Metric: Pauli-term updates per second = sum over the K + K' grouped operators
of the terms each was applied to, divided by the step time.

--gpus N under torchrun: every rank propagates its own seeded instance
(independent problems, no data-path collective): weak scaling.
--impl reference: the CPU oracle (std::map per generator, gate by gate) on
the host cores, each step advancing one heavy generator through a bounded
slice of the same circuit.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "fan_in_heavy_n50"
CONFIG = {
    "workload": WORKLOAD,
    "description": "n=50, 2000 gates (H/S/CNOT + 16 T + 16 RZ on 16 fan-out qubits), "
                   "generators Z_0..Z_49, 34 x 65536 + 16 x 2 = 2,228,256 final terms, "
                   "FP64 weights, eps=0",
    "n_qubits": 50,
    "gates": 2000,
    "final_terms": 2228256,
    "l2": "flushed between timed steps (512 MB write)",
}
METRIC = "Pauli-term updates/sec"
UNIT = "term-updates/s"
FLUSH_BYTES = 512 << 20
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


# Nominal FP64 rate of the GPU (FP64 is far below the tensor rates on this
# part): the ceiling of a merge wire, whose bytes stay in L2 between wires.
FP64_PEAK_TFLOPS = 1.25


def fp64_view(kernel, d, s0):
    """The dominant merge-wire class against the FP64 unit: each term of a
    two-member group takes two fused multiply-adds per wire (4 flops); on the
    bench workload that is every term but the 32 of the 16 two-term
    generators.  None for other classes."""
    if kernel != "merge_blocks" or d["ms"] <= 0:
        return None
    flops = 4.0 * s0["final_terms"]
    t = d["ms"] / max(1, d["launches"]) / 1e3
    tf = flops / t / 1e12
    return {"flops_per_launch": flops, "achieved_tflops": tf, "peak_tflops": FP64_PEAK_TFLOPS,
            "peak_source": "nominal (recipe)", "frac": tf / FP64_PEAK_TFLOPS}


def ncu_traffic(kernel):
    """Per-launch DRAM bytes of kernel class `kernel` from the committed ncu
    summary, if the capture was taken on the current source of that kernel
    (the file and its sha256 are recorded on the kernel's line)."""
    import hashlib
    summ = os.path.join(ROOT, "profiles", "ncu_traffic_fan_in_heavy_n50.txt")
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


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "out", "").splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


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
    from paper_2505_03307_gb300 import qx
    from paper_2505_03307_gb300 import workloads as W

    qx.load_library()
    n, instrs = W.fan_in_heavy(1 + rank)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        r = qx.propagate(plan)
        r.free()
    torch.cuda.synchronize()

    # ---- device-resident timed region
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, stats = [], []
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = qx.propagate(plan)
            e1.record(stream)
            stats.append(r.stats())
            r.free()
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    total_ms = sum(step_ms)
    updates = sum(s["term_updates"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    clocks = clk.summary()
    # ---- the same steps again with a CUDA event pair around every launch
    # (kernel shares and the roofline's per-launch times); the events and
    # their readout add host work, so these steps are not the timed ones
    kstats = []
    for _ in range(args.steps):
        flush.zero_()
        r = qx.propagate(plan, kernel_timing=True)
        kstats.append(r.stats())
        r.free()
    torch.cuda.synchronize()

    # ---- end to end through the C ABI: host circuit in, host result out.
    # The circuit is held as qx_instr records (24 B per gate, the C ABI's
    # host input); turning Python tuples into them is binding convenience
    # outside the ABI and happens once, here.
    e2e_ms = []
    h2d = d2h = 0
    e2e_updates = 0
    pinned = None
    recs = qx.instr_records([g for g, _, _, _ in instrs], [a for _, a, _, _ in instrs],
                            [b for _, _, b, _ in instrs], [th for _, _, _, th in instrs])
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = qx.group_ops(qx.load_circuit_records(n, recs))
        r = qx.propagate(p2)
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
            e2e_updates += r.stats()["term_updates"]
            h2d = len(instrs) * 24
            d2h = k * (2 * 8 * r.W + 8 + 4)
        r.free()
        del p2

    # ---- max of the time over ranks, sum of the work
    from paper_2505_03307_gb300 import dist as qdist
    total_ms_max, updates_all = qdist.reduce_step_times(total_ms, updates, device="cuda")
    e2e_ms_max, e2e_updates_all = qdist.reduce_step_times(sum(e2e_ms), e2e_updates,
                                                          device="cuda")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    value = updates_all / (total_ms_max / 1e3)
    # ---- roofline of the dominant kernel class
    kc = {}
    for s in kstats:
        for name, d in s["kernels"].items():
            a = kc.setdefault(name, {"launches": 0, "alg_bytes": 0, "ms": 0.0})
            a["launches"] += d["launches"]
            a["alg_bytes"] += d["alg_bytes"]
            a["ms"] += d["ms"]
    dom = max(kc, key=lambda k: kc[k]["ms"])
    d = kc[dom]
    peak, peak_kind = peaks()
    achieved = d["alg_bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] > 0 else 0.0
    traffic = ncu_traffic(dom)
    share = {k: round(v["ms"] / max(1e-9, sum(x["ms"] for x in kc.values())), 4)
             for k, v in kc.items() if v["launches"]}
    s0 = stats[0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded circuits; no dataset)",
        "config": dict(CONFIG, parallelism=f"independent circuits x{world}" if world > 1 else "single"),
        "e2e": {"value": e2e_updates_all / (e2e_ms_max / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms_max / args.steps,
                "path": "qx_load_circuit (host qx_instr records) -> qx_group_ops (new plan) -> "
                        "qx_propagate -> qx_result_raw into pinned host memory"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "alg_bytes_per_launch": d["alg_bytes"] / max(1, d["launches"]),
                     "avg_launch_ms": d["ms"] / max(1, d["launches"]),
                     "fp64": fp64_view(dom, d, s0)},
        "kernel_share": share,
        # per-step device time of each kernel class (CUDA events around its
        # launches); the rest of ms_per_step is time between classes
        "kernel_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in kc.items()
                               if v["launches"]},
        "per_step": {"term_updates": s0["term_updates"], "children": s0["children"],
                     "alg_bytes": s0["alg_bytes"], "kernel_launches": s0["kernel_launches"],
                     "host_syncs": s0["host_syncs"], "K": s0["K"], "Kp": s0["Kp"],
                     "final_terms": s0["final_terms"], "merge_passes": s0["merge_passes"],
                     "alg_gbs": s0["alg_bytes"] / (statistics.median(step_ms) / 1e3) / 1e9},
        "clocks": clocks,
        "wall_s": t_wall,
    }
    if world == 1 and args.serve_requests > 0:
        line["serving"] = serving_bench(qx, W, args.serve_requests, args.serve_rate)
    if world == 1 and args.adjoint_steps > 0:
        line["adjoint"] = adjoint_bench(qx, W, args.adjoint_steps)
    if world == 1 and args.fp32_steps > 0:
        line["fp32"] = fp32_bench(qx, plan, flush.zero_, args.fp32_steps, step_ms)
    if world == 1 and args.large_steps > 0:
        line["large"] = large_bench(qx, W, flush.zero_, args.large_steps, peak)
    if world == 1 and args.grouping_steps > 0:
        line["grouping"] = grouping_bench(qx, W, flush.zero_, args.grouping_steps)
    if world == 1 and args.xyz_repeats:
        line["xyz_chain"] = xyz_chain_bench(qx, W, [int(r) for r in args.xyz_repeats.split(",")],
                                            flush.zero_, oracle_sample=not args.no_cpu_baseline)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(plan_updates_per_gen(qx, plan, n), budget_s=20.0)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def serving_bench(qx, W, count, rate_hz, slots=8, baseline_count=300):
    """Serving stream (n in [10, 60], 200-5000 Clifford gates, 0-14 T/RZ,
    Poisson arrivals at rate_hz): circuits/s and p50/p99 latency of the
    request loop (FP32 weights, admission by HBM budget), next to the same
    circuits propagated one at a time in FP64 on the same GPU."""
    import threading
    import torch

    reqs = W.serving_stream(7, count=count, rate_hz=rate_hz)
    # the client's marshalling is done before the clock starts
    arrays = [qx.instr_array(instrs) for _, _, instrs in reqs]
    srv = qx.Server(slots=slots, hbm_budget=64 << 30, precision=32)
    # warm-up: a few requests through every slot
    for _, n, instrs in reqs[:2 * slots]:
        res, _ = srv.wait(srv.submit(n, instrs))
        res.free()
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for k, (at, n, _) in enumerate(reqs):
            delay = at - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets[k] = srv.submit(n, arrays[k])

    th = threading.Thread(target=submitter)
    th.start()
    lat = []
    for k in range(len(reqs)):
        while tickets[k] is None:
            time.sleep(0.0005)
        res, ms = srv.wait(tickets[k])
        lat.append(ms)
        res.free()
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    # one at a time, FP64, no overlap: the first baseline_count circuits
    torch.cuda.synchronize()
    b0 = time.perf_counter()
    for _, n, instrs in reqs[:baseline_count]:
        plan = qx.group_ops(qx.load_circuit(n, instrs))
        r = qx.propagate(plan)
        r.free()
    torch.cuda.synchronize()
    base = baseline_count / (time.perf_counter() - b0)
    lat.sort()
    return {"requests": count, "rate_hz": rate_hz, "slots": slots, "precision": 32,
            "hbm_budget_bytes": 64 << 30,
            "served_circuits_per_s": count / wall, "wall_s": wall,
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "retried_exclusive": st["retried_exclusive"], "failed": st["failed"],
            "one_at_a_time_fp64_circuits_per_s": base,
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


def fp32_bench(qx, plan, flush, steps, fp64_step_ms, warmup=3):
    """The main workload with FP32 weights and compensated arithmetic: time
    per step (CUDA events, L2 flushed) and the largest relative error against
    the FP64 result over three heavy generators (|w| > 1e-6)."""
    import torch

    times = []
    for k in range(warmup + steps):
        flush()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        r = qx.propagate(plan, precision=32)
        e1.record(s)
        torch.cuda.synchronize()
        if k >= warmup:
            times.append(e0.elapsed_time(e1))
        if k < warmup + steps - 1:
            r.free()
    st = r.stats()
    flush()
    kt = qx.propagate(plan, precision=32, kernel_timing=True).stats()["kernels"]
    ref = qx.propagate(plan)
    worst = 0.0
    for g in (16, 33, 49):
        a, b = r.export_dict(g), ref.export_dict(g)
        assert a.keys() == b.keys()
        for key, w in b.items():
            if abs(w) > 1e-6:
                worst = max(worst, abs(a[key] - w) / abs(w))
    ms = statistics.median(times)
    return {"precision": 32, "ms_per_step": ms, "term_updates_per_s": st["term_updates"] / (ms / 1e3),
            "speedup_vs_fp64": statistics.median(fp64_step_ms) / ms,
            "max_rel_error_vs_fp64": worst, "error_sample": "generators 16, 33, 49, |w| > 1e-6",
            "kernel_ms": {k: round(d["ms"], 4) for k, d in kt.items() if d["launches"]},
            "l2": "flushed between timed steps"}


def large_bench(qx, W, flush, steps, peak, warmup=3):
    """The HBM-scale configuration: fan_in_deep_n100 (n = 100, 20 RZ on 20
    fan-out qubits spread over 100,000 gates, 80 x 2^20 + 40 = 83,886,120
    final terms, 3.4 GB of FP64 terms).  Device time per propagation (CUDA
    events) and the dominant kernel class's achieved bandwidth (algorithmic
    bytes over its CUDA-event time, QX_FLAG_KERNEL_TIMING)."""
    import torch

    n, instrs = W.fan_in_deep(1)
    circ = qx.load_circuit(n, instrs)
    plan = qx.group_ops(circ)
    dag_ms = []
    dplan = qx.group_ops(circ, dag=True)
    for k in range(warmup + steps):  # the same circuit with qubit-wise grouping
        flush()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        r = qx.propagate(dplan)
        e1.record(s)
        torch.cuda.synchronize()
        if k >= warmup:
            dag_ms.append(e0.elapsed_time(e1))
        dag_terms = r.nterms
        r.free()
    del dplan
    times, st = [], None
    for k in range(warmup + steps):
        flush()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        r = qx.propagate(plan, kernel_timing=True)
        e1.record(s)
        torch.cuda.synchronize()
        if k >= warmup:
            times.append(e0.elapsed_time(e1))
            st = r.stats()
        nterms = r.nterms
        r.free()
    ms = statistics.median(times)
    kern = st["kernels"]
    dom = max(kern, key=lambda k: kern[k]["ms"])
    d = kern[dom]
    achieved = d["alg_bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] > 0 else 0.0
    return {"workload": "fan_in_deep_n100", "final_terms": nterms,
            "term_bytes": nterms * 44, "steps": steps, "warmup": warmup,
            "propagate_ms": ms, "term_updates_per_s": st["term_updates"] / (ms / 1e3),
            "children_per_s": st["children"] / (ms / 1e3),
            "dominant_kernel": dom, "dominant_share": d["ms"] / sum(v["ms"] for v in kern.values()),
            "dominant_achieved_gbs": achieved, "dominant_frac_of_peak": achieved / peak,
            "kernel_ms": {k: round(v["ms"], 3) for k, v in kern.items() if v["ms"] > 0},
            "qubit_wise_grouping": {"propagate_ms": statistics.median(dag_ms),
                                    "final_terms": dag_terms},
            "l2": "flushed between timed steps"}


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


def plan_updates_per_gen(qx, plan, n):
    """Term updates of one heavy generator (Z_16) in the library's own accounting."""
    r = qx.propagate(plan, gens=(16, 17))
    u = r.stats()["term_updates"]
    r.free()
    return u


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


def cpu_baseline(lib_updates_per_gen, budget_s):
    from paper_2505_03307_gb300 import workloads as W
    n, instrs = W.fan_in_heavy(1)
    st = OracleStepper(n, instrs, 16)
    done, secs = 0, 0.0
    while secs < budget_s:
        u, s = st.step(2_000_000)
        done += u
        secs += s
    return {"value": done / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"generator Z_16 (a 65,536-term generator) of the same circuit, gate by gate "
                      f"through whole operators for {secs:.1f} s ({done} term updates); "
                      f"single thread"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2505_03307_gb300 import workloads as W

    O.build()
    n, instrs = W.fan_in_heavy(1)
    st = OracleStepper(n, instrs, 16)
    budget = 3_000_000
    for _ in range(args.warmup):
        st.step(budget)
    times, done = [], 0
    for _ in range(args.steps):
        u, s = st.step(budget)
        done += u
        times.append(s)
    value = done / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded circuits; no dataset)", "config": dict(CONFIG),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "each step: about 3M term updates of generator Z_16 "
                                   "(65,536 terms at the heavy end), gate by gate through whole "
                                   "operators of the same circuit; single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream (0: skip; the full stream has 10000)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate (Hz)")
    ap.add_argument("--adjoint-steps", type=int, default=5,
                    help="timed steps of the gradient leg (0: skip)")
    ap.add_argument("--fp32-steps", type=int, default=5,
                    help="timed steps of the FP32 leg (0: skip)")
    ap.add_argument("--large-steps", type=int, default=3,
                    help="timed steps of the 84M-term fan_in_deep_n100 leg (0: skip)")
    ap.add_argument("--grouping-steps", type=int, default=5,
                    help="timed steps per case of the grouping comparison (0: skip)")
    ap.add_argument("--xyz-repeats", default="100,1000,10000,100000",
                    help="#Repeats of the XYZ + chain sweep, comma-separated ('' skips it)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
