#!/usr/bin/env python
"""Benchmark: the ADI-shaped plain-method set on GB300.

Workload (one step): one x-sweep and one y-sweep of a 2048 x 2048 grid for each of
r in {0.5, 2, 10}; every sweep is 2048 independent systems of n = 2048, solved by
NPDM, SPDM and SIP (ILU(0), Algorithm 1) on the pentadiagonal rows of the
second-order scheme and by NTDM and STDM on the tridiagonal analogue.  That is 30
batched solves and 125.8 M unknowns per step.  The x-sweep reads contiguous systems,
the y-sweep reads them at row stride (interleaved).

Metric: band unknowns solved per second (whole job), plus the roofline of the
dominant kernel and the CPU oracle as a reported baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import ctypes as ct
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "band unknowns solved/s & % HBM roofline; FP32+refine vs FP64 at rel err 1e-10"
UNIT = "unknowns/s"
GRID = 2048
SIP_TOL = 1e-10
SIP_MAX_IT = 200
# Algorithmic bytes and flops per unknown (inputs read once, output written once).
ALG_BYTES = {"npdm": 56, "spdm": 56, "ntdm": 40, "stdm": 40, "sip": 56}
ALG_FLOPS = {"npdm": 19, "spdm": 19, "ntdm": 9, "stdm": 9, "sip": 19 + 31}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# --------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world):
    """Maximum of a float over all ranks (the slowest rank's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# -------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

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
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workload
def host_workload(grid):
    """Host arrays of the 12 (r, sweep, bandwidth) batches of the step."""
    W = []
    for r in synth.ADI_R:
        for sweep in ("x", "y"):
            for k in (2, 1):
                B = synth.cfg1(r=r, k=k, sweep=sweep, grid=grid)
                W.append(dict(r=r, sweep=sweep, k=k, B=B))
    return W


def methods_for(k):
    return ("npdm", "spdm", "sip") if k == 2 else ("ntdm", "stdm")


def units_per_step(W):
    return sum(len(methods_for(w["k"])) * w["B"]["n"] * w["B"]["nsys"] for w in W)


class DeviceSet:
    """Device tensors, outputs and workspaces of the whole step (allocated once)."""

    def __init__(self, W, dev):
        import torch
        import paper_1804_09666_gb300 as band
        self.band = band
        self.items = []
        for w in W:
            B = w["B"]
            n, ns, ss, es = B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]
            keys = "abcdef" if w["k"] == 2 else "bcdf"
            host = {q: torch.from_numpy(B[q]).pin_memory() for q in keys}
            flat = {q: torch.empty(B[q].shape, dtype=torch.float64, device=dev) for q in keys}
            for q in keys:
                flat[q].copy_(host[q])
            view = {q: flat[q].as_strided((n, ns), (es, ss)) for q in keys}
            outs = {}
            for m in methods_for(w["k"]):
                xf = torch.empty(B["f"].shape, dtype=torch.float64, device=dev)
                outs[m] = dict(flat=xf, view=xf.as_strided((n, ns), (es, ss)),
                               host=torch.empty(B["f"].shape, dtype=torch.float64).pin_memory())
            self.items.append(dict(w=w, host=host, flat=flat, view=view, outs=outs, n=n, nsys=ns))
        self.h2d_bytes = sum(t.numel() * 8 for it in self.items for t in it["host"].values())
        self.d2h_bytes = sum(o["flat"].numel() * 8 for it in self.items for o in it["outs"].values())

    def step(self, events=None):
        band = self.band
        for it in self.items:
            v = it["view"]
            for m in methods_for(it["w"]["k"]):
                x = it["outs"][m]["view"]
                if events is not None:
                    e0, e1 = events.new(m)
                    e0.record()
                if m == "sip":
                    band.sip(v["a"], v["b"], v["c"], v["d"], v["e"], v["f"], tol=SIP_TOL,
                             max_it=SIP_MAX_IT, width=0, x=x)
                elif it["w"]["k"] == 2:
                    band.solve(v["a"], v["b"], v["c"], v["d"], v["e"], v["f"], method=m, x=x)
                else:
                    band.solve(None, v["b"], v["c"], v["d"], None, v["f"], method=m, x=x)
                if events is not None:
                    e1.record()

    def upload(self):
        for it in self.items:
            for q, h in it["host"].items():
                it["flat"][q].copy_(h, non_blocking=True)

    def download(self):
        for it in self.items:
            for o in it["outs"].values():
                o["host"].copy_(o["flat"], non_blocking=True)

    def statuses_ok(self):
        """Re-run the step once with status outputs and check that every system is OK."""
        import torch
        band = self.band
        bad = 0
        for it in self.items:
            v = it["view"]
            for m in methods_for(it["w"]["k"]):
                if m == "sip":
                    _, _, _, st = band.sip(v["a"], v["b"], v["c"], v["d"], v["e"], v["f"],
                                           tol=SIP_TOL, max_it=SIP_MAX_IT, width=0)
                elif it["w"]["k"] == 2:
                    _, st = band.solve(v["a"], v["b"], v["c"], v["d"], v["e"], v["f"], method=m)
                else:
                    _, st = band.solve(None, v["b"], v["c"], v["d"], None, v["f"], method=m)
                bad += int((st != 0).sum())
        torch.cuda.synchronize()
        return bad


class EventLog:
    def __init__(self):
        import torch
        self.torch = torch
        self.pairs = {}

    def new(self, name):
        e0 = self.torch.cuda.Event(enable_timing=True)
        e1 = self.torch.cuda.Event(enable_timing=True)
        self.pairs.setdefault(name, []).append((e0, e1))
        return e0, e1

    def summary(self):
        return {k: [a.elapsed_time(b) for a, b in v] for k, v in self.pairs.items()}


# ----------------------------------------------------------- CPU baselines
def oracle_sample(W, per_batch, nthreads):
    """Time the CPU oracle on the first `per_batch` systems of every batch and method."""
    import oracle
    units = 0
    t0 = time.perf_counter()
    for w in W:
        B = w["B"]
        ns = min(per_batch, B["nsys"])
        diags = [B[q] for q in "abcde"]
        for m in methods_for(w["k"]):
            kind = {"npdm": "direct", "ntdm": "direct", "spdm": "symbolic", "stdm": "symbolic",
                    "sip": "sip"}[m]
            x, st, _, _ = oracle.batch(kind, w["k"], diags, B["f"], ns, B["n"], B["sys_stride"],
                                       B["elem_stride"], nthreads=nthreads, tol=SIP_TOL,
                                       max_it=SIP_MAX_IT, hb_width=0)
            units += ns * B["n"]
    dt = time.perf_counter() - t0
    return units, dt


def cpu_baseline(W, budget_s=15.0):
    nthreads = os.cpu_count() or 1
    u, dt = oracle_sample(W, 4, nthreads)          # calibration
    per = max(4, min(W[0]["B"]["nsys"], int(4 * budget_s / max(dt, 1e-3))))
    u, dt = oracle_sample(W, per, nthreads)
    return {"value": u / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": "first %d systems of each of the 30 batched solves (every r, sweep and "
                      "method) of the same workload; %.1f s" % (per, dt)}


def run_reference(args, world, rank):
    if rank != 0:
        return
    W = host_workload(args.grid)
    nthreads = os.cpu_count() or 1
    per = 8
    for _ in range(args.warmup):
        oracle_sample(W, per, nthreads)
    units, total = 0, 0.0
    for _ in range(args.steps):
        u, dt = oracle_sample(W, per, nthreads)
        units += u
        total += dt
    value = units / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.grid, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": "first %d systems of each of the 30 batched solves per step"
                                       % per},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(grid, ngpus):
    return {"workload": "ADI %dx%d grid, x- and y-sweep, r in {0.5, 2, 10}; PD rows solved by "
                        "NPDM, SPDM, SIP (ILU(0), Algorithm 1); TD rows by NTDM, STDM" % (grid, grid),
            "systems_per_sweep": grid, "n": grid, "solves_per_step": 30,
            "layouts": "x-sweep contiguous systems, y-sweep interleaved (row stride)",
            "l2": "inputs larger than L2 (one PD sweep reads 192 MiB)",
            "parallelism": "replicas: every rank solves its own full set" if ngpus > 1 else "1 GPU"}


# ---------------------------------------------------------------------- main
def main():
    args = parse()
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        if args.impl == "reference":
            dist.init_process_group("gloo")
        else:
            import torch
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.impl == "reference":
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import _lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = band.load()
    W = host_workload(args.grid)
    D = DeviceSet(W, dev)
    units = units_per_step(W)

    # FP64 FMA rate of this GPU (the ALU roofline of the FP64 recurrences)
    scratch = torch.empty(8 * 256 * 8 * 256, dtype=torch.uint8, device=dev)
    fma_rate = lib.band_fp64_fma_rate(ct.c_void_p(scratch.data_ptr()), scratch.numel(),
                                      ct.c_void_p(torch.cuda.current_stream().cuda_stream))

    for _ in range(max(args.warmup, 3)):
        D.step()
    torch.cuda.synchronize()
    bad = D.statuses_ok()

    # timed region: inputs resident in HBM
    clocks = ClockSampler(torch.cuda.current_device())
    events = EventLog()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        D.step(events)
    t1.record()
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    ms = max_over_ranks(ms, world)
    value = units * args.steps * world / (ms * 1e-3)

    # end to end: pinned host inputs -> device -> solves -> host, every step
    for _ in range(2):
        D.upload(); D.step(); D.download()
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        D.upload()
        D.step()
        D.download()
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), world)
    e2e = {"value": units * args.steps * world / (ms_e2e * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": D.h2d_bytes, "d2h_bytes_per_step": D.d2h_bytes}

    # per-method launch times (CUDA events on the launching stream, inside the timed region)
    per = events.summary()
    per_call_units = W[0]["B"]["n"] * W[0]["B"]["nsys"]
    methods = {}
    for m, times in per.items():
        avg = float(np.mean(times))
        methods[m] = {"ms_per_launch": avg, "launches": len(times),
                      "share": float(np.sum(times)) / sum(float(np.sum(t)) for t in per.values()),
                      "unknowns_per_s": per_call_units / (avg * 1e-3),
                      "alg_GBps": ALG_BYTES[m] * per_call_units / (avg * 1e-3) / 1e9,
                      "alg_TFLOPs": ALG_FLOPS[m] * per_call_units / (avg * 1e-3) / 1e12}
    dom = max(methods, key=lambda m: methods[m]["share"])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak_tf = 2.0 * fma_rate / 1e12 if fma_rate > 0 else 1.25
    mm = methods[dom]
    frac_hbm = mm["alg_GBps"] / hbm_peak
    frac_alu = mm["alg_TFLOPs"] / fp64_peak_tf
    if frac_alu >= frac_hbm:
        roof = {"bound": "alu", "achieved": mm["alg_TFLOPs"], "peak": fp64_peak_tf,
                "unit": "TFLOP/s", "frac": frac_alu, "traffic": None,
                "kernel": dom, "peak_source": "measured FP64 FMA rate (band_fp64_fma_rate) x 2",
                "hbm_frac_of_measured": frac_hbm}
    else:
        roof = {"bound": "hbm", "achieved": mm["alg_GBps"], "peak": hbm_peak, "unit": "GB/s",
                "frac": frac_hbm, "traffic": None, "kernel": dom,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs", "alu_frac": frac_alu}

    launches_per_step = sum(
        {"npdm": 1, "ntdm": 1, "spdm": 2, "stdm": 2, "sip": 2}[m]
        for it in D.items for m in methods_for(it["w"]["k"]))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.grid, world),
            "clocks": ck, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "methods": methods, "bad_systems": bad,
            "fp64_fma_per_s": fma_rate}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
