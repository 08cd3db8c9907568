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
# flops per Table 7: NPDM 19N-29, NTDM 9N+2, SIP 31N-36 per iteration (one iteration on
# this set) plus ILU(0)'s 10 per row; SPDM/STDM do NPDM/NTDM's work when no pivot is 0.
ALG_FLOPS = {"npdm": 19, "spdm": 19, "ntdm": 9, "stdm": 9, "sip": 10 + 31}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ragged, precision, adjoint and SIP workloads (N = 1 only)")
    ap.add_argument("--ragged-nsys", type=int, default=65536,
                    help="systems of the ragged workload (a smaller case for profiling)")
    ap.add_argument("--workload", choices=sorted(EXTRA_WORKLOADS),
                    help="run only this one of the other workloads on GPU 0 and print its "
                         "result as a JSON line (for profiling it alone)")
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
    """Device inputs, the batched plan of the 30 solves and its CUDA graph."""

    def __init__(self, W, dev, use_graph=True, host=None):
        """host: another DeviceSet whose pinned host inputs this one shares."""
        import torch
        import paper_1804_09666_gb300 as band
        self.torch = torch
        self.items = []
        specs, self.spec_methods = [], []
        for wi, w in enumerate(W):
            B = w["B"]
            n, ns, ss, es = B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]
            keys = "abcdef" if w["k"] == 2 else "bcdf"
            host_in = {q: torch.from_numpy(B[q]).pin_memory() for q in keys} if host is None \
                else host.items[wi]["host"]
            flat = {q: torch.empty(B[q].shape, dtype=torch.float64, device=dev) for q in keys}
            for q in keys:
                flat[q].copy_(host_in[q])
            view = {q: flat[q].as_strided((n, ns), (es, ss)) for q in keys}
            self.items.append(dict(w=w, host=host_in, flat=flat, view=view, n=n, nsys=ns))
        # heaviest problems first: SIP, then the PD sweeps, then the TD sweeps
        self.spec_items = []
        for kind in ("sip", "npdm", "spdm", "ntdm", "stdm"):
            for it in self.items:
                if kind not in methods_for(it["w"]["k"]):
                    continue
                v = it["view"]
                if kind == "sip":
                    sp = dict(op="sip", tol=SIP_TOL, max_it=SIP_MAX_IT, **v)
                elif it["w"]["k"] == 2:
                    sp = dict(method=kind, **v)
                else:
                    sp = dict(method=kind, a=None, e=None, **v)
                specs.append(sp)
                self.spec_methods.append((kind, it["n"] * it["nsys"]))
                self.spec_items.append(it)
        self.plan = band.BatchPlan(specs)
        # outputs are compact strided views; copy their storage as flat buffers
        self.out_flat = [r["x"].as_strided((r["x"].numel(),), (1,)) for r in self.plan.results]
        self.out_host = [torch.empty(t.numel(), dtype=torch.float64).pin_memory()
                         for t in self.out_flat]
        self.h2d_bytes = sum(t.numel() * 8 for it in self.items for t in it["host"].values())
        self.d2h_bytes = sum(r["x"].numel() * 8 for r in self.plan.results)
        self.graph = None
        if use_graph:
            self.plan.run()
            torch.cuda.synchronize()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    self.plan.run()
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            self.graph = g

    def alg(self, table):
        return sum(table[m] * units for m, units in self.spec_methods)

    def step(self, events=None):
        if events is not None:
            e0, e1 = events.new("batch")
            e0.record()
        if self.graph is not None:
            self.graph.replay()
        else:
            self.plan.run()
        if events is not None:
            e1.record()

    def upload(self):
        for it in self.items:
            for q, h in it["host"].items():
                it["flat"][q].copy_(h, non_blocking=True)

    def download(self):
        for t, h in zip(self.out_flat, self.out_host):
            h.copy_(t, non_blocking=True)

    def statuses(self):
        """Systems per status other than OK after one step, by method."""
        from paper_1804_09666_gb300 import _lib
        self.step()
        self.torch.cuda.synchronize()
        out = {}
        for (kind, _), r in zip(self.spec_methods, self.plan.results):
            codes, counts = self.torch.unique(r["status"].cpu(), return_counts=True)
            for c, k in zip(codes.tolist(), counts.tolist()):
                if c != 0:
                    key = "%s:%s" % (kind, _lib.STATUS_NAMES.get(c, str(c)))
                    out[key] = out.get(key, 0) + k
        return out

    def kernels_per_step(self):
        """Kernels band_solve_batch launches for this plan: the batched sweep, the
        symbolic fix-up when a symbolic solve is present, and for SIP solves the
        residual, decision and tail passes."""
        kinds = {k for k, _ in self.spec_methods}
        return 1 + int(bool(kinds & {"spdm", "stdm"})) + 3 * int("sip" in kinds)


def accuracy_report(D, sample_every=128):
    """Forward errors of one step's results: every system against its manufactured
    solution, and every `sample_every`-th system of every solve against the CPU oracle's
    result for the same method (relative max-norm per system, maxed).  SIP systems that
    stop NOT_CONVERGED at their rounding floor are reported on their own."""
    import oracle
    D.step()
    D.torch.cuda.synchronize()
    kind_of = {"npdm": "direct", "ntdm": "direct", "spdm": "symbolic", "stdm": "symbolic",
               "sip": "sip"}
    worst_oracle, worst_true, checked = 0.0, 0.0, 0
    per_method = {}
    sip_floor = {"systems": 0, "max_err_vs_manufactured": 0.0}
    for (kind, _), it, r in zip(D.spec_methods, D.spec_items, D.plan.results):
        B = it["w"]["B"]
        n, ns, ss, es = B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]
        x = r["x"].cpu().numpy()                       # (n, nsys) view of the output
        st = r["status"].cpu().numpy()
        xt = B["x_true"]
        idx = np.arange(ns)[None, :] * ss + np.arange(n)[:, None] * es
        xtrue = xt[idx]
        err_true = np.abs(x - xtrue).max(0) / np.abs(xtrue).max(0)
        ok = st == 0
        worst_true = max(worst_true, float(err_true[ok].max()) if ok.any() else 0.0)
        if kind == "sip" and (~ok).any():
            sip_floor["systems"] += int((~ok).sum())
            sip_floor["max_err_vs_manufactured"] = max(sip_floor["max_err_vs_manufactured"],
                                                       float(err_true[~ok].max()))
        nsamp = (ns + sample_every - 1) // sample_every
        diags = [B[q] if it["w"]["k"] == 2 or q in "bcd" else None for q in "abcde"]
        xo, so, _, _ = oracle.batch(kind_of[kind], it["w"]["k"], diags, B["f"], nsamp, n,
                                    ss * sample_every, es, tol=SIP_TOL, max_it=SIP_MAX_IT,
                                    hb_width=0)
        cols = np.arange(0, ns, sample_every)
        io = np.arange(nsamp)[None, :] * (ss * sample_every) + np.arange(n)[:, None] * es
        xo = xo[io]
        good = (so == 0) & ok[cols]
        if good.any():
            e = np.abs(x[:, cols] - xo).max(0) / np.abs(xo).max(0)
            worst_oracle = max(worst_oracle, float(e[good].max()))
            per_method[kind] = max(per_method.get(kind, 0.0), float(e[good].max()))
        checked += int(good.sum())
    return {"max_rel_err_vs_oracle": worst_oracle, "oracle_systems_checked": checked,
            "max_rel_err_vs_oracle_by_method": per_method,
            "max_rel_err_vs_manufactured": worst_true,
            "sip_not_converged_at_rounding_floor": sip_floor}


def e2e_serial(D, steps, world):
    """H2D, solves and D2H of each step one after the other on one stream (ms)."""
    import torch
    for _ in range(2):
        D.upload(); D.step(); D.download()
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        D.upload()
        D.step()
        D.download()
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(e0.elapsed_time(e1), world)


def e2e_pipelined(sets, steps, world):
    """Steps k and k+1 use different device sets; each step's H2D, solves and D2H run on
    their own streams, ordered by events (ms for `steps` steps, all copies included)."""
    import torch
    main = torch.cuda.current_stream()
    sh, sc, sd = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = {name: [torch.cuda.Event() for _ in sets] for name in ("h2d", "cmp", "d2h")}

    def run(nsteps):
        for k in range(nsteps):
            j = k % len(sets)
            S = sets[j]
            with torch.cuda.stream(sh):
                sh.wait_event(ev["cmp"][j])        # the set's previous solves read its inputs
                S.upload()
                ev["h2d"][j].record(sh)
            with torch.cuda.stream(sc):
                sc.wait_event(ev["h2d"][j])
                sc.wait_event(ev["d2h"][j])        # its previous results have been read
                S.step()
                ev["cmp"][j].record(sc)
            with torch.cuda.stream(sd):
                sd.wait_event(ev["cmp"][j])
                S.download()
                ev["d2h"][j].record(sd)
        for s in (sh, sc, sd):
            main.wait_stream(s)

    for s in (sh, sc, sd):
        s.wait_stream(main)
    run(2)
    torch.cuda.synchronize()
    barrier(world)
    for s in (sh, sc, sd):
        s.wait_stream(main)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for s in (sh, sc, sd):
        s.wait_stream(main)
    run(steps)
    e1.record(main)
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(e0.elapsed_time(e1), world)


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
def oracle_sample(W, per_batch, nthreads, by_method=None):
    """Time the CPU oracle on the first `per_batch` systems of every batch and method;
    by_method (a dict, optional) collects [units, seconds] per method."""
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
            tm = time.perf_counter()
            x, st, _, _ = oracle.batch(kind, w["k"], diags, B["f"], ns, B["n"], B["sys_stride"],
                                       B["elem_stride"], nthreads=nthreads, tol=SIP_TOL,
                                       max_it=SIP_MAX_IT, hb_width=0)
            units += ns * B["n"]
            if by_method is not None:
                acc = by_method.setdefault(m, [0, 0.0])
                acc[0] += ns * B["n"]
                acc[1] += time.perf_counter() - tm
    dt = time.perf_counter() - t0
    return units, dt


def cpu_baseline(W, budget_s=15.0):
    """The oracle on the host cores: systems per batch grown until one sample takes
    about budget_s seconds (or covers every system)."""
    nthreads = os.cpu_count() or 1
    nsys = W[0]["B"]["nsys"]
    per = 4
    u, dt = oracle_sample(W, per, nthreads)
    while dt < 0.5 * budget_s and per < nsys:
        per = max(per + 1, min(nsys, int(per * budget_s / max(dt, 1e-3))))
        u, dt = oracle_sample(W, per, nthreads)
    reps = 1
    if dt < 0.5 * budget_s:                      # the whole workload is quick: repeat it
        reps = max(1, int(budget_s / max(dt, 1e-3)))
        u, dt = 0, 0.0
        for _ in range(reps):
            ui, di = oracle_sample(W, per, nthreads)
            u, dt = u + ui, dt + di
    bym = {}
    u1, dt1 = oracle_sample(W, 64, 1, bym)
    return {"value": u / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": "first %d systems of each of the 30 batched solves (every r, sweep and "
                      "method) of the same workload, %d pass(es); %.1f s" % (per, reps, dt),
            "one_core": {"value": u1 / dt1, "unit": UNIT, "cores": 1,
                         "sample": "first 64 systems of each of the 30 solves; %.1f s" % dt1,
                         "per_method": {m: {"value": v[0] / v[1], "unit": UNIT}
                                        for m, v in bym.items() if v[1] > 0}}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    W = host_workload(args.grid)
    nthreads = os.cpu_count() or 1
    per = max(8, nthreads)          # at least one system per host core in every solve
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
                             "sample": "first %d systems of each of the 30 batched solves per step "
                                       "(at least one per host core)" % per},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Sources that k_batch is compiled from: an ncu traffic figure applies only while their
# code is unchanged since the capture that measured it (comments and layout are not code).
K_BATCH_SOURCES = ("include/band.h", "paper_1804_09666_gb300/csrc/batch_kernel.cuh",
                   "paper_1804_09666_gb300/csrc/batch.cu",
                   "paper_1804_09666_gb300/csrc/api_util.h", "paper_1804_09666_gb300/csrc/kernels.h",
                   "paper_1804_09666_gb300/csrc/common.cuh", "paper_1804_09666_gb300/csrc/sweeps.cuh",
                   "paper_1804_09666_gb300/csrc/sip_impl.cuh",
                   "paper_1804_09666_gb300/csrc/partition.cuh")
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "k_batch_adi2048_dram.md")


def code_text(src):
    """C / C++ / CUDA source without its comments, blank lines and runs of white space:
    what the compiler sees up to layout.  Quotes inside comments are ignored; string and
    character literals are kept whole (with their escapes)."""
    out, i, n, state, quote = [], 0, len(src), "code", ""
    while i < n:
        ch = src[i]
        if state == "code":
            if src.startswith("//", i):
                state, i = "line", i + 2
            elif src.startswith("/*", i):
                state, i = "block", i + 2
                out.append(" ")
            else:
                if ch in "\"'":
                    state, quote = "literal", ch
                out.append(ch)
                i += 1
        elif state == "line":
            if ch == "\n":
                state = "code"
                out.append(ch)
            i += 1
        elif state == "block":
            if src.startswith("*/", i):
                state, i = "code", i + 2
            else:
                if ch == "\n":
                    out.append(ch)
                i += 1
        else:                                   # inside a string or character literal
            out.append(ch)
            if ch == "\\" and i + 1 < n:
                out.append(src[i + 1])
                i += 2
                continue
            if ch == quote or ch == "\n":
                state = "code"
            i += 1
    lines = (" ".join(line.split()) for line in "".join(out).split("\n"))
    return "\n".join(line for line in lines if line)


def sources_sha256(paths=K_BATCH_SOURCES, read=None):
    """SHA-256 over the code (code_text) of the given files, in order, each followed by
    a NUL byte.  read(rel) -> source text; the working tree's files by default."""
    import hashlib
    if read is None:
        def read(rel):
            with open(os.path.join(ROOT, rel), encoding="utf-8") as fh:
                return fh.read()
    h = hashlib.sha256()
    for rel in paths:
        h.update(code_text(read(rel)).encode("utf-8"))
        h.update(b"\0")
    return h.hexdigest()


def recorded_traffic(grid):
    """DRAM bytes per k_batch launch from the committed ncu summary, or None when the
    workload differs or the kernel's sources changed since the capture."""
    import re
    if grid != GRID or not os.path.exists(TRAFFIC_RECORD):
        return None
    text = open(TRAFFIC_RECORD).read()
    mb = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    mh = re.search(r"code_sha256:\s*([0-9a-f]{64})", text)
    if not mb or not mh or mh.group(1) != sources_sha256():
        return None
    return int(mb.group(1))


def workload_config(grid, ngpus):
    return {"workload": "ADI %dx%d grid, x- and y-sweep, r in {0.5, 2, 10}; PD rows solved by "
                        "NPDM, SPDM, SIP (ILU(0), Algorithm 1); TD rows by NTDM, STDM" % (grid, grid),
            "systems_per_sweep": grid, "n": grid, "solves_per_step": 30,
            "layouts": "x-sweep contiguous systems, y-sweep interleaved (row stride)",
            "l2": "inputs larger than L2 (one PD sweep reads %d MiB)" % (6 * grid * grid * 8 >> 20),
            "parallelism": "replicas: every rank solves its own full set" if ngpus > 1 else "1 GPU"}


# ------------------------------------------------------- the other workloads
def _time(fn, reps=5, warm=2):
    """Best of `reps` CUDA-event timings (ms) of fn() on the current stream."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def per_method_workload(D):
    """Each method's six solves of the step (3 r x 2 sweeps) alone, as one batched launch
    on the step's own device data: unknowns/s per method (SIP: Algorithm 1 with its
    residual pass, decision and tail)."""
    import paper_1804_09666_gb300 as band
    out = {"workload": "each method's 6 solves of the ADI step (2048 systems of n = 2048 "
                       "each) in one batched launch", "unit": UNIT}
    for kind in ("npdm", "spdm", "sip", "ntdm", "stdm"):
        specs = []
        for it in D.items:
            if kind not in methods_for(it["w"]["k"]):
                continue
            v = it["view"]
            if kind == "sip":
                specs.append(dict(op="sip", tol=SIP_TOL, max_it=SIP_MAX_IT, **v))
            elif it["w"]["k"] == 2:
                specs.append(dict(method=kind, **v))
            else:
                specs.append(dict(method=kind, a=None, e=None, **v))
        plan = band.BatchPlan(specs)
        ms = _time(plan.run, reps=5)
        units = sum(it["n"] * it["nsys"] for it in D.items if kind in methods_for(it["w"]["k"]))
        out[kind] = {"value": units / (ms * 1e-3), "ms": ms}
    return out


def ragged_workload(dev, nsys=65536):
    """65536 systems, n log-uniform in [16, 8192], half TD / half PD, packed ragged:
    size buckets with autotuned schedules in one graph-captured launch, against the
    whole packing on one thread per system.  The timed replays sit in the NVTX range
    "ragged_replay" (for a profiler's range filter)."""
    import torch
    import paper_1804_09666_gb300 as band
    B = synth.cfg2(nsys=nsys)
    d = {q: torch.from_numpy(B[q]).to(dev) for q in "abcdef"}
    units = int(B["offsets"][-1])
    plan = band.RaggedPlan(*(d[q] for q in "abcdef"), B["offsets"], B["hbw"], schedule="tune")
    plan.run()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.nvtx.range_push("ragged_replay")
    ms = _time(g.replay, reps=10)
    torch.cuda.nvtx.range_pop()
    x, st = plan.x, plan.status
    err = np.maximum.reduceat(np.abs(x.cpu().numpy() - B["x_true"]), B["offsets"][:-1])
    offs = torch.from_numpy(B["offsets"]).to(dev)
    hbw = torch.from_numpy(B["hbw"]).to(dev)
    ms_whole = _time(lambda: band.solve_ragged(*(d[q] for q in "abcdef"), offs, hbw,
                                               n_max=int(B["sizes"].max()), total_rows=units),
                     reps=5)
    two = band.RaggedPlan(*(d[q] for q in "abcdef"), B["offsets"], B["hbw"], schedule="two_sided")
    ms_two = _time(two.run, reps=5)
    parted = [{"n_max": int(bk[2]), "half_bw": int(bk[3]), "systems": int(bk[1]), "chunks": int(c)}
              for bk, v, c in zip(plan.buckets, plan.schedules, plan.chunks) if v == 3]
    return {"workload": "%d ragged systems, n log-uniform in [16, 8192], half TD / half PD, "
                        "dominant (%d unknowns)" % (nsys, units),
            "value": units / (ms * 1e-3), "unit": UNIT, "ms": ms,
            "buckets": len(plan.buckets),
            "two_sided_buckets": int(sum(1 for v in plan.schedules if v == 2)),
            "partitioned_buckets": parted,
            "status_not_ok": int((st != 0).sum()), "max_err_vs_manufactured": float(err.max()),
            "all_buckets_two_sided": {"value": units / (ms_two * 1e-3), "ms": ms_two},
            "whole_packing_thread_per_system": {"value": units / (ms_whole * 1e-3), "ms": ms_whole}}


def small_batch_workload(dev):
    """A batch too small to fill the GPU: 64 dominant PD systems of n = 65536 (one
    thread or two per system leave most SMs idle), two-sided against partitioned."""
    import torch
    import paper_1804_09666_gb300 as band
    B = synth.cfg0(nsys=64, n=65536, seed_salt=80)
    n, nsys = B["n"], B["nsys"]
    d = {q: torch.from_numpy(B[q]).to(dev).view(n, nsys) for q in "abcdef"}
    xt = torch.from_numpy(B["x_true"]).to(dev).view(n, nsys)
    units = n * nsys
    out = {"workload": "64 PD systems, n = 65536 (dominant, interleaved)"}
    for sched in ("two_sided", "partitioned"):
        x = torch.empty_like(d["f"])
        res = {}

        def run():
            res["x"], res["st"] = band.solve(*(d[q] for q in "abcdef"), method="npdm", x=x,
                                             schedule=sched)
        ms = _time(run)
        err = float(((res["x"] - xt).abs().amax(0) / xt.abs().amax(0)).max())
        out[sched] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms": ms,
                      "status_not_ok": int((res["st"] != 0).sum()), "max_rel_err": err}
    return out


def precision_workload(dev):
    """16384 PD systems of n = 4096 stored in FP32 (dominance ratio in {1.01, 1.1, 2} with
    5 % of the diagonal signs flipped): FP32 + refinement against plain FP64 NPDM on
    the same matrices (their FP64 values), both at the forward error they reach."""
    import torch
    import paper_1804_09666_gb300 as band
    nsys, n = 16384, 4096
    B = synth.cfg3()
    d32 = {q: torch.from_numpy(B[q]).to(dev).view(n, nsys) for q in "abcde"}
    d64 = {q: d32[q].double() for q in "abcde"}
    f = torch.from_numpy(B["f"]).to(dev).view(n, nsys)
    xt = torch.from_numpy(B["x_true"]).to(dev).view(n, nsys)
    units = n * nsys

    def rel(x):
        return float(((x - xt).abs().amax(0) / xt.abs().amax(0)).max())

    out = {}
    x64 = torch.empty_like(f)
    ms64 = _time(lambda: band.solve(*(d64[q] for q in "abcde"), f, method="npdm", x=x64))
    out["fp64_npdm"] = {"value": units / (ms64 * 1e-3), "ms": ms64, "max_rel_err": rel(x64)}
    import oracle
    sample = np.random.default_rng(5).choice(nsys, 8, replace=False)
    truth = {}
    for s_ in sample:
        S = {q: B[q].reshape(n, nsys)[:, s_].astype(np.float64) for q in "abcde"}
        truth[int(s_)] = oracle.gepp_band(2, *(S[q] for q in "abcde"),
                                          B["f"].reshape(n, nsys)[:, s_])[0]

    def vs_oracle(x):
        xg = x.cpu().numpy()
        return max(float(np.abs(xg[:, s_] - xo).max() / np.abs(xo).max())
                   for s_, xo in truth.items())

    # the FP32 solve alone on each schedule (the refinement's dominant part)
    f32 = f.float()
    x32 = torch.empty_like(f32)
    sched_ms = {}
    for sched, ch in (("two_sided", 0), ("partitioned", 8), ("partitioned", 16),
                      ("partitioned", 32)):
        sched_ms["%s%s" % (sched, "_%d" % ch if ch else "")] = _time(
            lambda: band.solve(*(d32[q] for q in "abcde"), f32, method="npdm", x=x32,
                               schedule=sched, chunks=ch))
    out["fp32_npdm_solve_ms"] = sched_ms
    best = min(sched_ms, key=sched_ms.get)
    bsched, bch = ("partitioned", int(best.split("_")[-1])) if best.startswith("partitioned") \
        else (best, 0)
    out["fp32_schedule_used"] = best
    for name, pairs in (("fp32_refine", False), ("fp32_refine_pairs", True)):
        res = {}

        def run_refine():
            res["x"], res["steps"], res["st"] = band.refine_solve(*(d32[q] for q in "abcde"), f,
                                                                  pairs=pairs, schedule=bsched,
                                                                  chunks=bch)
        msr = _time(run_refine)
        steps = res["steps"].cpu().numpy()
        out[name] = {"value": units / (msr * 1e-3), "ms": msr, "max_rel_err": rel(res["x"]),
                     "max_rel_err_vs_oracle_gepp": vs_oracle(res["x"]),
                     "steps_max": int(steps.max()), "steps_mean": float(steps.mean()),
                     "status_not_ok": int((res["st"] != 0).sum()),
                     "residual_and_update": "FP32 pairs" if pairs else "FP64"}
    out["fp64_npdm"]["max_rel_err_vs_oracle_gepp"] = vs_oracle(x64)
    out["workload"] = "16384 PD systems, n = 4096, FP32 storage (%d unknowns)" % units
    out["unit"] = UNIT
    out["refine_over_fp64"] = out["fp32_refine"]["value"] / out["fp64_npdm"]["value"]
    out["refine_pairs_over_fp64"] = out["fp32_refine_pairs"]["value"] / out["fp64_npdm"]["value"]
    return out


def sip_workload(dev):
    """SIP on 4096 dominant PD systems of n = 1024 (cfg0's recipe): Algorithm 1 with the
    exact ILU(0) substitutions, and with Hotelling-Bodewig inverses kept to 5
    diagonals (ILU(0), the two HB iterations and the correction-form updates)."""
    import torch
    import paper_1804_09666_gb300 as band
    nsys, n = 4096, 1024
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=7)
    d = {q: torch.from_numpy(B[q]).to(dev).view(n, nsys) for q in "abcdef"}
    xt = torch.from_numpy(B["x_true"]).to(dev).view(n, nsys)
    units = n * nsys
    out = {"workload": "4096 dominant PD systems, n = 1024, tol 1e-10", "unit": UNIT}
    for name, width in (("algorithm1_exact", 0), ("hb_w5", 5)):
        res = {}

        def run():
            res["x"], res["it"], res["rs"], res["st"] = band.sip(
                *(d[q] for q in "abcdef"), tol=1e-10, max_it=200, width=width)
        ms = _time(run)
        err = float(((res["x"] - xt).abs().amax(0) / xt.abs().amax(0)).max())
        out[name] = {"value": units / (ms * 1e-3), "ms": ms,
                     "iters_mean": float(res["it"].float().mean()),
                     "status_not_ok": int((res["st"] != 0).sum()), "max_rel_err": err}
    return out


def adjoint_workload(dev):
    """4096 PD systems of n = 1024: NPDM solve plus the adjoint (all six gradients)."""
    import torch
    import paper_1804_09666_gb300 as band
    nsys, n = 4096, 1024
    B = synth.cfg4()
    d = {q: torch.from_numpy(B[q]).to(dev).view(n, nsys) for q in "abcdefw"}
    units = n * nsys

    out = {"workload": "4096 PD systems, n = 1024: solve + adjoint", "unit": UNIT}
    for sched in ("auto", "partitioned"):
        def step():
            x, _ = band.solve(*(d[q] for q in "abcdef"), method="npdm", schedule=sched)
            band.adjoint(*(d[q] for q in "abcde"), x, d["w"], schedule=sched)
        ms = _time(step)
        if sched == "auto":
            out.update(value=units / (ms * 1e-3), ms=ms)
        else:       # these systems are dominant: the partitioned solves keep NPDM's accuracy
            out["partitioned"] = {"value": units / (ms * 1e-3), "ms": ms}
    return out


def cfg0_workload(dev):
    """The small plain-NPDM configuration (1024 dominant PD systems of n = 128, 7 MiB:
    fits in L2): latency of one band_solve, against the oracle on every system."""
    import torch
    import oracle
    import paper_1804_09666_gb300 as band
    B = synth.cfg0()
    n, ns = B["n"], B["nsys"]
    d = {q: torch.from_numpy(B[q].reshape(n, ns)).to(dev) for q in "abcdef"}
    x = torch.empty_like(d["f"])
    res = {}

    def run():
        res["x"], res["st"] = band.solve(*(d[q] for q in "abcdef"), method="npdm", x=x)
    ms = _time(run, reps=20, warm=3)
    xo, so, _, _ = oracle.batch("direct", 2, [B[q] for q in "abcde"], B["f"], ns, n, 1, ns)
    xg = res["x"].cpu().numpy().reshape(-1)
    err = (np.abs(xg - xo).reshape(n, ns).max(0) / np.abs(xo).reshape(n, ns).max(0)).max()
    return {"workload": "1024 PD systems, n = 128, NPDM (fits in L2: latency, not roofline)",
            "latency_ms": ms, "value": n * ns / (ms * 1e-3), "unit": UNIT,
            "status_not_ok": int((res["st"] != 0).sum()), "max_rel_err_vs_oracle": float(err)}


def symbolic_workload(dev):
    """SPDM on one ADI sweep (2048 PD systems of n = 2048, r = 2, y-sweep: interleaved)
    with an exact zero pivot planted in 0 %, 1 % and 10 % of the systems (row j of a
    planted system gets a_j = b_j = c_j = 0, so its pivot mu_j is 0 in any arithmetic;
    f = A x_true).  Planted systems take the Laurent-series fix-up (one warp each, dense
    double-double series from row j on); the share of the fix-up in the solve time is
    the time beyond the unplanted solve."""
    import torch
    import paper_1804_09666_gb300 as band
    grid = GRID
    B = synth.cfg1(r=2.0, k=2, sweep="y", grid=grid)
    n, nsys = B["n"], B["nsys"]
    xt = B["x_true"].reshape(n, nsys)
    units = n * nsys
    out = {"workload": "SPDM, ADI y-sweep r = 2, %d PD systems of n = %d, exact zero pivots "
                       "planted" % (nsys, n), "unit": UNIT}
    base_ms = None
    for frac in (0.0, 0.01, 0.1):
        D = {q: B[q].reshape(n, nsys).copy() for q in "abcde"}
        rng = np.random.default_rng(90 + int(1000 * frac))
        planted = rng.choice(nsys, size=int(round(frac * nsys)), replace=False)
        rows = rng.integers(4, n - 4, size=len(planted))
        for sy, j in zip(planted, rows):
            D["a"][j, sy] = D["b"][j, sy] = D["c"][j, sy] = 0.0
        f = synth.band_matvec(2, D["a"], D["b"], D["c"], D["d"], D["e"], xt)
        d = {q: torch.from_numpy(D[q]).to(dev) for q in "abcde"}
        ft = torch.from_numpy(f).to(dev)
        x = torch.empty_like(ft)
        res = {}

        def run():
            res["x"], res["st"] = band.solve(*(d[q] for q in "abcde"), ft, method="spdm", x=x)
        ms = _time(run, reps=3, warm=1)
        xg = res["x"].cpu().numpy()
        err = np.abs(xg - xt).max(0) / np.abs(xt).max(0)
        key = "planted_%g%%" % (100 * frac)
        out[key] = {"systems_planted": int(len(planted)), "value": units / (ms * 1e-3), "ms": ms,
                    "status_not_ok": int((res["st"] != 0).sum()),
                    "max_rel_err_vs_manufactured": float(err.max()),
                    "max_rel_err_planted": float(err[planted].max()) if len(planted) else None}
        if frac == 0.0:
            base_ms = ms
        else:
            out[key]["fixup_share"] = max(0.0, (ms - base_ms) / ms)
    return out


def mnpdm_workload(dev):
    """PD systems whose outer diagonals are mostly zero (Sec. 3.2 Remark 2: K << N rows
    carry them): 2048 dominant systems of n = 2048, off-diagonal magnitudes in [0.5, 1],
    outer entries kept on 1 % of the rows; MNPDM against NPDM (one thread per system and
    the automatic schedule) on the same matrices, interleaved."""
    import torch
    import paper_1804_09666_gb300 as band
    nsys, n = 2048, 2048
    rng = np.random.default_rng(1804_09666 + 200)
    # off-diagonals bounded away from 0 (as a stencil's are): MNPDM divides by them
    mag = lambda: rng.uniform(0.5, 1.0, (n, nsys)) * rng.choice([-1.0, 1.0], (n, nsys))
    D = {q: mag() for q in "abde"}
    keep = rng.random((n, nsys)) < 0.01
    D["a"] = np.where(keep, D["a"], 0.0)
    D["e"] = np.where(keep, D["e"], 0.0)
    D["a"][:2] = D["b"][:1] = 0.0
    D["d"][n - 1:] = D["e"][n - 2:] = 0.0
    D["c"] = 1.0 + sum(np.abs(D[q]) for q in "abde")
    xt, f = synth.manufactured(rng, 2, D, nsys, n)
    d = {q: torch.from_numpy(D[q]).to(dev) for q in "abcde"}
    ft = torch.from_numpy(f).to(dev)
    xtd = torch.from_numpy(xt).to(dev)
    units = n * nsys
    out = {"workload": "2048 PD systems, n = 2048, outer entries on 1 %% of the rows (K = %d "
                       "per system on average)" % int(keep.sum() / nsys), "unit": UNIT}
    for method, sched in (("mnpdm", "auto"), ("npdm", "thread"), ("npdm", "auto")):
        x = torch.empty_like(ft)
        res = {}

        def run():
            res["x"], res["st"] = band.solve(*(d[q] for q in "abcde"), ft, method=method, x=x,
                                             schedule=sched)
        ms = _time(run)
        err = float(((res["x"] - xtd).abs().amax(0) / xtd.abs().amax(0)).max())
        out["%s_%s" % (method, sched)] = {"value": units / (ms * 1e-3), "ms": ms,
                                          "status_not_ok": int((res["st"] != 0).sum()),
                                          "max_rel_err_vs_manufactured": err}
    return out


def adi_time_workload(dev, n=GRID, steps=10):
    """Time-stepping of u_t = Delta u + u (1 - u) + s on the 2048 x 2048 grid by
    Peaceman-Rachford ADI (band_adi_step): per step the right-hand-side stencil kernel,
    2048 row systems, the second stencil kernel, 2048 column systems; PD lines
    (fourth-order stencil, NPDM) and TD lines (3-point, NTDM); `steps` steps captured in
    one CUDA graph and replayed."""
    import torch
    import paper_1804_09666_gb300 as band
    rng = np.random.default_rng(1804_09666 + 300)
    src = torch.from_numpy(rng.uniform(-1, 1, (n, n))).to(dev)
    u0 = torch.from_numpy(rng.uniform(0, 1, (n, n))).to(dev)
    out = {"workload": "ADI time steps of u_t = Delta u + u (1 - u) + s, %d x %d grid, tau = "
                       "1e-4, %d steps per graph replay" % (n, n, steps), "unit": UNIT}
    for k, name in ((2, "pd_npdm"), (1, "td_ntdm")):
        stepper = band.AdiStepper(n, 1e-4, 1.0, src, half_bw=k)
        u = u0.clone()
        stepper.step(u)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                stepper.step(u, steps=steps)
        torch.cuda.current_stream().wait_stream(st)
        ms = _time(g.replay, reps=5) / steps
        bad = int((stepper.status != 0).sum())
        out[name] = {"ms_per_step": ms, "value": 2 * n * n / (ms * 1e-3),
                     "line_status_not_ok": bad,
                     "finite": bool(torch.isfinite(u).all().item())}
    return out


def sip2d_workload(dev, nsys=16384, nx=32, ny=32):
    """Stone's method where ILU(0) is incomplete: 16384 two-dimensional five-point systems
    of 32 x 32 unknowns (backward-Euler-like rows: neighbours -r times [0.5, 1], diagonal
    1 + 4r + [0, 0.1), r in [0.5, 4] per system: diagonally dominant M-matrices, for which
    ILU(0) is a regular splitting and Algorithm 1 converges), tol 1e-10, interleaved."""
    import torch
    import paper_1804_09666_gb300 as band
    rng = np.random.default_rng(1804_09666 + 400)
    N = nx * ny
    r = rng.uniform(0.5, 4.0, nsys)[None, :]
    d = {q: torch.from_numpy(-r * rng.uniform(0.5, 1.0, (N, nsys))).to(dev) for q in "swet"}
    d["c"] = torch.from_numpy(1 + 4 * r + rng.uniform(0, 0.1, (N, nsys))).to(dev)
    f = torch.from_numpy(rng.uniform(-1, 1, (N, nsys))).to(dev)
    res = {}

    def run():
        res["x"], res["it"], res["rs"], res["st"] = band.sip2d(
            d["s"], d["w"], d["c"], d["e"], d["t"], f, nx, tol=1e-10, max_it=500)
    ms = _time(run)
    units = N * nsys
    it = res["it"].float()
    return {"workload": "Stone's method on %d 2-D five-point systems of %d x %d, tol 1e-10"
                        % (nsys, nx, ny), "unit": UNIT, "value": units / (ms * 1e-3), "ms": ms,
            "iters_mean": float(it.mean()), "iters_max": int(it.max()),
            "status_not_ok": int((res["st"] != 0).sum()),
            "max_resid": float(res["rs"].max())}


# The paper's single-system timings at N = 10^8 (Table 3, HybriLIT, one Xeon E5-2695v2
# core, double precision): NPDM 2.7946627 s, NTDM 2.0525187 s.  Context only.
PAPER_1E8_S = {"npdm": 2.7946627, "ntdm": 2.0525187}


def single_system_workload(dev, n=100_000_000):
    """One dominant system of n = 10^8 rows (the paper's largest N), PD by NPDM and TD by
    NTDM, on the grid schedule (all SMs on one system), against the manufactured
    solution.  The paper's one-core times at the same N are quoted for context."""
    import torch
    import paper_1804_09666_gb300 as band
    out = {"workload": "one system of n = %d rows, dominant (cfg0 recipe), grid schedule" % n,
           "unit": UNIT}
    for k, method in ((2, "npdm"), (1, "ntdm")):
        rng = np.random.default_rng(1804_09666 + 100 + k)
        D = synth.dominant(rng, 1, n, k=k)
        xt, f = synth.manufactured(rng, k, D, 1, n)
        d = {q: torch.from_numpy(D[q]).to(dev) for q in "abcde"}
        ft = torch.from_numpy(f).to(dev)
        del D, f
        xtd = torch.from_numpy(xt).to(dev)
        del xt
        x = torch.empty_like(ft)
        desc = band.desc_for(ft, k, "grid")
        ws = torch.empty(band.load().band_workspace_size(ct.byref(desc), 0, 1 if k == 2 else 0, 0),
                         dtype=torch.uint8, device=dev)
        res = {}

        def run():
            res["x"], res["st"] = band.solve(d["a"] if k == 2 else None, d["b"], d["c"], d["d"],
                                             d["e"] if k == 2 else None, ft, method=method, x=x,
                                             schedule="grid", ws=ws)
        run()
        torch.cuda.synchronize()
        ms = _time(run, reps=5, warm=1)
        err = float(((res["x"] - xtd).abs().max() / xtd.abs().max()).item())
        flops = (19 if k == 2 else 9) * n
        out[method] = {"value": n / (ms * 1e-3), "ms": ms, "status": int(res["st"].item()),
                       "max_rel_err_vs_manufactured": err,
                       "alg_GBps": (56 if k == 2 else 40) * n / (ms * 1e-3) / 1e9,
                       "table7_TFLOPs": flops / (ms * 1e-3) / 1e12,
                       "paper_one_core_s": PAPER_1E8_S[method],
                       "paper_one_core_unknowns_per_s": n / PAPER_1E8_S[method]}
        del d, ft, xtd, x, res
        torch.cuda.empty_cache()
    return out


EXTRA_WORKLOADS = {"ragged": "ragged_workload", "small_batch": "small_batch_workload",
                   "precision": "precision_workload", "adjoint": "adjoint_workload",
                   "sip": "sip_workload", "symbolic": "symbolic_workload",
                   "single": "single_system_workload", "mnpdm": "mnpdm_workload",
                   "adi_time": "adi_time_workload", "sip2d": "sip2d_workload",
                   "cfg0": "cfg0_workload"}


# ---------------------------------------------------------------------- main
def main():
    args = parse()
    if args.workload:
        import torch
        dev = torch.device("cuda", 0)
        fn = globals()[EXTRA_WORKLOADS[args.workload]]
        out = fn(dev, nsys=args.ragged_nsys) if args.workload == "ragged" else fn(dev)
        print(json.dumps({"workload": args.workload, "result": out}))
        return
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
    D = DeviceSet(W, dev, use_graph=not args.no_graph)
    units = units_per_step(W)

    # FP64 FMA rate of this GPU (the ALU roofline of the FP64 recurrences)
    scratch = torch.empty(8 * 256 * 8 * 256, dtype=torch.uint8, device=dev)
    fma_rate = lib.band_fp64_fma_rate(ct.c_void_p(scratch.data_ptr()), scratch.numel(),
                                      ct.c_void_p(torch.cuda.current_stream().cuda_stream))

    bad = D.statuses()
    for _ in range(max(args.warmup, 3)):
        D.step()
    torch.cuda.synchronize()

    # timed region: inputs resident in HBM.  The clock sampler starts first and gets
    # half a second to deliver its first sample while the GPU is kept busy.
    clocks = ClockSampler(torch.cuda.current_device())
    events = EventLog()
    clocks.start()
    t_spin = time.perf_counter()
    while time.perf_counter() - t_spin < 0.5:
        D.step()
        torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
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

    # end to end: every step copies its inputs from pinned host memory, solves them
    # through the batched plan and reads its results back into pinned host memory.
    # Consecutive steps overlap on three streams (H2D of step k+1, the solves of step k,
    # D2H of step k-1) with two device sets used in turn.
    D2 = DeviceSet(W, dev, use_graph=not args.no_graph, host=D)
    ms_e2e = e2e_pipelined([D, D2], args.steps, world)
    ms_serial = e2e_serial(D, args.steps, world)
    e2e = {"value": units * args.steps * world / (ms_e2e * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": D.h2d_bytes, "d2h_bytes_per_step": D.d2h_bytes,
           "overlap": "H2D of step k+1, solves of step k and D2H of step k-1 on three streams",
           "serial_value": units * args.steps * world / (ms_serial * 1e-3)}

    # the batched launch's time per step (CUDA events on the launching stream inside the
    # timed region) against the algorithmic bytes and flops of the 30 solves it does
    per = events.summary()["batch"]
    avg_ms = float(np.mean(per))
    alg_bytes, alg_flops = D.alg(ALG_BYTES), D.alg(ALG_FLOPS)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak_tf = 2.0 * fma_rate / 1e12 if fma_rate > 0 else 1.25
    gbps = alg_bytes / (avg_ms * 1e-3) / 1e9
    tflops = alg_flops / (avg_ms * 1e-3) / 1e12
    frac_hbm, frac_alu = gbps / hbm_peak, tflops / fp64_peak_tf
    common = {"kernel": "k_batch (one launch: the 30 solves of a step); the events bracket the "
                        "step's graph replay, which adds the symbolic fix-up and SIP tail launches",
              "ms_per_launch": avg_ms, "launches": len(per),
              "alg_bytes_per_launch": alg_bytes, "alg_flops_per_launch": alg_flops}
    traffic = recorded_traffic(args.grid)
    if frac_alu >= frac_hbm:
        roof = dict({"bound": "alu", "achieved": tflops, "peak": fp64_peak_tf, "unit": "TFLOP/s",
                     "frac": frac_alu, "traffic": traffic,
                     "peak_source": "measured FP64 FMA rate (band_fp64_fma_rate) x 2",
                     "hbm_GBps": gbps, "hbm_frac_of_measured": frac_hbm}, **common)
    else:
        roof = dict({"bound": "hbm", "achieved": gbps, "peak": hbm_peak, "unit": "GB/s",
                     "frac": frac_hbm, "traffic": traffic, "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                     "fp64_TFLOPs": tflops, "alu_frac_of_measured": frac_alu}, **common)
    launches_per_step = D.kernels_per_step()     # plus one counter memset per SIP/symbolic solve

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.grid, world),
            "clocks": ck, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "status_not_ok": bad,
            "fp64_fma_per_s": fma_rate}
    if rank == 0:
        line["accuracy"] = accuracy_report(D)
    if rank == 0 and world == 1 and not args.no_extras and args.grid == GRID:
        line["workloads"] = {"per_method": per_method_workload(D),
                             "cfg0": cfg0_workload(dev), "ragged": ragged_workload(dev),
                             "small_batch": small_batch_workload(dev),
                             "precision": precision_workload(dev),
                             "adjoint": adjoint_workload(dev), "sip": sip_workload(dev),
                             "symbolic": symbolic_workload(dev),
                             "single": single_system_workload(dev),
                             "mnpdm": mnpdm_workload(dev),
                             "adi_time": adi_time_workload(dev),
                             "sip2d": sip2d_workload(dev)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
