"""The autotuner's persisted decisions (band_autotune with BAND_TUNE_CACHE): a tuning
process writes one JSON line per decision, keyed by the GPU and the CUDA version; a
second process reads them back instead of timing (a planted file is obeyed: schedules
flipped by hand come back flipped, the planted block size is the one band_solve_batch
launches with), lines of another GPU or CUDA version are ignored, and the kernel's one-,
two- and four-warp blocks give the same solutions bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# tune: tune jointly and save the solutions; load: take the persisted decisions
# (flags 0: no timing of anything already decided), report them, then solve on the
# first process's schedules and save the solutions
SCRIPT = r"""
import ctypes as ct, json, sys
import numpy as np, torch
sys.path[:0] = [sys.argv[3], sys.argv[3] + "/tests"]
import synth
from gpu_helpers import to_dev
import paper_1804_09666_gb300 as band
from paper_1804_09666_gb300 import _lib as L
from paper_1804_09666_gb300.band import _stream
mode, out = sys.argv[1], sys.argv[2]
lib = L.load()
P = to_dev(synth.cfg0(nsys=300, n=200, seed_salt=11))
T = to_dev(synth.cfg0(nsys=90, n=40, k=1, layout="contiguous", seed_salt=12))
specs = [dict(method="npdm", **{q: P[q] for q in "abcdef"}),
         dict(method="ntdm", a=None, e=None, **{q: T[q] for q in "bcdf"})]
if mode == "tune":
    b = band.BatchPlan(specs, tune=True)
    info = dict(schedules=b.schedules, chunks=b.chunks)
else:
    b = band.BatchPlan(specs)
    s = (ct.c_int32 * 2)()
    c = (ct.c_int32 * 2)()
    L.check(lib.band_autotune(b.arr, 2, 3, 0, s, c, _stream()), "band_autotune")
    info = dict(schedules=list(s), chunks=list(c))
    first = json.load(open(out + ".tune.json"))
    names = {1: "thread", 2: "two_sided", 3: "partitioned"}
    for sp, sch, ch in zip(specs, first["schedules"], first["chunks"]):
        sp.update(schedule=names[sch], chunks=ch)
    b = band.BatchPlan(specs)
info["warps"] = lib.band_batch_warps(torch.cuda.current_device())
b.run()
torch.cuda.synchronize()
assert all((r["status"] == 0).all().item() for r in b.results)
np.savez(out + "." + mode + ".npz", *[r["x"].cpu().numpy() for r in b.results])
json.dump(info, open(out + "." + mode + ".json", "w"))
"""


def _run(mode, out, cache):
    env = dict(os.environ, BAND_TUNE_CACHE=cache)
    subprocess.run([sys.executable, "-c", SCRIPT, mode, out, ROOT], env=env, check=True,
                   cwd=ROOT, timeout=600)
    return json.load(open(out + "." + mode + ".json"))


def _xs(out, mode):
    z = np.load(out + "." + mode + ".npz")
    return [z["arr_%d" % i] for i in range(len(z.files))]


def test_persisted_decisions(tmp_path):
    from paper_1804_09666_gb300 import build
    build.build()
    cache = str(tmp_path / "sub" / "tune.jsonl")     # the directory is created
    out = str(tmp_path / "run")
    first = _run("tune", out, cache)
    assert first["warps"] in (1, 2, 4)
    lines = [json.loads(s) for s in open(cache)]
    kinds = [ln["kind"] for ln in lines]
    assert kinds.count("schedule") == 2 and kinds.count("batch_warps") == 1
    gpu = {(ln["gpu"], ln["cc"], ln["cuda"]) for ln in lines}
    assert len(gpu) == 1
    sched = [ln for ln in lines if ln["kind"] == "schedule"]
    assert sorted(ln["key"][2] for ln in sched) == [1, 2]         # half bandwidths
    assert {ln["value"] for ln in sched} <= {1, 2}
    for ln in lines:
        if ln["kind"] == "batch_warps":
            assert ln["value"] == first["warps"]
    # the NTDM problem (n = 40 < 64) is never partitioned: its step-1 choice stands
    td = next(ln for ln in sched if ln["key"][2] == 1)
    assert first["schedules"][1] == td["value"]

    want = _xs(out, "tune")
    for planted in (1, 4):
        flipped = []
        for ln in lines:
            ln = dict(ln)
            if ln["kind"] == "schedule":
                ln["value"] = 3 - ln["value"]            # THREAD <-> TWO_SIDED
            else:
                ln["value"] = planted
            flipped.append(ln)
        # another GPU's and another CUDA version's lines come last and must not win
        other = dict(flipped[-1], gpu="another device", value=2 if planted != 2 else 1)
        old = dict(flipped[-1], cuda=flipped[-1]["cuda"] - 10, value=2 if planted != 2 else 1)
        with open(cache, "w") as fp:
            for ln in flipped + [other, old]:
                fp.write(json.dumps(ln) + "\n")
        got = _run("load", out, cache)
        by_hbw = {ln["key"][2]: ln["value"] for ln in flipped if ln["kind"] == "schedule"}
        assert got["schedules"] == [by_hbw[2], by_hbw[1]]
        assert got["warps"] == planted
        for a, b in zip(want, _xs(out, "load")):
            assert np.array_equal(a, b), planted


def test_no_file_when_disabled(tmp_path):
    """An empty BAND_TUNE_CACHE keeps every decision in the process."""
    from paper_1804_09666_gb300 import build
    build.build()
    out = str(tmp_path / "run")
    env_home = str(tmp_path / "home")
    os.makedirs(env_home)
    env = dict(os.environ, BAND_TUNE_CACHE="", HOME=env_home)
    subprocess.run([sys.executable, "-c", SCRIPT, "tune", out, ROOT], env=env, check=True,
                   cwd=ROOT, timeout=600)
    assert not os.path.exists(os.path.join(env_home, ".cache"))
