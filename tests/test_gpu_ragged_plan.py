"""GPU parity of the batch runtime on ragged batches: size buckets (band_plan_ragged)
solved in one batched launch on each schedule, the autotuner's choice, symbolic
fix-ups inside buckets, and capture in a CUDA graph."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import DEV

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


@pytest.fixture(scope="module")
def ragged():
    B = synth.cfg2(nsys=3000, nmin=16, nmax=2000, seed_salt=5)
    dev = {q: torch.from_numpy(B[q]).to(DEV) for q in "abcdef"}
    return B, dev


def _per_system_err(B, x):
    err = np.abs(x - B["x_true"])
    return np.maximum.reduceat(err, B["offsets"][:-1])


@pytest.mark.parametrize("schedule", ["thread", "two_sided", "auto", "tune"])
def test_buckets_every_schedule(band, ragged, schedule):
    B, dev = ragged
    plan = band.RaggedPlan(*(dev[q] for q in "abcdef"), B["offsets"], B["hbw"], schedule=schedule)
    x, st = plan.run()
    torch.cuda.synchronize()
    assert (st.cpu() == 0).all()
    assert _per_system_err(B, x.cpu().numpy()).max() <= 1e-12
    assert len(plan.buckets) == len({(int(k), int(np.log2(n))) for k, n in zip(B["hbw"], B["sizes"])})
    if schedule == "tune":
        assert set(plan.schedules) <= {1, 2, 3}       # the joint search may partition
        assert all((v == 3) == (c in (8, 16, 32)) for v, c in zip(plan.schedules, plan.chunks))
    # against the oracle on a sample of systems from every bucket
    xg = x.cpu().numpy()
    order = plan.order.cpu().numpy()
    for first, count, n_max, k in plan.buckets:
        for s in order[first:first + count][:: max(1, count // 3)]:
            S = synth.system(B, int(s))
            xo, _ = (oracle.ntdm(S["b"], S["c"], S["d"], S["f"]) if k == 1
                     else oracle.npdm(*(S[q] for q in "abcdef")))
            lo, hi = int(B["offsets"][s]), int(B["offsets"][s + 1])
            assert np.abs(xg[lo:hi] - xo).max() / np.abs(xo).max() <= 1e-12


def test_thread_buckets_equal_the_whole_packing(band, ragged):
    """One thread per system in buckets does the same arithmetic as the whole-packing
    solve (only the scratch rows sit elsewhere): bitwise equal."""
    B, dev = ragged
    plan = band.RaggedPlan(*(dev[q] for q in "abcdef"), B["offsets"], B["hbw"], schedule="thread")
    x1, st1 = plan.run()
    offs = torch.from_numpy(B["offsets"]).to(DEV)
    hbw = torch.from_numpy(B["hbw"]).to(DEV)
    x2, st2 = band.solve_ragged(*(dev[q] for q in "abcdef"), offs, hbw,
                                n_max=int(B["sizes"].max()), total_rows=int(B["offsets"][-1]))
    torch.cuda.synchronize()
    assert torch.equal(st1, st2) and torch.equal(x1, x2)


def test_symbolic_buckets_with_zero_pivots(band):
    """The hand-made zero-pivot systems packed ragged between dominant ones: STDM/SPDM
    buckets on the two-sided schedule return the exact solutions (or SINGULAR)."""
    cases = json.load(open(os.path.join(GOLD, "zero_pivot_cases.json")))["cases"]
    rng = np.random.default_rng(3)
    arrays = {q: [] for q in "abcdef"}
    sizes, hbw, want = [], [], []
    for rep in range(8):
        for case in cases:
            k, n = case["k"], case["n"]
            for q in "abcdef":
                arrays[q].append(np.array([float(Fraction(v)) for v in case[q]]))
            sizes.append(n)
            hbw.append(k)
            want.append((case["status"], np.array([float(Fraction(v)) for v in case["x"]])
                         if case["status"] == "OK" else None))
            n2 = int(rng.integers(40, 300))
            D = synth.dominant(rng, 1, n2, k=k)
            xt, f = synth.manufactured(rng, k, D, 1, n2)
            for q in "abcde":
                arrays[q].append(D[q][:, 0])
            arrays["f"].append(f[:, 0])
            sizes.append(n2)
            hbw.append(k)
            want.append(("OK", xt[:, 0]))
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    dev = {q: torch.from_numpy(np.concatenate(arrays[q])).to(DEV) for q in "abcdef"}
    for schedule in ("two_sided", "thread", "partitioned"):
        plan = band.RaggedPlan(*(dev[q] for q in "abcdef"), offs, np.array(hbw, np.int8),
                               method="symbolic", schedule=schedule, chunks=8 if schedule == "partitioned" else 0)
        x, st = plan.run()
        torch.cuda.synchronize()
        xg, st = x.cpu().numpy(), st.cpu().numpy()
        for s, (status, xw) in enumerate(want):
            if status == "SINGULAR":
                assert st[s] == 4, (schedule, s)
                continue
            assert st[s] == 0, (schedule, s, st[s])
            xs = xg[offs[s]:offs[s + 1]]
            assert np.abs(xs - xw).max() <= 1e-12 * max(1.0, np.abs(xw).max()), (schedule, s)


def test_graph_capture(band, ragged):
    B, dev = ragged
    plan = band.RaggedPlan(*(dev[q] for q in "abcdef"), B["offsets"], B["hbw"], schedule="tune")
    x, st = plan.run()
    torch.cuda.synchronize()
    want = x.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        x.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(x, want)
