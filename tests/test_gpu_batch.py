"""GPU parity: band_solve_batch (several problems in one launch) against the single-
problem calls (same sweeps, so bitwise equal) and the CPU oracle, and its capture in a
CUDA graph."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import DEV, flat_of, per_system_rel, to_dev

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _zero_pivot_batch(k):
    """40 copies of a golden zero-pivot case of bandwidth k, interleaved."""
    cases = json.load(open(os.path.join(GOLD, "zero_pivot_cases.json")))["cases"]
    case = next(c for c in cases if c["k"] == k and c["status"] == "OK" and c["n"] >= 7)
    n, nsys = case["n"], 40
    B = dict(n=n, nsys=nsys, sys_stride=1, elem_stride=nsys)
    for q in "abcdef":
        v = np.array([float(Fraction(t)) for t in case[q]])
        B[q] = np.repeat(v[:, None], nsys, axis=1).reshape(-1)
    return B, np.array([float(Fraction(t)) for t in case["x"]])


def _specs(band):
    P0 = to_dev(synth.cfg0(nsys=100, n=257, seed_salt=1))
    T1 = to_dev(synth.cfg0(nsys=70, n=90, k=1, layout="contiguous", seed_salt=2))
    Z2, xz2 = _zero_pivot_batch(2)
    Z1, xz1 = _zero_pivot_batch(1)
    Z2d, Z1d = to_dev(Z2), to_dev(Z1)
    P32 = to_dev(synth.cfg0(nsys=64, n=130, seed_salt=3), dtype=torch.float32)
    S = to_dev(synth.cfg1(r=2.0, k=2, sweep="y", grid=512, nsys=96))
    specs = [
        dict(method="npdm", **{q: P0[q] for q in "abcdef"}),
        dict(method="ntdm", a=None, e=None, **{q: T1[q] for q in "bcdf"}),
        dict(method="spdm", **{q: Z2d[q] for q in "abcdef"}),
        dict(method="stdm", a=None, e=None, **{q: Z1d[q] for q in "bcdf"}),
        dict(method="npdm", **{q: P32[q] for q in "abcdef"}),
        dict(op="sip", tol=1e-10, max_it=200, **{q: S[q] for q in "abcdef"}),
        dict(method="spdm", **{q: P0[q] for q in "abcdef"}),
    ]
    return specs, (xz2, xz1)


def _single(band, sp):
    if sp.get("op") == "sip":
        # the batched kernel runs SIP on one thread per system
        x, it, rs, st = band.sip(*(sp[q] for q in "abcdef"), tol=sp["tol"], max_it=sp["max_it"],
                                 width=0, schedule="thread")
        return dict(x=x, status=st, iters=it, resid=rs)
    # inside a batch AUTO stays two-sided for n >= 32 (the other problems fill the GPU);
    # a single call on AUTO would take the partitioned schedule for these small batches
    sched = "two_sided" if sp["c"].shape[0] >= 32 else "auto"
    x, st = band.solve(*(sp.get(q) for q in "abcdef"), method=sp["method"], schedule=sched)
    return dict(x=x, status=st)


def test_batch_equals_single_calls(band):
    specs, (xz2, xz1) = _specs(band)
    plan = band.BatchPlan(specs)
    res = plan.run()
    torch.cuda.synchronize()
    for sp, r in zip(specs, res):
        ref = _single(band, sp)
        torch.cuda.synchronize()
        assert torch.equal(r["status"], ref["status"])
        assert torch.equal(r["x"], ref["x"]), sp.get("method", sp.get("op"))
        if "iters" in r:
            assert torch.equal(r["iters"], ref["iters"])
    # every status OK; the symbolic problems return the exact rational solutions
    for r in res:
        assert (r["status"].cpu() == 0).all()
    for r, want in ((res[2], xz2), (res[3], xz1)):
        xg = r["x"].cpu().numpy()
        assert np.abs(xg - want[:, None]).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_batch_against_oracle(band):
    B = synth.cfg1(r=10.0, k=2, sweep="x", grid=1024, nsys=128)
    T = to_dev(B)
    res = band.solve_batch([dict(method="npdm", **{q: T[q] for q in "abcdef"}),
                            dict(op="sip", **{q: T[q] for q in "abcdef"})])
    torch.cuda.synchronize()
    args = (B["n"], B["nsys"], B["sys_stride"], B["elem_stride"])
    oargs = (B["nsys"], B["n"], B["sys_stride"], B["elem_stride"])
    xo, so, _, _ = oracle.batch("direct", 2, [B[q] for q in "abcde"], B["f"], *oargs)
    xt, _, _, _ = oracle.batch("gepp", 2, [B[q] for q in "abcde"], B["f"], *oargs)
    err_o = per_system_rel(xo, xt, *args)
    for r in res:
        err = per_system_rel(flat_of(r["x"]), xt, *args)
        assert (err <= np.maximum(1e-10, 10 * err_o)).all()


def test_batch_capture_in_cuda_graph(band):
    specs, _ = _specs(band)
    plan = band.BatchPlan(specs)
    plan.run()
    torch.cuda.synchronize()
    want = [r["x"].clone() for r in plan.results]
    for r in plan.results:
        r["x"].zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for r in plan.results:
            r["x"].zero_()
        g.replay()
        torch.cuda.synchronize()
        for r, w in zip(plan.results, want):
            assert torch.equal(r["x"], w)


def test_batch_argument_errors(band):
    import ctypes as ct
    from paper_1804_09666_gb300 import _lib as L
    lib = band.load()
    arr = (L.BandProblem * 65)()
    assert lib.band_solve_batch(arr, 65, None) == L.ERR_ARG
    assert lib.band_solve_batch(arr, 1, None) == L.ERR_ARG          # desc NULL
    assert lib.band_solve_batch(None, 0, None) == L.OK
    T = to_dev(synth.cfg0(nsys=32, n=16))
    plan = band.BatchPlan([dict(method="npdm", **{q: T[q] for q in "abcdef"})])
    plan.arr[0].ws_bytes = 8                                          # too small
    assert lib.band_solve_batch(plan.arr, 1, None) == L.ERR_WORKSPACE
