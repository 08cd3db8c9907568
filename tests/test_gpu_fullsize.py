"""GPU parity at the workloads' full sizes, in the launch configurations the library
uses for them: whole-batch properties that hold at any size (every status, the forward
error of the manufactured solution) and sampled systems that the CPU oracle recomputes
one by one.  (The ADI workload's full-size check sits in test_gpu_direct.py.)"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import DEV, flat_of, strided_view, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def test_ragged_65536_systems(band):
    """The batching workload: 65536 systems, n log-uniform in [16, 8192] (~86 M rows),
    half TD / half PD, packed with offsets, one thread per system."""
    B = synth.cfg2()
    dev = {q: torch.from_numpy(B[q]).to(DEV) for q in "abcdef"}
    offs = torch.from_numpy(B["offsets"]).to(DEV)
    hbw = torch.from_numpy(B["hbw"]).to(DEV)
    x, st = band.solve_ragged(dev["a"], dev["b"], dev["c"], dev["d"], dev["e"], dev["f"], offs,
                              hbw, n_max=int(B["sizes"].max()), total_rows=int(B["offsets"][-1]),
                              method="auto")
    torch.cuda.synchronize()
    assert (st.cpu() == 0).all()
    xg = x.cpu().numpy()
    # every system against its manufactured solution (dominant: error ~ n u)
    err = np.abs(xg - B["x_true"])
    per = np.maximum.reduceat(err, B["offsets"][:-1])
    assert per.max() <= 1e-12
    # 64 sampled systems, shortest and longest included, against the oracle
    rng = np.random.default_rng(7)
    sizes = B["sizes"]
    pick = set(rng.choice(len(sizes), 62, replace=False).tolist())
    pick |= {int(np.argmin(sizes)), int(np.argmax(sizes))}
    for s in sorted(pick):
        S = synth.system(B, s)
        if B["hbw"][s] == 1:
            xo, so = oracle.ntdm(S["b"], S["c"], S["d"], S["f"])
        else:
            xo, so = oracle.npdm(*(S[q] for q in "abcdef"))
        lo, hi = int(B["offsets"][s]), int(B["offsets"][s + 1])
        assert np.abs(xg[lo:hi] - xo).max() / np.abs(xo).max() <= 1e-12, s


def test_ragged_65536_systems_tuned_buckets(band):
    """The same batch in bench.py's configuration: size buckets in one batched launch,
    schedules from the joint autotuner (the longest buckets partitioned), replayed from a
    CUDA graph.  Every system against its manufactured solution; sampled systems from
    every bucket, the longest of each included, against the oracle."""
    B = synth.cfg2()
    dev = {q: torch.from_numpy(B[q]).to(DEV) for q in "abcdef"}
    plan = band.RaggedPlan(*(dev[q] for q in "abcdef"), B["offsets"], B["hbw"], schedule="tune")
    assert 3 in plan.schedules                     # some bucket runs partitioned
    plan.run()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    plan.x.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert (plan.status.cpu() == 0).all()
    xg = plan.x.cpu().numpy()
    per = np.maximum.reduceat(np.abs(xg - B["x_true"]), B["offsets"][:-1])
    assert per.max() <= 1e-12
    order = plan.order.cpu().numpy()
    rng = np.random.default_rng(8)
    for (first, count, n_max, k), sched in zip(plan.buckets, plan.schedules):
        ids = order[first:first + count]
        pick = {int(ids[0])} | set(rng.choice(ids, min(3, count), replace=False).tolist())
        for sid in sorted(pick):
            S = synth.system(B, sid)
            if k == 1:
                xo, _ = oracle.ntdm(S["b"], S["c"], S["d"], S["f"])
            else:
                xo, _ = oracle.npdm(*(S[q] for q in "abcdef"))
            lo, hi = int(B["offsets"][sid]), int(B["offsets"][sid + 1])
            assert np.abs(xg[lo:hi] - xo).max() / np.abs(xo).max() <= 1e-12, (sid, sched)


def test_small_batch_64_x_65536_partitioned(band):
    """bench.py's small batch: 64 PD systems of n = 65536 on the partitioned schedule with
    the library's chunk count (a block of warps per system).  Every system against its
    manufactured solution, and 4 of them against the oracle."""
    B = synth.cfg0(nsys=64, n=65536, seed_salt=80)
    T = to_dev(B)
    x, st = band.solve(*(T[q] for q in "abcdef"), method="npdm", schedule="partitioned")
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    n, ns = B["n"], B["nsys"]
    xg = flat_of(x).reshape(n, ns)
    xt = B["x_true"].reshape(n, ns)
    assert (np.abs(xg - xt).max(0) / np.abs(xt).max(0)).max() <= 1e-12
    for s_ in (0, 21, 42, 63):
        col = {q: B[q].reshape(n, ns)[:, s_] for q in "abcdef"}
        xo, _ = oracle.npdm(*(col[q] for q in "abcdef"))
        assert np.abs(xg[:, s_] - xo).max() / np.abs(xo).max() <= 1e-12, s_


@pytest.mark.parametrize("pairs", [False, True])
def test_refine_16384_x_4096(band, pairs):
    """The precision workload: 16384 PD systems of n = 4096 in FP32, refined with the
    residual and update in FP64 (or FP32 pairs).  Every system reaches relative forward
    error <= 1e-10 against its manufactured solution; 12 sampled systems also against
    the oracle's GEPP and refinement (step counts within one)."""
    nsys, n = 16384, 4096
    B = synth.cfg3()
    T = to_dev(B, keys="abcde", dtype=torch.float32)
    f = strided_view(B["f"], n, nsys, 1, nsys)
    x, steps, st = band.refine_solve(T["a"], T["b"], T["c"], T["d"], T["e"], f, pairs=pairs)
    torch.cuda.synchronize()
    assert (st.cpu() == 0).all()
    steps = steps.cpu().numpy()
    assert (steps >= 1).all() and (steps <= 10).all()
    xg = x.cpu().numpy()
    xt = B["x_true"].reshape(n, nsys)
    rel = np.abs(xg - xt).max(0) / np.abs(xt).max(0)
    assert rel.max() <= 1e-10
    for s in np.random.default_rng(8).choice(nsys, 12, replace=False):
        S = {q: B[q].reshape(n, nsys)[:, s] for q in "abcde"}
        fs = B["f"].reshape(n, nsys)[:, s]
        xo, so, _ = oracle.gepp_band(2, *(S[q].astype(np.float64) for q in "abcde"), fs)
        assert np.abs(xg[:, s] - xo).max() / np.abs(xo).max() <= 1e-10
        _, ko, sto = oracle.refine(*(S[q] for q in "abcde"), fs)
        assert sto == "OK" and abs(int(steps[s]) - ko) <= 1


def test_adjoint_4096_x_1024(band):
    """The differentiation workload: gradients of sum(w * x) for 4096 PD systems of
    n = 1024; 16 sampled systems against the oracle's adjoint (rel. 1e-11)."""
    nsys, n = 4096, 1024
    B = synth.cfg4()
    T = to_dev(B, keys="abcdefw")
    x, st = band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], T["f"], method="npdm")
    (ga, gb, gc, gd, ge), gf, sta = band.adjoint(T["a"], T["b"], T["c"], T["d"], T["e"], x, T["w"])
    torch.cuda.synchronize()
    assert (st.cpu() == 0).all() and (sta.cpu() == 0).all()
    xg = x.cpu().numpy()
    G = [g.cpu().numpy() for g in (ga, gb, gc, gd, ge, gf)]
    w = B["w"].reshape(n, nsys)
    for s in np.random.default_rng(9).choice(nsys, 16, replace=False):
        S = synth.system(B, int(s))
        go, gfo, sto = oracle.adjoint(2, *(S[q] for q in "abcde"), xg[:, s], w[:, s])
        assert sto == "OK"
        for g_gpu, g_orc in zip(G, list(go) + [gfo]):
            den = max(np.abs(g_orc).max(), 1e-300)
            assert np.abs(g_gpu[:, s] - g_orc).max() / den <= 1e-11
