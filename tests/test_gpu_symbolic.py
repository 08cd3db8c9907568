"""GPU parity of STDM / SPDM (Sec. 1) and of the O(N) determinant (Sec. 3.2, Remark 1)
where zero pivots crowd, against exact rational functions of t.

Integer systems whose diagonal is mostly 0 (so several pivots vanish and the symbol
meets itself in later pivots: poles, exact cancellations of series coefficients) are
solved through the C ABI on every schedule and through band_solve_batch.  Every system
whose exact elimination meets a zero pivot is compared with oracle.exact's rational
limit: a nonsingular matrix must give the exact solution (to the rounding of its
condition) with status OK, or SYMBOLIC_RANGE on at most 1 % of them; a singular one
must give SINGULAR, or SYMBOLIC_RANGE (the series pass could not decide) on at most
1 % of them.  No wrong result with status OK, no false SINGULAR.  Planted zero
pivots at the ADI workload's size check the series pass on long systems.
"""
import multiprocessing as mp

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import DEV
from oracle import exact

pytestmark = pytest.mark.gpu

U = np.finfo(np.float64).eps / 2
OK, SINGULAR, NONFINITE, RANGE = 0, 4, 5, 7


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _draw(k, seed, trials):
    """Crowded-zero integer systems (n = 3 .. 16) and their exact symbolic solutions;
    only systems whose exact elimination meets a zero pivot are kept."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(trials):
        n = int(rng.integers(3, 17))
        pick = lambda vals: [int(v) for v in rng.choice(vals, n)]
        a, b, d, e, f = (pick([-2, -1, 0, 0, 1, 2]) for _ in range(5))
        c = pick([0, 0, 0, 1, -1])
        if k == 1:
            a, e = [0] * n, [0] * n
        sym = exact.symbolic_solve(k, a, b, c, d, e, f)
        if sym["nflag"] == 0:
            continue
        out.append(dict(k=k, n=n, a=a, b=b, c=c, d=d, e=e, f=f, status=sym["status"],
                        x=[float(v) if v is not None else np.nan for v in sym["x"]],
                        det=float(sym["det"])))
    return out


@pytest.fixture(scope="module")
def crowded():
    """At least 1100 flagged systems per bandwidth (TD and PD), exact results computed
    in spawned worker processes (forked ones would inherit the CUDA context)."""
    jobs = [(k, 600 + 10 * k + j, 400) for k in (1, 2) for j in range(3)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(6, mp.cpu_count())) as pool:
        parts = pool.starmap(_draw, jobs)
    by_k = {1: [], 2: []}
    for p in parts:
        for sy in p:
            by_k[sy["k"]].append(sy)
    assert len(by_k[1]) >= 1000 and len(by_k[2]) >= 1000
    return by_k


def _groups(systems):
    """Uniform interleaved batches, one per system size: {n: (tensors, systems)}."""
    out = {}
    for n in sorted({s["n"] for s in systems}):
        group = [s for s in systems if s["n"] == n]
        T = {q: torch.tensor(np.array([s[q] for s in group], dtype=np.float64).T.copy(),
                             device=DEV) for q in "abcdef"}
        out[n] = (T, group)
    return out


def _classify(x, st, group, k):
    """Compare one group's results with the exact limits; returns counts."""
    res = dict(ok=0, range=0, nonsingular=0, singular=0, singular_range=0)
    for j, sy in enumerate(group):
        if sy["status"] == "SINGULAR":
            res["singular"] += 1
            assert st[j] in (SINGULAR, RANGE), (sy, st[j])
            res["singular_range"] += st[j] == RANGE
            continue
        res["nonsingular"] += 1
        if st[j] == RANGE:
            res["range"] += 1
            continue
        assert st[j] == OK, (sy, st[j])
        xe = np.array(sy["x"])
        A = exact.dense(k, sy["a"], sy["b"], sy["c"], sy["d"], sy["e"])
        kappa = np.linalg.cond(np.array(A, dtype=float), np.inf)
        err = np.abs(x[:, j] - xe).max()
        assert err <= 1e3 * kappa * U * max(1.0, np.abs(xe).max()), (sy, x[:, j], err)
        res["ok"] += 1
    return res


def _tally(total, res):
    for key, v in res.items():
        total[key] = total.get(key, 0) + v


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("schedule,chunks", [("thread", 0), ("two_sided", 0),
                                             ("partitioned", 8)])
def test_crowded_zero_pivots_every_schedule(band, crowded, k, schedule, chunks):
    method = "spdm" if k == 2 else "stdm"
    total = {}
    for n, (T, group) in _groups(crowded[k]).items():
        a, e = (T["a"], T["e"]) if k == 2 else (None, None)
        x, st = band.solve(a, T["b"], T["c"], T["d"], e, T["f"], method=method,
                           schedule=schedule, chunks=chunks)
        torch.cuda.synchronize()
        _tally(total, _classify(x.cpu().numpy(), st.cpu().numpy(), group, k))
    assert total["nonsingular"] >= 100 and total["singular"] >= 100
    assert total["range"] <= total["nonsingular"] // 100, total
    assert total["singular_range"] <= total["singular"] // 100, total


def test_crowded_zero_pivots_batched(band, crowded):
    """Every size group of both bandwidths as one band_solve_batch launch (the batched
    symbolic fix-up serves all problems' flagged systems at once)."""
    specs = []
    for k in (1, 2):
        for n, (T, group) in _groups(crowded[k]).items():
            specs.append((k, T, group))
    assert len(specs) <= 64
    plan = band.BatchPlan([dict(op="solve", method="spdm" if k == 2 else "stdm",
                                a=T["a"] if k == 2 else None, b=T["b"], c=T["c"], d=T["d"],
                                e=T["e"] if k == 2 else None, f=T["f"])
                           for k, T, group in specs])
    outs = plan.run()
    torch.cuda.synchronize()
    total = {}
    for (k, T, group), res in zip(specs, outs):
        _tally(total, _classify(res["x"].cpu().numpy(), res["status"].cpu().numpy(), group, k))
    assert total["range"] <= total["nonsingular"] // 100, total
    assert total["singular_range"] <= total["singular"] // 100, total


@pytest.mark.parametrize("k", [1, 2])
def test_crowded_determinants(band, crowded, k):
    """band_det against the exact determinant: SINGULAR exactly where it is 0, else the
    exact value to the rounding of the pivot product."""
    total = dict(range=0, nonsingular=0)
    for n, (T, group) in _groups(crowded[k]).items():
        mant, ex, st = band.det(T["a"], T["b"], T["c"], T["d"], T["e"], half_bw=k)
        torch.cuda.synchronize()
        mant, ex, st = mant.cpu().numpy(), ex.cpu().numpy(), st.cpu().numpy()
        for j, sy in enumerate(group):
            if sy["status"] == "SINGULAR":
                assert st[j] in (SINGULAR, RANGE) and mant[j] == 0.0, (sy, st[j])
                total["singular_range"] = total.get("singular_range", 0) + (st[j] == RANGE)
                total["singular"] = total.get("singular", 0) + 1
                continue
            total["nonsingular"] += 1
            if st[j] == RANGE:
                total["range"] += 1
                continue
            assert st[j] == OK, (sy, st[j])
            got = mant[j] * 2.0 ** int(ex[j])
            assert abs(got - sy["det"]) <= 1e-9 * abs(sy["det"]), (sy, got)
    assert total["range"] <= total["nonsingular"] // 100, total
    assert total.get("singular_range", 0) <= total.get("singular", 0) // 100, total


def _planted_adi(r, k, nsys, frac, seed):
    """ADI rows (n = 2048) with an exact zero pivot planted in a fraction of the
    systems: row j gets a_j = b_j = c_j = 0, so gamma_j = 0 and mu_j = c_j = 0 in any
    arithmetic.  f = A x_true is recomputed for the planted matrices."""
    B = synth.cfg1(r=r, k=k, sweep="y", grid=2048, nsys=nsys)
    n = B["n"]
    rng = np.random.default_rng(seed)
    D = {q: B[q].reshape(n, nsys).copy() for q in "abcde"}
    planted = rng.choice(nsys, size=max(1, int(round(frac * nsys))), replace=False)
    rows = rng.integers(4, n - 4, size=len(planted))
    for s, j in zip(planted, rows):
        D["a"][j, s] = 0.0
        D["b"][j, s] = 0.0
        D["c"][j, s] = 0.0
    xt = B["x_true"].reshape(n, nsys)
    f = synth.band_matvec(k, D["a"], D["b"], D["c"], D["d"], D["e"], xt)
    return D, f, xt, planted, rows


@pytest.mark.parametrize("k,r", [(2, 2.0), (2, 10.0), (1, 2.0)])
def test_planted_zero_pivots_full_length(band, k, r):
    """Long systems (n = 2048, the ADI workload's lines) with one exact zero pivot in 10 %
    of them: the planted systems go through the series pass (dense series from the zero
    row to the end), the others through the numeric sweep.  Against the oracle's SPDM /
    STDM and the GEPP truth, sampled systems; every status OK."""
    nsys = 64
    D, f, xt, planted, rows = _planted_adi(r, k, nsys, 0.1, seed=int(10 * r) + k)
    n = D["c"].shape[0]
    T = {q: torch.tensor(D[q], device=DEV) for q in "abcde"}
    Tf = torch.tensor(f, device=DEV)
    method = "spdm" if k == 2 else "stdm"
    a, e = (T["a"], T["e"]) if k == 2 else (None, None)
    for schedule in ("thread", "two_sided"):
        x, st = band.solve(a, T["b"], T["c"], T["d"], e, Tf, method=method, schedule=schedule)
        torch.cuda.synchronize()
        st = st.cpu().numpy()
        assert (st == OK).all(), (schedule, st)
        xg = x.cpu().numpy()
        check = list(planted) + [s for s in range(nsys) if s not in set(planted)][:6]
        for s in check:
            args = [D[q][:, s] for q in "abcde"] + [f[:, s]]
            xo, so, _, _, nf = oracle.symbolic(k, *args)
            assert so == "OK"
            if s in set(planted) and schedule == "thread":
                assert nf >= 1
            xg_s = xg[:, s]
            den = np.abs(xo).max()
            assert np.abs(xg_s - xo).max() <= 1e-10 * den, (schedule, s)
            xr, sr, _ = oracle.gepp_band(k, *args)
            assert np.abs(xg_s - xr).max() <= 1e-10 * np.abs(xr).max(), (schedule, s)
    # the determinant of the same systems: planted ones from the series pass
    mant, ex, st = band.det(T["a"], T["b"], T["c"], T["d"], T["e"], half_bw=k)
    torch.cuda.synchronize()
    mant, ex, st = mant.cpu().numpy(), ex.cpu().numpy(), st.cpu().numpy()
    assert (st == OK).all()
    for s in list(planted)[:4] + [s for s in range(nsys) if s not in set(planted)][:4]:
        args = [D[q][:, s] for q in "abcde"] + [f[:, s]]
        _, _, dm, dex, _ = oracle.symbolic(k, *args)
        # compare log2|det| and the sign
        lg = np.log2(abs(mant[s])) + ex[s]
        lo = np.log2(abs(dm)) + dex
        assert np.sign(mant[s]) == np.sign(dm)
        assert abs(lg - lo) <= 1e-9 * max(1.0, abs(lo)), (s, lg, lo)


def test_determinant_dominant_batch(band):
    """band_det on the small plain-NPDM workload's systems (1024 x 128) against the
    oracle's pivot product, and against numpy's slogdet of the dense matrix on a few."""
    B = synth.cfg0()
    n, ns = B["n"], B["nsys"]
    T = {q: torch.tensor(B[q].reshape(n, ns), device=DEV) for q in "abcde"}
    mant, ex, st = band.det(T["a"], T["b"], T["c"], T["d"], T["e"])
    sign, logabs, st2 = band.slogdet(T["a"], T["b"], T["c"], T["d"], T["e"])
    torch.cuda.synchronize()
    assert (st.cpu() == OK).all() and (st2.cpu() == OK).all()
    mant, ex = mant.cpu().numpy(), ex.cpu().numpy()
    sign, logabs = sign.cpu().numpy(), logabs.cpu().numpy()
    for s in range(0, ns, 97):
        S = synth.system(B, s)
        _, so, dm, dex, _ = oracle.symbolic(2, *[S[q] for q in "abcdef"])
        assert so == "OK"
        assert np.sign(mant[s]) == np.sign(dm)
        assert abs(np.log2(abs(mant[s])) + ex[s] - (np.log2(abs(dm)) + dex)) <= 1e-12 * 128
        A = exact.dense(2, *[S[q] for q in "abcde"])
        sd, ld = np.linalg.slogdet(np.array(A, dtype=float))
        assert sign[s] == sd and abs(logabs[s] - ld) <= 1e-11 * max(1.0, abs(ld))


def test_fixup_slots_follow_the_workspace(band):
    """More flagged systems (256) than the stated workspace's fix-up slots (152): the
    warps loop over them; a workspace with room for 256 slots runs them all at once.
    Both give the same bits."""
    import ctypes as ct
    from paper_1804_09666_gb300 import _lib as L
    nsys, k = 256, 2
    D, f, xt, planted, rows = _planted_adi(2.0, k, nsys, 1.0, seed=5)
    n = D["c"].shape[0]
    T = {q: torch.tensor(D[q], device=DEV) for q in "abcde"}
    Tf = torch.tensor(f, device=DEV)
    lib = L.load()
    desc = band.desc_for(T["c"], 2, "thread")
    need = lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE, L.SPDM, 0)
    x1, s1 = band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], Tf, method="spdm",
                        schedule="thread")
    big = torch.empty(need + (nsys - 152) * 1584 * n, dtype=torch.uint8, device=DEV)
    x2, s2 = band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], Tf, method="spdm",
                        schedule="thread", ws=big)
    torch.cuda.synchronize()
    assert (s1.cpu() == OK).all() and (s2.cpu() == OK).all()
    assert torch.equal(x1, x2)
    for s in planted[:3]:
        xr, sr, _ = oracle.gepp_band(k, *[D[q][:, s] for q in "abcde"], f[:, s])
        assert np.abs(x1.cpu().numpy()[:, s] - xr).max() <= 1e-10 * np.abs(xr).max()
