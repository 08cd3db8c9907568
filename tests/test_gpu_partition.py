"""GPU parity of the partitioned schedule (P lanes per system, each eliminating one
chunk of rows with NPDM's recurrence while carrying the coupling columns; a
block-tridiagonal interface system over the chunks' boundary rows; a second
back-substitution) against the CPU oracle.

The partition is a reordering of Gaussian elimination without pivoting, so, like the
two-sided schedule, it is held to the oracle's bounds against the exact or GEPP
solution: 1e-12 on dominant systems, and on the non-dominant ADI systems 1e-10 (PD) /
1e-12 (TD) or 10x the oracle's own distance from GEPP, whichever is larger.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import flat_of, per_system_rel, to_dev

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PARTS = [4, 8, 16, 32]              # lanes of one warp
BLOCK_PARTS = [64, 128, 256]        # a block of 2, 4, 8 warps per system


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _solve(band, T, k, chunks, method=None, **kw):
    a, e = (T["a"], T["e"]) if k == 2 else (None, None)
    method = method or ("npdm" if k == 2 else "ntdm")
    x, st = band.solve(a, T["b"], T["c"], T["d"], e, T["f"], method=method,
                       schedule="partitioned", chunks=chunks, **kw)
    torch.cuda.synchronize()
    return x, st.cpu().numpy()


def _oracle(B, k, method="direct"):
    return oracle.batch(method, k, [B[q] for q in "abcde"], B["f"], B["nsys"], B["n"],
                        B["sys_stride"], B["elem_stride"])


def _args(B):
    return B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]


# n below 8 P (one lane solves the system), exactly 8 P, chunk lengths with every
# remainder pattern, and a long case; 37 systems leave a partial warp for every P.
@pytest.mark.parametrize("n", [5, 31, 32, 33, 64, 127, 256, 257, 300, 1000, 2048, 4099])
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("P", PARTS + BLOCK_PARTS)
def test_partition_dominant(band, n, k, P):
    B = synth.cfg0(nsys=37, n=n, k=k, seed_salt=61)
    x, st = _solve(band, to_dev(B), k, P)
    assert (st == 0).all(), st
    xo, so, _, _ = _oracle(B, k)
    assert (so == 0).all()
    xg = flat_of(x)
    assert per_system_rel(xg, xo, *_args(B)).max() <= 1e-12
    assert per_system_rel(xg, B["x_true"], *_args(B)).max() <= 1e-12


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("P", BLOCK_PARTS)
def test_partition_block_long(band, k, P):
    """A few long systems on a block of warps each (chunks of ~80 .. 320 rows, ragged
    chunk lengths)."""
    B = synth.cfg0(nsys=5, n=20481, k=k, seed_salt=74)
    x, st = _solve(band, to_dev(B), k, P)
    assert (st == 0).all(), st
    xo, _, _, _ = _oracle(B, k)
    assert per_system_rel(flat_of(x), xo, *_args(B)).max() <= 1e-12
    assert per_system_rel(flat_of(x), B["x_true"], *_args(B)).max() <= 1e-12


@pytest.mark.parametrize("layout", ["contiguous", "general"])
@pytest.mark.parametrize("k", [1, 2])
def test_partition_layouts(band, layout, k):
    n, nsys = 333, 45
    if layout == "contiguous":
        B = synth.cfg0(nsys=nsys, n=n, k=k, layout="contiguous", seed_salt=62)
    else:
        ss, es = 3, 3 * nsys + 7
        base = synth.cfg0(nsys=nsys, n=n, k=k, seed_salt=62)
        idx = np.arange(nsys)[None, :] * ss + np.arange(n)[:, None] * es
        B = dict(n=n, nsys=nsys, sys_stride=ss, elem_stride=es)
        for q in "abcdef":
            flat = np.full(int(idx.max()) + 1, np.nan)
            flat[idx] = base[q].reshape(n, nsys)
            B[q] = flat
    xo, _, _, _ = _oracle(B, k)
    for P in (8, 32, 64):
        x, st = _solve(band, to_dev(B), k, P)
        assert (st == 0).all()
        assert per_system_rel(flat_of(x), xo, *_args(B)).max() <= 1e-12


@pytest.mark.parametrize("r", synth.ADI_R)
def test_partition_adi_nondominant(band, r):
    """The ADI systems of the benchmark (n = 2048, both sweeps), PD and TD.

    At r = 2 the PD matrices are indefinite (c ~ -4 against off-diagonal sums ~ 5.7); a
    chunk restarting the recurrence can meet pivots far smaller than NPDM's, and without
    the pivot guard a plain FP64 emulation of the elimination gives errors up to 8e-10
    there against NPDM's 1.3e-12.  With the guard (such systems are redone by NPDM) every
    case is held to NPDM's bounds."""
    for sweep in ("x", "y"):
        for k in (2, 1):
            B = synth.cfg1(r=r, k=k, sweep=sweep, grid=2048, nsys=40)
            xo, _, _, _ = _oracle(B, k)
            xt, _, _, _ = _oracle(B, k, "gepp")
            err_o = per_system_rel(xo, xt, *_args(B))
            tol = 1e-10 if k == 2 else 1e-12
            bound = np.maximum(tol, 10 * err_o)
            for P in (8, 16, 32, 128):
                x, st = _solve(band, to_dev(B), k, P)
                assert (st == 0).all(), (sweep, k, P, st)
                err = per_system_rel(flat_of(x), xt, *_args(B))
                assert (err <= bound).all(), (sweep, k, P, err.max())


def _biased_exponent(v):
    """IEEE binary64 biased exponent of |v| (0 for zero), as the guard compares them."""
    mant, e = np.frexp(np.abs(v))
    return np.where(v == 0, 0, e + 1022)


def _chunk_guard_trips(B, P, tiny=17):
    """Systems (PD) whose chunk sweep meets a pivot the partitioned schedule's guard
    treats as zero: a pivot whose binary exponent lies `tiny` or more below that of the
    largest entry of its row (chunk k of P restarts NPDM's recurrence at its first row,
    rows [k L0 + min(k, r), ...) with n = L0 P + r).  A plain numpy model of that one
    decision, all chunks of all systems at once; it shares nothing with the kernels."""
    n, ns = B["n"], B["nsys"]
    idx = np.arange(ns)[None, :] * B["sys_stride"] + np.arange(n)[:, None] * B["elem_stride"]
    A = {q: B[q][idx] for q in "abcde"}                     # [row, system]
    L0, rem = divmod(n, P)
    ks = np.arange(P)
    Ls = (L0 + (ks < rem))[:, None]                         # [chunk, 1]
    s0 = (ks * L0 + np.minimum(ks, rem))[:, None]
    al1, al2, be1, be2 = (np.zeros((P, ns)) for _ in range(4))
    trip = np.zeros((P, ns), bool)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for j in range(int(Ls.max())):
            live = j < Ls
            i = np.minimum(s0 + j, n - 1)[:, 0]
            ag = np.where((i >= 2)[:, None], A["a"][i], 0.0)
            bg = np.where((i >= 1)[:, None], A["b"][i], 0.0)
            dg = np.where((i + 1 < n)[:, None], A["d"][i], 0.0)
            eg = np.where((i + 2 < n)[:, None], A["e"][i], 0.0)
            cc = A["c"][i]
            aa = ag if j >= 2 else np.zeros_like(ag)
            bb = bg if j >= 1 else np.zeros_like(bg)
            dd = np.where(j + 1 < Ls, dg, 0.0)
            ee = np.where(j + 2 < Ls, eg, 0.0)
            g = bb - al2 * aa
            m = cc - be2 * aa - al1 * g
            ex = np.maximum.reduce([_biased_exponent(v) for v in (cc, bg, dg, ag, eg)])
            trip |= live & ((m == 0) | (_biased_exponent(m) + tiny <= ex))
            alv, bev = (dd - be1 * g) / m, ee / m
            al2, al1 = np.where(live, al1, al2), np.where(live, alv, al1)
            be2, be1 = np.where(live, be1, be2), np.where(live, bev, be1)
    return np.flatnonzero(trip.any(0)).tolist()


@pytest.mark.parametrize("sweep", ["x", "y"])
def test_partition_redoes_exactly_the_tripped_systems(band, sweep):
    """On the indefinite r = 2 PD ADI rows the pivot guard sends some systems back to
    NPDM in one lane (bitwise the thread schedule's result) and leaves every other
    system of the warp partitioned: the redone set is exactly the systems whose chunk
    sweep trips the guard in a plain numpy model of it.  (The interface's guards do not
    trip on these inputs.)  A group's failure that leaked into the warp's other groups,
    as a skipped warp vote once did, redoes whole warps and fails this test."""
    B = synth.cfg1(r=2.0, k=2, sweep=sweep, grid=2048, nsys=40)
    T = to_dev(B)
    x1, _ = band.solve(*(T[q] for q in "abcdef"), method="npdm", schedule="thread")
    xt, _, _, _ = _oracle(B, 2, "gepp")
    xo, _, _, _ = _oracle(B, 2)
    bound = np.maximum(1e-10, 10 * per_system_rel(xo, xt, *_args(B)))
    tripped_any = False
    for P in PARTS:
        want = _chunk_guard_trips(B, P)
        tripped_any |= bool(want)
        x, st = _solve(band, T, 2, P)
        assert (st == 0).all(), (sweep, P)
        redone = [s for s in range(B["nsys"]) if torch.equal(x[:, s], x1[:, s])]
        assert redone == want, (sweep, P, redone, want)
        assert (per_system_rel(flat_of(x), xt, *_args(B)) <= bound).all(), (sweep, P)
    assert tripped_any


@pytest.mark.parametrize("k", [1, 2])
def test_partition_fp32(band, k):
    """FP32 data: within a factor of 4 (or 1e-6) of one thread per system's distance
    from the exact solution of the FP32 system."""
    n, nsys = 1000, 50
    B = synth.cfg0(nsys=nsys, n=n, k=k, seed_salt=63)
    B32 = dict(B)
    for q in "abcdef":
        B32[q] = B[q].astype(np.float32).astype(np.float64)
    T = to_dev(B32, dtype=torch.float32)
    xo, _, _, _ = _oracle(B32, k)
    x1, st1 = band.solve(T["a"] if k == 2 else None, T["b"], T["c"], T["d"],
                         T["e"] if k == 2 else None, T["f"],
                         method="npdm" if k == 2 else "ntdm", schedule="thread")
    torch.cuda.synchronize()
    e1 = per_system_rel(flat_of(x1).astype(np.float64), xo, *_args(B))
    for P in PARTS + [64]:
        x, st = _solve(band, T, k, P)
        assert (st == 0).all()
        e = per_system_rel(flat_of(x).astype(np.float64), xo, *_args(B))
        assert (e <= np.maximum(4 * e1, 1e-6)).all(), (P, e.max(), e1.max())


def test_partition_x_aliases_f(band):
    B = synth.cfg0(nsys=21, n=500, seed_salt=64)
    T = to_dev(B)
    xo, _, _, _ = _oracle(B, 2)
    f0 = T["f"].clone()
    _solve(band, T, 2, 16, x=T["f"])
    assert per_system_rel(flat_of(T["f"]), xo, *_args(B)).max() <= 1e-12
    T["f"].copy_(f0)
    _solve(band, T, 2, 64, x=T["f"])
    assert per_system_rel(flat_of(T["f"]), xo, *_args(B)).max() <= 1e-12


def test_partition_nonfinite_inputs(band):
    n, nsys = 512, 12
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=65)
    xo, _, _, _ = _oracle(B, 2)
    C = dict(B)
    f = B["f"].copy().reshape(n, nsys)
    c = B["c"].copy().reshape(n, nsys)
    f[3, 2] = np.nan        # first chunk
    f[300, 7] = np.inf      # a middle chunk
    c[511, 9] = np.nan      # last row
    C["f"], C["c"] = f.reshape(-1), c.reshape(-1)
    x, st = _solve(band, to_dev(C), 2, 8)
    hit = np.zeros(nsys, bool)
    hit[[2, 7, 9]] = True
    assert (st[hit] == 5).all(), st
    assert (st[~hit] == 0).all()
    assert per_system_rel(flat_of(x), xo, *_args(B))[~hit].max() <= 1e-12


def test_partition_chunk_zero_pivot(band):
    """c = 0 in the first row of chunk 1 (P = 8, n = 200: rows 25 ..): the chunk's own
    first pivot is exactly 0, while NPDM's pivot there (c minus the fill from the rows
    above) is not.  The system is redone by its first lane with NPDM and comes back OK
    with NPDM's solution; SPDM sends it to the fix-up, which solves it too."""
    n, nsys = 200, 24
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=66)
    B["c"].reshape(n, nsys)[25, 0:8] = 0.0
    B["c"].reshape(n, nsys)[30, 8:16] = 0.0      # inside a chunk: no zero pivot there
    T = to_dev(B)
    xo, so, _, _ = _oracle(B, 2)
    xt, _, _, _ = _oracle(B, 2, "gepp")
    assert (so == 0).all()
    err_o = per_system_rel(xo, xt, *_args(B))
    bound = np.maximum(1e-12, 10 * err_o)
    for method in ("npdm", "spdm"):
        x, st = _solve(band, T, 2, 8, method=method)
        assert (st == 0).all(), (method, st)
        err = per_system_rel(flat_of(x), xt, *_args(B))
        assert (err <= bound).all(), (method, err.max())
    # the redone systems (0..7) carry NPDM's own rounding: bitwise the thread schedule's
    x, _ = _solve(band, T, 2, 8)
    x1, _ = band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], T["f"], method="npdm",
                       schedule="thread")
    torch.cuda.synchronize()
    assert torch.equal(x[:, 0:8], x1[:, 0:8])
    assert not torch.equal(x[:, 16:], x1[:, 16:])


def test_partition_block_chunk_zero_pivot(band):
    """The same on a block of two warps (P = 64, n = 1280: chunk 1 starts at row 20):
    the first thread redoes the system with NPDM (bitwise the thread schedule's)."""
    n, nsys = 1280, 12
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=75)
    B["c"].reshape(n, nsys)[20, 0:4] = 0.0
    T = to_dev(B)
    xt, _, _, _ = _oracle(B, 2, "gepp")
    xo, so, _, _ = _oracle(B, 2)
    assert (so == 0).all()
    bound = np.maximum(1e-12, 10 * per_system_rel(xo, xt, *_args(B)))
    for method in ("npdm", "spdm"):
        x, st = _solve(band, T, 2, 64, method=method)
        assert (st == 0).all(), (method, st)
        assert (per_system_rel(flat_of(x), xt, *_args(B)) <= bound).all()
    x, _ = _solve(band, T, 2, 64)
    x1, _ = band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], T["f"], method="npdm",
                       schedule="thread")
    torch.cuda.synchronize()
    assert torch.equal(x[:, 0:4], x1[:, 0:4])


def test_partition_planted_npdm_zero_pivots(band):
    """a_i = b_i = c_i = 0 (and a_{i+2} = 0) in one row: NPDM's pivot there is exactly 0
    whatever came before.  NPDM on the partitioned schedule still reports ZERO_PIVOT
    (the first lane's redo meets it); SPDM solves the systems through the fix-up."""
    n, nsys = 600, 16
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=67)
    for i, sl in ((20, slice(0, 8)), (333, slice(8, 16))):
        for q, r in (("a", i), ("b", i), ("c", i), ("a", i + 2)):
            B[q].reshape(n, nsys)[r, sl] = 0.0
    T = to_dev(B)
    xt, _, _, _ = _oracle(B, 2, "gepp")
    xs, ss, _, _ = _oracle(B, 2, "symbolic")
    assert (ss == 0).all()
    bound = np.maximum(1e-12, 10 * per_system_rel(xs, xt, *_args(B)))
    for P in (8, 32, 64):
        _, st = _solve(band, T, 2, P)
        assert (st == 3).all(), (P, st)
        x, st = _solve(band, T, 2, P, method="spdm")
        assert (st == 0).all(), (P, st)
        assert (per_system_rel(flat_of(x), xt, *_args(B)) <= bound).all()


def _golden():
    return json.load(open(os.path.join(GOLD, "zero_pivot_cases.json")))["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_partition_golden_zero_pivots(band, case):
    """The hand-made zero-pivot systems (short: one lane runs NPDM / the fix-up)."""
    k, n = case["k"], case["n"]
    fl = lambda key: np.array([float(Fraction(v)) for v in case[key]])
    nsys = 9
    B = dict(n=n, nsys=nsys, sys_stride=1, elem_stride=nsys)
    for q in "abcdef":
        B[q] = np.repeat(fl(q)[:, None], nsys, axis=1).reshape(-1)
    T = to_dev(B)
    _, st = _solve(band, T, k, 8)
    _, st1 = band.solve(T["a"] if k == 2 else None, T["b"], T["c"], T["d"],
                        T["e"] if k == 2 else None, T["f"], method="npdm" if k == 2 else "ntdm",
                        schedule="thread")
    torch.cuda.synchronize()
    assert (st == st1.cpu().numpy()).all()
    x, st = _solve(band, T, k, 8, method="spdm" if k == 2 else "stdm")
    if case["status"] == "SINGULAR":
        assert (st == 4).all(), st
        return
    assert (st == 0).all(), st
    want = fl("x")
    xg = flat_of(x).reshape(n, nsys)
    assert np.abs(xg - want[:, None]).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_partition_auto_chunks(band):
    """chunks = 0: the library picks P from nsys and n; the result is one of the fixed-P
    results bitwise."""
    B = synth.cfg0(nsys=30, n=2048, seed_salt=68)
    T = to_dev(B)
    x0, st = _solve(band, T, 2, 0)
    assert (st == 0).all()
    assert any(torch.equal(x0, _solve(band, T, 2, P)[0]) for P in PARTS + BLOCK_PARTS)


def test_partition_in_batch_equals_single(band):
    """band_solve_batch runs the same partitioned sweep (bitwise), beside two-sided,
    thread-per-system and SIP problems in the same launch."""
    P1 = to_dev(synth.cfg0(nsys=37, n=1000, seed_salt=69))
    P2 = to_dev(synth.cfg0(nsys=50, n=300, k=1, layout="contiguous", seed_salt=70))
    P3 = to_dev(synth.cfg0(nsys=11, n=777, seed_salt=71), dtype=torch.float32)
    S = to_dev(synth.cfg1(r=2.0, k=2, sweep="y", grid=512, nsys=64))
    specs = [
        dict(method="npdm", schedule="partitioned", chunks=32, **{q: P1[q] for q in "abcdef"}),
        dict(method="ntdm", schedule="partitioned", chunks=8, a=None, e=None,
             **{q: P2[q] for q in "bcdf"}),
        dict(method="npdm", schedule="partitioned", chunks=8, **{q: P3[q] for q in "abcdef"}),
        dict(method="npdm", schedule="two_sided", **{q: P1[q] for q in "abcdef"}),
        dict(op="sip", tol=1e-10, max_it=200, **{q: S[q] for q in "abcdef"}),
        dict(method="npdm", schedule="partitioned", chunks=128, **{q: P1[q] for q in "abcdef"}),
    ]
    res = band.BatchPlan(specs).run()
    torch.cuda.synchronize()
    for sp, r in zip(specs[:3], res[:3]):
        k = 1 if sp["method"] == "ntdm" else 2
        x, st = _solve(band, {q: sp[q] for q in "abcdef"}, k, sp["chunks"])
        assert torch.equal(r["x"], x)
        assert (r["status"].cpu().numpy() == st).all()
        assert (st == 0).all()
    assert torch.allclose(res[0]["x"], res[3]["x"], rtol=0, atol=1e-12)
    assert (res[4]["status"].cpu().numpy() == 0).all()
    # a batched task is one warp: 128 chunks run as 32
    assert torch.equal(res[5]["x"], res[0]["x"])


def test_partition_ragged_buckets(band):
    """A ragged packing (n in [16, 3000], TD and PD) as size buckets on the partitioned
    schedule (buckets whose systems are too short for their chunks fall back to one lane)
    against the oracle, system by system."""
    B = synth.cfg2(nsys=300, nmin=16, nmax=3000, seed_salt=72)
    d = {q: torch.from_numpy(B[q]).to("cuda") for q in "abcdef"}
    offs = B["offsets"]
    ref = []
    for s in range(B["nsys"]):
        S = synth.system(B, s)
        xo, _ = (oracle.ntdm(S["b"], S["c"], S["d"], S["f"]) if B["hbw"][s] == 1
                 else oracle.npdm(*(S[q] for q in "abcdef")))
        ref.append(xo)
    for chunks in (0, 8, 32):
        plan = band.RaggedPlan(*(d[q] for q in "abcdef"), offs, B["hbw"],
                               schedule="partitioned", chunks=chunks)
        x, st = plan.run()
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        xg = x.cpu().numpy()
        for s, xo in enumerate(ref):
            lo, hi = int(offs[s]), int(offs[s + 1])
            rel = np.abs(xg[lo:hi] - xo).max() / np.abs(xo).max()
            assert rel <= 1e-12, (chunks, s, rel)


def test_autotune_joint(band):
    """The joint tuner's choice per bucket is a valid schedule, and the tuned plan
    solves the packing."""
    from paper_1804_09666_gb300 import _lib as L
    B = synth.cfg2(nsys=2000, nmin=16, nmax=4096, seed_salt=73)
    d = {q: torch.from_numpy(B[q]).to("cuda") for q in "abcdef"}
    L.load().band_autotune_reset()
    plan = band.RaggedPlan(*(d[q] for q in "abcdef"), B["offsets"], B["hbw"], schedule="tune")
    for sch, ch in zip(plan.schedules, plan.chunks):
        assert sch in (1, 2, 3)
        assert (sch == 3) == (ch in (8, 16, 32))
    x, st = plan.run()
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    err = np.maximum.reduceat(np.abs(x.cpu().numpy() - B["x_true"]), B["offsets"][:-1])
    assert err.max() <= 1e-11


def _packed(B):
    """A uniform batch repacked as a ragged packing (system after system)."""
    n, ns, ss, es = B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]
    idx = np.arange(ns)[:, None] * ss + np.arange(n)[None, :] * es     # [system, row]
    packed = {q: np.ascontiguousarray(B[q][idx].reshape(-1)) for q in "abcdef"}
    offsets = np.arange(ns + 1, dtype=np.int64) * n
    return packed, offsets


def test_autotune_joint_dominance_gate(band):
    """64 systems of n = 2048 fill a twentieth of the GPU: the joint tuner moves a
    diagonally dominant bucket to the partitioned schedule, and never a non-dominant one
    (the ADI rows at r = 2), whose chunks may be far worse conditioned than the matrix."""
    from paper_1804_09666_gb300 import _lib as L
    cases = [("dominant", synth.cfg0(nsys=64, n=2048, seed_salt=76), True),
             ("adi r=2", synth.cfg1(r=2.0, k=2, sweep="y", grid=2048, nsys=64), False)]
    for name, B, may_partition in cases:
        packed, offs = _packed(B)
        d = {q: torch.from_numpy(packed[q]).to("cuda") for q in "abcdef"}
        L.load().band_autotune_reset()
        plan = band.RaggedPlan(*(d[q] for q in "abcdef"), offs, np.full(64, 2, np.int8),
                               schedule="tune")
        if may_partition:
            assert 3 in plan.schedules, (name, plan.schedules)
        else:
            assert 3 not in plan.schedules, (name, plan.schedules)
        x, st = plan.run()
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()


@pytest.mark.parametrize("chunks", [8, 64])
def test_refine_and_adjoint_on_the_partitioned_schedule(band, chunks):
    """The refinement's FP32 correction solves and the adjoint's transposed solve run on
    the descriptor's schedule: partitioned, they reach the same bounds as the default."""
    # refinement: FP32 storage, FP64 result within 1e-10 of the FP64 truth
    rng = np.random.default_rng(77)
    nsys, n = 40, 1024
    D = synth.dominant(rng, nsys, n, k=2, dtype=np.float32, ratio=1.1)
    xt, f = synth.manufactured(rng, 2, D, nsys, n)
    B = synth.batch(D, f, 2, nsys, n)
    T = to_dev(B, keys="abcde", dtype=torch.float32)
    fd = to_dev(B, keys="f")["f"]
    x, steps, st = band.refine_solve(*(T[q] for q in "abcde"), fd, schedule="partitioned",
                                     chunks=chunks)
    torch.cuda.synchronize()
    assert (st.cpu() == 0).all()
    xtruth, _, _, _ = oracle.batch("gepp", 2, [B[q].astype(np.float64) for q in "abcde"], B["f"],
                                   nsys, n, B["sys_stride"], B["elem_stride"])
    assert per_system_rel(flat_of(x), xtruth, *_args(B)).max() <= 1e-10
    # adjoint: against the default schedule's gradients and the oracle's
    C = synth.cfg4(nsys=nsys, n=n)
    Tc = to_dev(C, keys="abcdefw")
    xs, _ = band.solve(*(Tc[q] for q in "abcdef"), method="npdm")
    g_def, gf_def, _ = band.adjoint(*(Tc[q] for q in "abcde"), xs, Tc["w"])
    g_par, gf_par, stp = band.adjoint(*(Tc[q] for q in "abcde"), xs, Tc["w"],
                                      schedule="partitioned", chunks=chunks)
    torch.cuda.synchronize()
    assert (stp.cpu() == 0).all()
    for g1, g2 in list(zip(g_par, g_def)) + [(gf_par, gf_def)]:
        den = g2.abs().amax(0).clamp_min(1e-300)
        assert ((g1 - g2).abs().amax(0) / den).max().item() <= 1e-12
    S = synth.system(C, 3)
    go, gfo, sto = oracle.adjoint(2, *(S[q] for q in "abcde"), xs.cpu().numpy()[:, 3],
                                  C["w"].reshape(n, nsys)[:, 3])
    assert sto == "OK"
    assert np.abs(gf_par.cpu().numpy()[:, 3] - gfo).max() / np.abs(gfo).max() <= 1e-11


def test_batchplan_tune(band):
    """BatchPlan(tune=True): the joint tuner partitions the dominant problem whose few
    long systems bound the launch, keeps the non-dominant ADI problem off the
    partitioned schedule, and the tuned plan solves both (GEPP-bounded for the ADI
    rows)."""
    D = synth.cfg0(nsys=64, n=8192, seed_salt=78)
    A = synth.cfg1(r=2.0, k=2, sweep="x", grid=2048, nsys=256)
    TD, TA = to_dev(D), to_dev(A)
    specs = [dict(method="npdm", **{q: TD[q] for q in "abcdef"}),
             dict(method="npdm", **{q: TA[q] for q in "abcdef"})]
    plan = band.BatchPlan(specs, tune=True)
    assert plan.schedules[0] == 3 and plan.chunks[0] in (8, 16, 32), plan.schedules
    assert plan.schedules[1] in (1, 2), plan.schedules
    res = plan.run()
    torch.cuda.synchronize()
    for r in res:
        assert (r["status"].cpu().numpy() == 0).all()
    xo, _, _, _ = _oracle(D, 2)
    assert per_system_rel(flat_of(res[0]["x"]), xo, *_args(D)).max() <= 1e-12
    xo, _, _, _ = _oracle(A, 2)
    xt, _, _, _ = _oracle(A, 2, "gepp")
    bound = np.maximum(1e-10, 10 * per_system_rel(xo, xt, *_args(A)))
    assert (per_system_rel(flat_of(res[1]["x"]), xt, *_args(A)) <= bound).all()


def test_four_chunks_single_calls_only(band):
    """P = 4 runs in band_solve (parity above); band_solve_batch rejects it (its code in
    the batched kernel would cost every other task registers)."""
    from paper_1804_09666_gb300 import _lib as L
    T = to_dev(synth.cfg0(nsys=64, n=512, seed_salt=91))
    spec = dict(method="npdm", schedule="partitioned", chunks=4, **{q: T[q] for q in "abcdef"})
    with pytest.raises(L.BandError):
        band.BatchPlan([spec]).run()
