"""GPU parity of the two-sided schedule of the numeric direct solves (two threads per
system: NPDM's recurrence from the top, its mirror image from the bottom, a small
interface system in the middle) against the CPU oracle.

The two-sided elimination is a reordering of Gaussian elimination without pivoting, not
the oracle's order of operations, so it is held to the oracle's bounds against the
exact or GEPP solution: 1e-12 on dominant systems, and on the non-dominant ADI systems
1e-10 or 10x the oracle's own distance from GEPP, whichever is larger.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import DEV, flat_of, per_system_rel, strided_view, to_dev

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _solve(band, T, k, schedule, **kw):
    a, e = (T["a"], T["e"]) if k == 2 else (None, None)
    x, st = band.solve(a, T["b"], T["c"], T["d"], e, T["f"], method="npdm" if k == 2 else "ntdm",
                       schedule=schedule, **kw)
    torch.cuda.synchronize()
    return x, st.cpu().numpy()


def _oracle(B, k, method="direct"):
    return oracle.batch(method, k, [B[q] for q in "abcde"], B["f"], B["nsys"], B["n"],
                        B["sys_stride"], B["elem_stride"])


def _args(B):
    return B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]


# n = 1..9 covers the one-thread fallback (n < 4 PD, n < 2 TD) and both parities of n
# around the smallest split; 31..33 and 257 span several staging blocks with ragged ends.
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 31, 32, 33, 257])
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("layout", ["interleaved", "contiguous"])
def test_two_sided_dominant(band, n, k, layout):
    """37 systems: two full 16-system warps and a tail of 5."""
    B = synth.cfg0(nsys=37, n=n, k=k, layout=layout, seed_salt=21)
    x, st = _solve(band, to_dev(B), k, "two_sided")
    assert (st == 0).all()
    xo, so, _, _ = _oracle(B, k)
    assert (so == 0).all()
    xg = flat_of(x)
    assert per_system_rel(xg, xo, *_args(B)).max() <= 1e-12
    assert per_system_rel(xg, B["x_true"], *_args(B)).max() <= 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_two_sided_general_strides(band, k):
    """A padded, non-unit-stride layout (neither index contiguous)."""
    n, nsys, ss, es = 120, 50, 3, 3 * 50 + 7
    base = synth.cfg0(nsys=nsys, n=n, k=k, seed_salt=22)
    idx = np.arange(nsys)[None, :] * ss + np.arange(n)[:, None] * es
    size = int(idx.max()) + 1
    B = dict(n=n, nsys=nsys, sys_stride=ss, elem_stride=es)
    for q in "abcdef":
        flat = np.full(size, np.nan)
        flat[idx] = base[q].reshape(n, nsys)
        B[q] = flat
    x, st = _solve(band, to_dev(B), k, "two_sided")
    assert (st == 0).all()
    xo, _, _, _ = _oracle(B, k)
    assert per_system_rel(flat_of(x), xo, *_args(B)).max() <= 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_two_sided_fp32(band, k):
    """FP32 data: the two-sided result is as close to the exact solution of the FP32
    system (the oracle in FP64 on the same values) as one thread per system is, within
    a factor of 4 or one part in 1e6."""
    n, nsys = 257, 100
    B = synth.cfg0(nsys=nsys, n=n, k=k, seed_salt=23)
    B32 = dict(B)
    for q in "abcdef":
        B32[q] = B[q].astype(np.float32).astype(np.float64)
    T = to_dev(B32, dtype=torch.float32)
    xo, _, _, _ = _oracle(B32, k)
    x2, st2 = _solve(band, T, k, "two_sided")
    x1, st1 = _solve(band, T, k, "thread")
    assert (st1 == 0).all() and (st2 == 0).all()
    e2 = per_system_rel(flat_of(x2).astype(np.float64), xo, *_args(B))
    e1 = per_system_rel(flat_of(x1).astype(np.float64), xo, *_args(B))
    assert (e2 <= np.maximum(4 * e1, 1e-6)).all(), (e2.max(), e1.max())
    assert e2.max() <= 1e-5


@pytest.mark.parametrize("r", synth.ADI_R)
def test_two_sided_adi_nondominant(band, r):
    """The ADI systems, both sweeps, at the benchmark's n = 2048 (96 lines each)."""
    for sweep in ("x", "y"):
        for k in (2, 1):
            B = synth.cfg1(r=r, k=k, sweep=sweep, grid=2048, nsys=96)
            x, st = _solve(band, to_dev(B), k, "two_sided")
            assert (st == 0).all()
            xo, _, _, _ = _oracle(B, k)
            xt, _, _, _ = _oracle(B, k, "gepp")
            err_o = per_system_rel(xo, xt, *_args(B))
            err = per_system_rel(flat_of(x), xt, *_args(B))
            tol = 1e-10 if k == 2 else 1e-12
            assert (err <= np.maximum(tol, 10 * err_o)).all(), (sweep, k, err.max())


def test_two_sided_x_aliases_f(band):
    B = synth.cfg0(nsys=48, n=90, seed_salt=24)
    T = to_dev(B)
    x, st = _solve(band, T, 2, "two_sided", x=T["f"])
    assert (st == 0).all()
    xo, _, _, _ = _oracle(B, 2)
    assert per_system_rel(flat_of(T["f"]), xo, *_args(B)).max() <= 1e-12


def test_two_sided_nonfinite_inputs(band):
    """A NaN in f in the top half, in the bottom half, or on the diagonal: that system
    reports NONFINITE, the others are unaffected."""
    n, nsys = 64, 40
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=25)
    xo, _, _, _ = _oracle(B, 2)
    C = dict(B)
    f = B["f"].copy().reshape(n, nsys)
    c = B["c"].copy().reshape(n, nsys)
    f[3, 5] = np.nan
    f[60, 17] = np.nan
    c[40, 30] = np.nan
    C["f"], C["c"] = f.reshape(-1), c.reshape(-1)
    x, st = _solve(band, to_dev(C), 2, "two_sided")
    hit = np.zeros(nsys, bool)
    hit[[5, 17, 30]] = True
    assert (st[hit] == 5).all(), st
    assert (st[~hit] == 0).all()
    err = per_system_rel(flat_of(x), xo, *_args(B))
    assert err[~hit].max() <= 1e-12


def _golden():
    return json.load(open(os.path.join(GOLD, "zero_pivot_cases.json")))["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_two_sided_zero_pivots(band, case):
    """The hand-made zero-pivot systems.  A zero pivot met by either half makes the
    first thread redo the system with NPDM, which reports ZERO_PIVOT; pd_near_end has
    its zero pivot in NPDM's order below the middle, where the two-sided elimination
    meets none, and is solved exactly; singular systems never come back OK."""
    k, n = case["k"], case["n"]
    fl = lambda key: np.array([float(Fraction(v)) for v in case[key]])
    nsys = 20
    B = dict(n=n, nsys=nsys, sys_stride=1, elem_stride=nsys)
    for q in "abcdef":
        B[q] = np.repeat(fl(q)[:, None], nsys, axis=1).reshape(-1)
    x, st = _solve(band, to_dev(B), k, "two_sided")
    if case["status"] == "SINGULAR":
        assert (st != 0).all(), st
        return
    if case["name"] == "pd_near_end":
        assert (st == 0).all(), st
    assert np.isin(st, (0, 3)).all(), st
    if (st == 0).any():
        want = fl("x")
        xg = flat_of(x).reshape(n, nsys)[:, st == 0]
        assert np.abs(xg - want[:, None]).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_two_sided_in_batch_equals_single(band):
    """The batched kernel runs the same two-sided sweep (bitwise equal results), next
    to a thread-per-system problem and a SIP problem in the same launch."""
    P = to_dev(synth.cfg0(nsys=70, n=200, seed_salt=26))
    Tt = to_dev(synth.cfg0(nsys=33, n=150, k=1, layout="contiguous", seed_salt=27))
    P32 = to_dev(synth.cfg0(nsys=40, n=99, seed_salt=28), dtype=torch.float32)
    S = to_dev(synth.cfg1(r=2.0, k=2, sweep="y", grid=512, nsys=64))
    specs = [
        dict(method="npdm", schedule="two_sided", **{q: P[q] for q in "abcdef"}),
        dict(method="ntdm", schedule="two_sided", a=None, e=None, **{q: Tt[q] for q in "bcdf"}),
        dict(method="npdm", schedule="two_sided", **{q: P32[q] for q in "abcdef"}),
        dict(method="npdm", schedule="thread", **{q: P[q] for q in "abcdef"}),
        dict(op="sip", tol=1e-10, max_it=200, **{q: S[q] for q in "abcdef"}),
    ]
    res = band.BatchPlan(specs).run()
    torch.cuda.synchronize()
    for sp, r in zip(specs[:4], res[:4]):
        k = 1 if sp["method"] == "ntdm" else 2
        x, st = _solve(band, {q: sp[q] for q in "abcdef"}, k, sp["schedule"])
        assert torch.equal(r["x"], x)
        assert (r["status"].cpu().numpy() == st).all()
        assert (st == 0).all()
    assert not torch.equal(res[0]["x"], res[3]["x"])     # the two orders round differently
    assert torch.allclose(res[0]["x"], res[3]["x"], rtol=0, atol=1e-12)


def test_auto_schedule_rule(band):
    """AUTO takes the two-sided sweep for systems of 32 rows or more and one thread per
    system for shorter ones or when x aliases f (bitwise comparison with the forced
    schedules)."""
    long_ = to_dev(synth.cfg0(nsys=64, n=64, seed_salt=29))
    short = to_dev(synth.cfg0(nsys=64, n=16, seed_salt=30))
    xa, _ = _solve(band, long_, 2, "auto")
    x2, _ = _solve(band, long_, 2, "two_sided")
    x1, _ = _solve(band, long_, 2, "thread")
    assert torch.equal(xa, x2) and not torch.equal(x1, x2)
    xa, _ = _solve(band, short, 2, "auto")
    x1, _ = _solve(band, short, 2, "thread")
    assert torch.equal(xa, x1)
    x1, _ = _solve(band, long_, 2, "thread")
    f = long_["f"].clone()
    _solve(band, dict(long_, f=f), 2, "auto", x=f)
    assert torch.equal(f, x1)


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_two_sided_symbolic_zero_pivots(band, case):
    """STDM / SPDM with the two-sided sweep: a zero pivot in either half goes to the
    symbolic fix-up, which returns the exact solution (or SINGULAR)."""
    k, n = case["k"], case["n"]
    fl = lambda key: np.array([float(Fraction(v)) for v in case[key]])
    nsys = 20
    B = dict(n=n, nsys=nsys, sys_stride=1, elem_stride=nsys)
    for q in "abcdef":
        B[q] = np.repeat(fl(q)[:, None], nsys, axis=1).reshape(-1)
    T = to_dev(B)
    a, e = (T["a"], T["e"]) if k == 2 else (None, None)
    x, st = band.solve(a, T["b"], T["c"], T["d"], e, T["f"], method="spdm" if k == 2 else "stdm",
                       schedule="two_sided")
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    if case["status"] == "SINGULAR":
        assert (st == 4).all(), st
        return
    assert (st == 0).all(), st
    want = fl("x")
    xg = flat_of(x).reshape(n, nsys)
    assert np.abs(xg - want[:, None]).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_two_sided_planted_zero_pivots(band):
    """Long systems with a_i = b_i = c_i = 0 in one row i, which makes NPDM's pivot of
    that row exactly 0 (gamma_i = 0, mu_i = c_i = 0 whatever came before).  With the
    symbolic pivot t there, mu_{i+1} = -alpha_i gamma_{i+1} is of order 1/t, and with
    a_{i+2} = 0 too every later pivot is of order 1: the orders cancel (the matrix is
    nonsingular) and the symbolic expansion stays short.
    Planted in the top half (systems 0..9): the two-sided sweep meets it too; NPDM reports
    ZERO_PIVOT and SPDM goes through the fix-up.  Planted in the bottom half (systems
    10..19): the mirrored elimination meets a nonzero pivot there, so both methods solve
    it directly.  Every solution is held to GEPP's."""
    n, nsys = 100, 40
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=31)
    for i, sl in ((20, slice(0, 10)), (80, slice(10, 20))):
        for q, r in (("a", i), ("b", i), ("c", i), ("a", i + 2)):
            B[q].reshape(n, nsys)[r, sl] = 0.0
    T = to_dev(B)
    xt, _, _, _ = _oracle(B, 2, "gepp")
    xs, ss, _, _ = _oracle(B, 2, "symbolic")
    assert (ss == 0).all()
    err_o = per_system_rel(xs, xt, *_args(B))
    bound = np.maximum(1e-12, 10 * err_o)

    x, st = _solve(band, T, 2, "two_sided")
    assert (st[0:10] == 3).all() and (st[10:] == 0).all(), st
    err = per_system_rel(flat_of(x), xt, *_args(B))
    assert (err[10:] <= bound[10:]).all()
    _, st1 = _solve(band, T, 2, "thread")
    assert (st1[0:20] == 3).all() and (st1[20:] == 0).all(), st1

    for sched in ("two_sided", "thread"):
        x, st = band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], T["f"], method="spdm",
                           schedule=sched)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        err = per_system_rel(flat_of(x), xt, *_args(B))
        assert (err <= bound).all(), (sched, err.max())
