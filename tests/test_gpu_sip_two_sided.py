"""GPU parity of Algorithm 1's first update on the two-sided schedule (two threads per
system; the lower half of the exact ILU(0) = LU factorisation taken bottom-up) against
the one-thread schedule, which follows the printed order of operations, and the CPU
oracle.  Systems that need more updates, and those the two-sided elimination cannot
start (a zero pivot in either half, a singular interface system, n < 4), go to the
block-cooperative tail, which rebuilds the top-down factors first."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import flat_of, per_system_rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _sip(band, T, schedule, tol=1e-10, max_it=200):
    x, it, rs, st = band.sip(*(T[q] for q in "abcdef"), tol=tol, max_it=max_it, width=0,
                             schedule=schedule)
    torch.cuda.synchronize()
    return x, it.cpu().numpy(), rs.cpu().numpy(), st.cpu().numpy()


def _args(B):
    return B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 33, 300])
@pytest.mark.parametrize("layout", ["interleaved", "contiguous"])
def test_dominant_matches_one_thread(band, n, layout):
    """Dominant systems (37: two 16-system warps and a tail of 5): both schedules stop
    after one update with max|r| < tol and agree to 1e-12; n < 4 runs through the tail
    from x^0 = 0."""
    B = synth.cfg0(nsys=37, n=n, layout=layout, seed_salt=41)
    T = to_dev(B)
    x2, it2, rs2, st2 = _sip(band, T, "two_sided")
    x1, it1, rs1, st1 = _sip(band, T, "thread")
    assert (st1 == 0).all() and (st2 == 0).all()
    assert (np.abs(it2 - it1) <= 1).all()
    assert (rs2 < 1e-10).all()
    args = _args(B)
    assert per_system_rel(flat_of(x2), flat_of(x1), *args).max() <= 1e-12
    assert per_system_rel(flat_of(x2), B["x_true"], *args).max() <= 1e-12


@pytest.mark.parametrize("r", synth.ADI_R)
def test_adi_against_oracle(band, r):
    """The non-dominant ADI systems at n = 2048 (96 lines of each sweep): statuses and
    iteration counts as the oracle's (within one), the solution held to GEPP's like the
    oracle's own Algorithm 1 result."""
    for sweep in ("x", "y"):
        B = synth.cfg1(r=r, k=2, sweep=sweep, grid=2048, nsys=96)
        T = to_dev(B)
        x, it, rs, st = _sip(band, T, "two_sided")
        args = _args(B)
        xo, so, ito, _ = oracle.batch("sip", 2, [B[q] for q in "abcde"], B["f"], B["nsys"],
                                      B["n"], B["sys_stride"], B["elem_stride"], hb_width=0,
                                      tol=1e-10)
        xt, _, _, _ = oracle.batch("gepp", 2, [B[q] for q in "abcde"], B["f"], B["nsys"], B["n"],
                                   B["sys_stride"], B["elem_stride"])
        assert (np.abs(it - ito) <= 1).all()
        ok = (st == 0) & (so == 0)
        assert ok.sum() >= len(st) - 4          # a few may sit at the rounding floor
        err_o = per_system_rel(xo, xt, *args)
        err = per_system_rel(flat_of(x), xt, *args)
        assert (err[ok] <= np.maximum(1e-10, 10 * err_o[ok])).all()
        # systems that stop above tol do so for the reason the oracle gives
        assert np.isin(st[~ok], (0, 6)).all()


def test_special_stops(band):
    """f = 0: no update (x = 0, 0 iterations, OK).  max_it = 0: no update and
    NOT_CONVERGED.  max_it = 1: one update.  A NaN in f in either half: NONFINITE."""
    n, nsys = 64, 32
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=42)
    T = to_dev(B)
    Z = dict(T, f=torch.zeros_like(T["f"]))
    x, it, rs, st = _sip(band, Z, "two_sided")
    assert (st == 0).all() and (it == 0).all() and (flat_of(x) == 0).all()
    x, it, rs, st = _sip(band, T, "two_sided", max_it=0)
    assert (st == 6).all() and (it == 0).all()
    x, it, rs, st = _sip(band, T, "two_sided", max_it=1)
    assert (it == 1).all() and (st == 0).all()
    f = B["f"].copy().reshape(n, nsys)
    f[3, 4] = np.nan
    f[60, 9] = np.nan
    C = dict(B, f=f.reshape(-1))
    x, it, rs, st = _sip(band, to_dev(C), "two_sided")
    assert st[4] == 5 and st[9] == 5
    assert (np.delete(st, [4, 9]) == 0).all()


def test_zero_pivots(band):
    """Rows with a_i = b_i = c_i = 0 (and a_{i+2} = 0) make the top-down pivot of row i
    exactly 0.  In the top half (systems 0..9) the two-sided sweep meets it as well and
    the tail, factoring top-down, reports ZERO_PIVOT like the one-thread schedule.  In
    the bottom half (systems 10..19) the mirrored elimination meets a nonzero pivot and
    solves the system in one update; the one-thread schedule reports ZERO_PIVOT."""
    n, nsys = 100, 40
    B = synth.cfg0(nsys=nsys, n=n, seed_salt=43)
    for i, sl in ((20, slice(0, 10)), (80, slice(10, 20))):
        for q, r in (("a", i), ("b", i), ("c", i), ("a", i + 2)):
            B[q].reshape(n, nsys)[r, sl] = 0.0
    T = to_dev(B)
    x2, it2, rs2, st2 = _sip(band, T, "two_sided")
    x1, it1, rs1, st1 = _sip(band, T, "thread")
    assert (st1[:20] == 3).all() and (st1[20:] == 0).all()
    assert (st2[:10] == 3).all() and (st2[10:] == 0).all(), st2
    xt, _, _, _ = oracle.batch("gepp", 2, [B[q] for q in "abcde"], B["f"], nsys, n, 1, nsys)
    err = per_system_rel(flat_of(x2), xt, n, nsys, 1, nsys)
    assert err[10:20].max() <= 1e-10
    assert per_system_rel(flat_of(x2), flat_of(x1), n, nsys, 1, nsys)[20:].max() <= 1e-12


def test_batch_runs_one_thread_per_system(band):
    """The batched kernel keeps SIP on one thread per system whatever the schedule says
    (bitwise equal to band_sip on that schedule)."""
    S = to_dev(synth.cfg1(r=0.5, k=2, sweep="y", grid=1024, nsys=80))
    P = to_dev(synth.cfg0(nsys=50, n=120, seed_salt=44))
    specs = [dict(op="sip", schedule="two_sided", **S), dict(op="sip", schedule="two_sided", **P),
             dict(method="npdm", **P)]
    res = band.BatchPlan(specs).run()
    torch.cuda.synchronize()
    for sp, r in zip(specs[:2], res[:2]):
        T = {q: sp[q] for q in "abcdef"}
        x, it, rs, st = _sip(band, T, "thread")
        assert torch.equal(r["x"], x)
        assert (r["iters"].cpu().numpy() == it).all()
        assert (r["status"].cpu().numpy() == st).all()
