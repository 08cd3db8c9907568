"""The automatic schedule of single-problem calls.  A small batch of long NTDM / NPDM
systems (fewer than 32 per SM, n >= 256) runs partitioned; a system whose partitioned
elimination fails (a chunk pivot the guard rejects, on rows that are not diagonally
dominant) is listed and solved again by the AUTO sweep (two-sided, or one thread when x
aliases f) in a second launch.  On dominant rows the result is bit for bit the explicit
partitioned schedule's; on indefinite rows it holds the oracle's non-dominant bound; a
system whose failure is forced is bit for bit the AUTO sweep's solve; a captured graph
replays the same results."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _args(T, k):
    return [T[q] for q in "abcdef"] if k == 2 else [None, T["b"], T["c"], T["d"], None, T["f"]]


def _method(k):
    return "npdm" if k == 2 else "ntdm"


def _is_dominant(B, k):
    n, ns, ss, es = B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]
    idx = np.arange(ns)[None, :] * ss + np.arange(n)[:, None] * es
    g = {q: np.abs(B[q][idx]) for q in "abcde"}
    row = np.arange(n)[:, None]
    off = np.where(row >= 1, g["b"], 0) + np.where(row + 1 < n, g["d"], 0)
    if k == 2:
        off = off + np.where(row >= 2, g["a"], 0) + np.where(row + 2 < n, g["e"], 0)
    return bool((g["c"] >= off).all())


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("sweep", ["x", "y"])
def test_dominant_small_batch_runs_partitioned(band, k, sweep):
    B = synth.cfg1(r=0.5, k=k, sweep=sweep, grid=1024, nsys=512)
    T = to_dev(B)
    x, st = band.solve(*_args(T, k), method=_method(k))
    xp, stp = band.solve(*_args(T, k), method=_method(k), schedule="partitioned")
    torch.cuda.synchronize()
    assert (st.cpu() == 0).all()
    if _is_dominant(B, k):
        assert torch.equal(x, xp) and torch.equal(st, stp)


@pytest.mark.parametrize("r", [0.5, 2.0, 10.0])
def test_adi_rows_within_the_bound(band, r):
    """The PD ADI rows of this recipe are not diagonally dominant (at r = 2 indefinite):
    systems that fail in the partitioned sweep are redone; every system stays within
    1e-10 of the oracle's GEPP, with status OK."""
    B = synth.cfg1(r=r, k=2, sweep="y", grid=1024, nsys=512)
    T = to_dev(B)
    x, st = band.solve(*_args(T, 2), method="npdm")
    torch.cuda.synchronize()
    assert (st.cpu() == 0).all()
    xg = x.cpu().numpy()
    n, ns, ss, es = B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]
    for s in range(0, ns, 37):
        idx = s * ss + np.arange(n) * es
        xo = oracle.gepp_band(2, *[B[q][idx] for q in "abcde"], B["f"][idx])[0]
        assert np.abs(xg[:, s] - xo).max() / np.abs(xo).max() <= 1e-10, s


@pytest.mark.parametrize("alias", [False, True])
def test_forced_redo_equals_auto_sweep(band, alias):
    """Systems 3 and 40 get c_j = 0 at every row that is a multiple of 8 (every chunk
    start for the chunk counts the library can pick at n = 1024): the first pivot of
    each chunk of theirs is 0, so their partitioned elimination fails, while NPDM's
    pivot at such a row is c_j less nonzero terms.  The second launch solves them: bit
    for bit the two-sided solve (one thread when x aliases f); the other systems bit for
    bit the explicit partitioned schedule's."""
    B = synth.cfg0(nsys=300, n=1024, seed_salt=62)
    T = to_dev(B)
    c = T["c"].clone()
    for s in (3, 40):
        c[8::8, s] = 0.0
    args = [T["a"], T["b"], c, T["d"], T["e"]]
    ref, stref = band.solve(*args, T["f"], method="npdm",
                            schedule="thread" if alias else "two_sided")
    xp, stp = band.solve(*args, T["f"], method="npdm", schedule="partitioned")
    if alias:
        F = T["f"].clone()
        x, st = band.solve(*args, F, method="npdm", x=F)
        assert x.data_ptr() == F.data_ptr()
    else:
        x, st = band.solve(*args, T["f"], method="npdm")
    torch.cuda.synchronize()
    assert torch.equal(st, stref)
    assert (st.cpu() == 0).all()
    for s in range(300):
        want = ref[:, s] if s in (3, 40) else xp[:, s]
        assert torch.equal(x[:, s], want), s


def test_aliasing_dominant(band):
    """x aliasing f on a dominant small batch: the partitioned solve, in place."""
    B = synth.cfg0(nsys=300, n=700, seed_salt=61)
    T = to_dev(B)
    want_p, _ = band.solve(*_args(T, 2), method="npdm", schedule="partitioned")
    F = T["f"].clone()
    x, st = band.solve(*(_args(T, 2)[:5] + [F]), method="npdm", x=F)
    torch.cuda.synchronize()
    assert x.data_ptr() == F.data_ptr() and torch.equal(x, want_p)
    assert (st.cpu() == 0).all()


def test_graph_replay(band):
    """One captured AUTO solve replayed on r = 0.5, then r = 2, then r = 0.5 data in the
    same buffers: each replay equals the eager solve of that data (the redo list is
    rebuilt at every replay)."""
    Bd = synth.cfg1(r=0.5, k=2, sweep="y", grid=1024, nsys=512)
    Bn = synth.cfg1(r=2.0, k=2, sweep="y", grid=1024, nsys=512)
    Td, Tn = to_dev(Bd), to_dev(Bn)
    T = {q: Td[q].clone() for q in "abcdef"}
    want = {}
    for name, src in (("r0.5", Td), ("r2", Tn)):
        want[name], _ = band.solve(*_args(src, 2), method="npdm")
    x = torch.empty_like(T["f"])
    band.solve(*_args(T, 2), method="npdm", x=x)        # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            band.solve(*_args(T, 2), method="npdm", x=x)
    torch.cuda.current_stream().wait_stream(s)
    for name, src in (("r0.5", Td), ("r2", Tn), ("r0.5", Td)):
        for q in "abcdef":
            T[q].copy_(src[q])
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(x, want[name]), name
