"""GPU parity of MNPDM (Sec. 1; Sec. 3.2 Remark 2) against the CPU oracle's R2m on
pentadiagonal systems whose outer diagonals are mostly zero: element by element to
1e-12 relative against the manufactured solution (10x the oracle's own error where the
elimination's multipliers grow), on both layouts, with x aliasing f and in FP32; without
outer entries it is the thread-per-system NTDM sweep bit for bit; a zero divisor of the
elimination is ZERO_PIVOT."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import DEV

pytestmark = pytest.mark.gpu

OK, ZERO_PIVOT = 0, 3


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def sparse_pd(rng, nsys, n, frac, adjacent=False):
    """Dominant PD systems (cfg0 recipe) keeping the outer entries on a fraction of the
    rows only (clusters of adjacent rows when asked), canonical (n, nsys)."""
    D = synth.dominant(rng, nsys, n, k=2)
    keep = rng.random((n, nsys)) < frac
    if adjacent:
        keep |= np.roll(keep, 1, axis=0) | np.roll(keep, 2, axis=0)
    keep[2, :] = True               # the first and last rows that can hold both
    keep[n - 3, :] = True
    D["a"] = np.where(keep, D["a"], 0.0)
    D["e"] = np.where(keep, D["e"], 0.0)
    D["a"][:2] = 0.0
    D["e"][n - 2:] = 0.0
    D["c"] = 1.0 + sum(np.abs(D[q]) for q in "abde")
    xt, f = synth.manufactured(rng, 2, D, nsys, n)
    return D, f, xt


def _dev(D, f, layout, dtype=torch.float64):
    def put(v):
        t = torch.tensor(v, dtype=dtype, device=DEV)
        return t if layout == "interleaved" else t.T.contiguous().T
    return {q: put(D[q]) for q in "abcde"}, put(f)


@pytest.mark.parametrize("schedule", ["auto", "thread"])
@pytest.mark.parametrize("layout", ["interleaved", "contiguous"])
@pytest.mark.parametrize("frac,adjacent", [(0.01, False), (0.05, True), (1.0, False)])
def test_mnpdm_against_oracle(band, layout, frac, adjacent, schedule):
    """Both paths: the row-parallel eliminations with NTDM on the automatic schedule, and
    one thread per system."""
    nsys, n = 200, 1031
    rng = np.random.default_rng(int(1000 * frac) + adjacent)
    D, f, xt = sparse_pd(rng, nsys, n, frac, adjacent)
    T, F = _dev(D, f, layout)
    x, st = band.solve(*(T[q] for q in "abcde"), F, method="mnpdm", schedule=schedule)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == OK).all()
    xg = x.cpu().numpy()
    for s in range(0, nsys, 7):
        xo, so = oracle.mnpdm(*[D[q][:, s] for q in "abcde"], f[:, s])
        assert so == "OK"
        # the elimination divides by off-diagonal entries and does not pivot: where its
        # multipliers grow, the bound is 10x the oracle's own error (non-dominant rule)
        den = np.abs(xt[:, s]).max()
        own = np.abs(xo - xt[:, s]).max() / den
        assert np.abs(xg[:, s] - xt[:, s]).max() / den <= max(1e-12, 10 * own), s



@pytest.mark.parametrize("schedule", ["auto", "thread"])
def test_mnpdm_without_outer_entries_is_ntdm(band, schedule):
    """No outer entries: MNPDM is NTDM on the same schedule, bit for bit (the automatic
    one of a single call: partitioned for this small batch)."""
    rng = np.random.default_rng(4)
    D, f, xt = sparse_pd(rng, 64, 500, 0.0)
    for q in "ae":
        D[q][:] = 0.0
    D["c"] = 1.0 + np.abs(D["b"]) + np.abs(D["d"])
    f = synth.band_matvec(1, D["a"], D["b"], D["c"], D["d"], D["e"], xt)
    T, F = _dev(D, f, "interleaved")
    x, st = band.solve(*(T[q] for q in "abcde"), F, method="mnpdm", schedule=schedule)
    xt_, stt = band.solve(None, T["b"], T["c"], T["d"], None, F, method="ntdm", schedule=schedule)
    torch.cuda.synchronize()
    assert (st.cpu() == OK).all() and (stt.cpu() == OK).all()
    assert torch.equal(x, xt_)


def test_mnpdm_aliasing_and_fp32(band):
    rng = np.random.default_rng(5)
    D, f, xt = sparse_pd(rng, 96, 700, 0.02)
    T, F = _dev(D, f, "interleaved")
    want, _ = band.solve(*(T[q] for q in "abcde"), F, method="mnpdm")
    x, st = band.solve(*(T[q] for q in "abcde"), F, method="mnpdm", x=F)
    torch.cuda.synchronize()
    assert x.data_ptr() == F.data_ptr() and torch.equal(x, want)
    T32, F32 = _dev(D, f, "interleaved", torch.float32)
    x32, st32 = band.solve(*(T32[q] for q in "abcde"), F32, method="mnpdm")
    torch.cuda.synchronize()
    assert (st32.cpu() == OK).all()
    assert (np.abs(x32.cpu().numpy() - xt).max(0) / np.abs(xt).max(0)).max() <= 1e-4


@pytest.mark.parametrize("schedule", ["auto", "thread"])
def test_mnpdm_zero_divisor(band, schedule):
    """Row 2's e is eliminated with row 3, whose superdiagonal is 0: ZERO_PIVOT for that
    system only."""
    n, nsys = 8, 3
    D = {q: np.zeros((n, nsys)) for q in "abcde"}
    D["b"][1:] = 1.0
    D["d"][:-1] = 1.0
    D["c"][:] = 4.0
    D["e"][2, 1] = 1.0
    D["d"][3, 1] = 0.0
    f = np.ones((n, nsys))
    T, F = _dev(D, f, "interleaved")
    x, st = band.solve(*(T[q] for q in "abcde"), F, method="mnpdm", schedule=schedule)
    torch.cuda.synchronize()
    assert st.cpu().tolist() == [OK, ZERO_PIVOT, OK]
    assert oracle.mnpdm(*[D[q][:, 1] for q in "abcde"], f[:, 1])[1] == "ZERO_PIVOT"
