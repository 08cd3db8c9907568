"""GPU parity of the grid schedule (one system, or a few, over the whole GPU) against
the CPU oracle's NPDM / NTDM (R2 / R1) element by element, at sizes from one chunk to
the 10^7-row single system, on both layouts, with x aliasing f, in FP32, and on
indefinite ADI rows (where the schedule may decline a system with ZERO_PIVOT, never
return a wrong result).  Tolerances: 1e-12 relative on dominant systems, 1e-10 on the
ADI rows (FP64); FP32 against the FP64 oracle to 1e-4."""
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


def _oracle_x(k, D, f, s):
    if k == 2:
        x, st = oracle.npdm(*[D[q][:, s] for q in "abcde"], f[:, s])
    else:
        x, st = oracle.ntdm(D["b"][:, s], D["c"][:, s], D["d"][:, s], f[:, s])
    assert st == "OK"
    return x


def _canon(k, nsys, n, seed):
    rng = np.random.default_rng(seed)
    D = synth.dominant(rng, nsys, n, k=k)
    xt, f = synth.manufactured(rng, k, D, nsys, n)
    return D, f, xt


def _dev(D, f, layout, dtype=torch.float64):
    """Device views (n, nsys) in the layout: interleaved = contiguous (n, nsys) storage,
    contiguous systems = the transpose of contiguous (nsys, n) storage."""
    def put(v):
        t = torch.tensor(v, dtype=dtype, device=DEV)
        return t if layout == "interleaved" else t.T.contiguous().T
    return {q: put(D[q]) for q in "abcde"}, put(f)


def _rel(x, ref):
    return np.abs(x - ref).max(0) / np.abs(ref).max(0)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("nsys,n", [(1, 100), (1, 1000), (1, 77777), (1, 1000003), (3, 300001),
                                    (40, 20000)])
@pytest.mark.parametrize("layout", ["interleaved", "contiguous"])
def test_grid_against_oracle(band, k, nsys, n, layout):
    """Dominant systems; sizes from a single chunk (n < 128) through chunk counts that do
    not divide n to one system of 10^6 rows cut into ~15600 chunks."""
    D, f, xt = _canon(k, nsys, n, seed=n + nsys + 10 * k)
    T, F = _dev(D, f, layout)
    a, e = (T["a"], T["e"]) if k == 2 else (None, None)
    x, st = band.solve(a, T["b"], T["c"], T["d"], e, F, method="npdm" if k == 2 else "ntdm",
                       schedule="grid")
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == OK).all()
    xg = x.cpu().numpy()
    for s in range(min(nsys, 4)):
        xo = _oracle_x(k, D, f, s)
        assert np.abs(xg[:, s] - xo).max() <= 1e-12 * np.abs(xo).max(), s
    assert _rel(xg, xt).max() <= 1e-12


def test_grid_x_aliases_f(band):
    D, f, xt = _canon(2, 2, 500000, seed=3)
    T, F = _dev(D, f, "interleaved")
    x, st = band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], F, method="npdm", x=F,
                       schedule="grid")
    torch.cuda.synchronize()
    assert x.data_ptr() == F.data_ptr()
    assert (st.cpu().numpy() == OK).all()
    assert _rel(x.cpu().numpy(), xt).max() <= 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_grid_fp32(band, k):
    n = 400000
    rng = np.random.default_rng(11 + k)
    D = synth.dominant(rng, 1, n, k=k, dtype=np.float32)
    xt, f = synth.manufactured(rng, k, D, 1, n)
    T = {q: torch.tensor(D[q], device=DEV) for q in "abcde"}
    F = torch.tensor(f.astype(np.float32), device=DEV)
    a, e = (T["a"], T["e"]) if k == 2 else (None, None)
    x, st = band.solve(a, T["b"], T["c"], T["d"], e, F, method="npdm" if k == 2 else "ntdm",
                       schedule="grid")
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == OK).all()
    D64 = {q: D[q].astype(np.float64) for q in "abcde"}
    xo = _oracle_x(k, D64, f.astype(np.float32).astype(np.float64), 0)
    assert np.abs(x.cpu().numpy()[:, 0] - xo).max() <= 1e-4 * np.abs(xo).max()


@pytest.mark.parametrize("r", synth.ADI_R)
@pytest.mark.parametrize("k", [1, 2])
def test_grid_indefinite_adi_line(band, r, k):
    """One long line of the ADI rows (n = 2^20; the PD rows are indefinite): each system
    is either declined with ZERO_PIVOT or solved to the non-dominant bound, 1e-10 relative
    against the manufactured solution, or 10x the oracle NPDM's own error where LU
    without pivoting cannot reach 1e-10 on the line."""
    n, nsys = 1 << 20, 2
    rng = np.random.default_rng(int(10 * r) + k)
    g = rng.uniform(-1, 1, size=(n, nsys))
    D = synth.adi_rows(r, n, g, k)
    xt = rng.uniform(-1, 1, size=(n, nsys))
    f = synth.band_matvec(k, D["a"], D["b"], D["c"], D["d"], D["e"], xt)
    T, F = _dev(D, f, "interleaved")
    a, e = (T["a"], T["e"]) if k == 2 else (None, None)
    x, st = band.solve(a, T["b"], T["c"], T["d"], e, F, method="npdm" if k == 2 else "ntdm",
                       schedule="grid")
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert set(st.tolist()) <= {OK, ZERO_PIVOT}
    xg = x.cpu().numpy()
    for s in range(nsys):
        if st[s] != OK:
            continue
        xo = _oracle_x(k, D, f, s)
        den = np.abs(xt[:, s]).max()
        own = np.abs(xo - xt[:, s]).max() / den
        err = np.abs(xg[:, s] - xt[:, s]).max() / den
        assert err <= max(1e-10, 10 * own), (r, k, s, err, own)
    if k == 1:
        assert (st == OK).all()       # the TD rows are dominant


def test_grid_ten_million_rows(band):
    """One PD system of 10^7 rows against the oracle, element by element."""
    D, f, xt = _canon(2, 1, 10_000_000, seed=17)
    T, F = _dev(D, f, "interleaved")
    x, st = band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], F, method="npdm", schedule="grid")
    torch.cuda.synchronize()
    assert int(st.item()) == OK
    xo = _oracle_x(2, D, f, 0)
    assert np.abs(x.cpu().numpy()[:, 0] - xo).max() <= 1e-12 * np.abs(xo).max()


def test_grid_rejects_other_calls(band):
    """Only band_solve (numeric methods, no factors) takes the grid schedule."""
    D, f, xt = _canon(2, 1, 1000, seed=5)
    T, F = _dev(D, f, "interleaved")
    from paper_1804_09666_gb300 import BandError
    with pytest.raises(BandError):
        band.solve(T["a"], T["b"], T["c"], T["d"], T["e"], F, method="spdm", schedule="grid")
    with pytest.raises(BandError):
        band.BatchPlan([dict(method="npdm", schedule="grid", **T, f=F)]).run()
