"""GPU parity of Stone's method on 2-D five-point systems (band_sip2d) against the
oracle's R6b, system by system: the same number of updates (within one, the stopping
test sees different roundings), the solution to 1e-9 relative, statuses; both layouts,
non-square grids, the one-row grid that reduces to a tridiagonal solve in one update, the
update cap and a zero ILU(0) pivot."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV

pytestmark = pytest.mark.gpu

OK, ZERO_PIVOT, NOT_CONVERGED = 0, 3, 6


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def grid_batch(rng, nx, ny, nsys):
    """Backward-Euler-like 2-D five-point systems: neighbours -r times factors in
    [0.5, 1.5], diagonal 1 + 4r + [0, 0.1), r in [0.5, 4] per system; canonical (N, nsys)."""
    N = nx * ny
    r = rng.uniform(0.5, 4.0, nsys)[None, :]
    D = {q: -r * rng.uniform(0.5, 1.5, (N, nsys)) for q in "swet"}
    D["c"] = 1 + 4 * r + rng.uniform(0, 0.1, (N, nsys))
    f = rng.uniform(-1, 1, (N, nsys))
    return D, f


def _dev(v, layout):
    t = torch.tensor(v, device=DEV)
    return t if layout == "interleaved" else t.T.contiguous().T


@pytest.mark.parametrize("layout", ["interleaved", "contiguous"])
@pytest.mark.parametrize("nx,ny", [(16, 16), (12, 20), (37, 3), (50, 1)])
def test_sip2d_against_oracle(band, layout, nx, ny):
    nsys = 64
    rng = np.random.default_rng(nx * 100 + ny)
    D, f = grid_batch(rng, nx, ny, nsys)
    T = {q: _dev(D[q], layout) for q in "swcet"}
    F = _dev(f, layout)
    x, it, rs, st = band.sip2d(T["s"], T["w"], T["c"], T["e"], T["t"], F, nx, tol=1e-10,
                               max_it=500)
    torch.cuda.synchronize()
    x, it, rs, st = x.cpu().numpy(), it.cpu().numpy(), rs.cpu().numpy(), st.cpu().numpy()
    assert (st == OK).all()
    assert (rs < 1e-10).all()
    for s in range(0, nsys, 5):
        R = oracle.sip2d(nx, ny, *[D[q][:, s] for q in "swcet"], f[:, s], tol=1e-10, max_it=500)
        assert R["status"] == "OK"
        assert abs(int(it[s]) - R["iters"]) <= 1, (s, it[s], R["iters"])
        assert np.abs(x[:, s] - R["x"]).max() <= 1e-9 * np.abs(R["x"]).max(), s
        if ny == 1:
            assert it[s] == 1
        else:
            assert it[s] > 3


def test_sip2d_cap_and_zero_pivot(band):
    rng = np.random.default_rng(9)
    nx, ny, nsys = 16, 16, 8
    D, f = grid_batch(rng, nx, ny, nsys)
    D["c"][0, 3] = 0.0                # the first ILU(0) pivot of system 3
    T = {q: torch.tensor(D[q], device=DEV) for q in "swcet"}
    F = torch.tensor(f, device=DEV)
    x, it, rs, st = band.sip2d(T["s"], T["w"], T["c"], T["e"], T["t"], F, nx, tol=1e-10, max_it=3)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert st[3] == ZERO_PIVOT
    others = np.arange(nsys) != 3
    assert (st[others] == NOT_CONVERGED).all()
    assert (it.cpu().numpy()[others] == 3).all()
    R = oracle.sip2d(nx, ny, *[D[q][:, 0] for q in "swcet"], f[:, 0], tol=1e-10, max_it=3)
    assert R["status"] == "NOT_CONVERGED" and R["iters"] == 3
    assert abs(rs.cpu().numpy()[0] - R["resid"]) <= 1e-9 * R["resid"]


@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 5), (7, 9)])
def test_sip2d_layouts_agree_bitwise(band, nx, ny):
    """Interleaved batches are copied system-major for the warp kernel and x is copied
    back: the same grids in either layout give the same x, update counts and residuals
    bit for bit."""
    nsys = 45
    rng = np.random.default_rng(200 + nx + ny)
    D, f = grid_batch(rng, nx, ny, nsys)
    out = {}
    for layout in ("interleaved", "contiguous"):
        T = {q: _dev(D[q], layout) for q in "swcet"}
        out[layout] = band.sip2d(T["s"], T["w"], T["c"], T["e"], T["t"], _dev(f, layout), nx,
                                 tol=1e-10, max_it=500)
    torch.cuda.synchronize()
    (xi, ii, ri, si), (xc, ic, rc, sc) = out["interleaved"], out["contiguous"]
    assert xi.stride() != xc.stride()
    assert (si.cpu() == OK).all() and torch.equal(si, sc)
    assert torch.equal(xi.contiguous(), xc.contiguous())
    assert torch.equal(ii, ic) and torch.equal(ri, rc)


def test_sip2d_zero_pivot_keeps_x(band):
    """A system whose ILU(0) meets a zero pivot is not updated: its x keeps the caller's
    values, on the interleaved (staged) layout and on the contiguous one."""
    rng = np.random.default_rng(12)
    nx, ny, nsys = 16, 8, 40
    D, f = grid_batch(rng, nx, ny, nsys)
    D["c"][0, 5] = 0.0
    for layout in ("interleaved", "contiguous"):
        T = {q: _dev(D[q], layout) for q in "swcet"}
        x0 = _dev(np.full((nx * ny, nsys), 7.25), layout)
        x, it, rs, st = band.sip2d(T["s"], T["w"], T["c"], T["e"], T["t"], _dev(f, layout), nx,
                                   x=x0)
        torch.cuda.synchronize()
        st = st.cpu().numpy()
        assert st[5] == ZERO_PIVOT and (np.delete(st, 5) == OK).all()
        assert (x[:, 5].cpu().numpy() == 7.25).all(), layout
        assert not (x[:, 4].cpu().numpy() == 7.25).any()
