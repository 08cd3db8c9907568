"""Writes stay inside their arrays, on every schedule.

Each output (x and the statuses) and the workspace sits inside a larger buffer whose
other entries hold a sentinel: a head before the first element, the gaps between
systems that the strides leave, and a tail after the last one.  The inputs sit the
same way, their heads, gaps and tails NaN.  Heads of one element put the FP64 arrays
off the 16-byte boundary (plain loads), heads of two on it (the 16-byte granule ring
for contiguous systems).  After each solve every sentinel is unchanged and x matches
the oracle.  This is the bounds evidence of the device code that a memory checker
would otherwise give.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import DEV, per_system_rel
from paper_1804_09666_gb300 import _lib as L

pytestmark = pytest.mark.gpu

METHODS = {"ntdm": L.NTDM, "npdm": L.NPDM, "stdm": L.STDM, "spdm": L.SPDM}
X_SENT = -3.0e299               # a finite double no solve produces here
ST_SENT = 0x5A5A5A5A            # int32
WS_SENT = 0xA5                  # byte
TAIL = 40                       # elements after the last one
WS_PAD = 1024                   # bytes before and after the workspace (256-aligned)


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _strides(layout, nsys, n):
    return (1, nsys + 3) if layout == "interleaved" else (n + 5, 1)   # (sys, elem)


def _padded(canon, head, ss, es, fill):
    """Flat host buffer: `head` fill entries, then canon (n, nsys) at the given
    strides with fill in the gaps, then TAIL fill entries."""
    n, nsys = canon.shape
    span = (n - 1) * es + (nsys - 1) * ss + 1
    buf = np.full(head + span + TAIL, fill, dtype=np.float64)
    idx = head + np.arange(nsys)[None, :] * ss + np.arange(n)[:, None] * es
    buf[idx] = canon
    return buf, idx


def _system(k, nsys, n, seed, plant=None):
    """Dominant canonical systems; plant: (kind, systems) -- "zero_row" gives row 5 of
    each listed system a = b = c = 0 (a zero pivot in any arithmetic), "chunk_starts"
    sets c = 0 on every eighth row (the partitioned elimination's first pivot of every
    chunk is then 0)."""
    rng = np.random.default_rng(seed)
    D = synth.dominant(rng, nsys, n, k=k)
    D = {q: np.array(D[q], dtype=np.float64) for q in "abcde"}
    if plant is not None:
        kind, systems = plant
        for s in systems:
            if kind == "zero_row":
                D["a"][5, s] = D["b"][5, s] = D["c"][5, s] = 0.0
            else:
                D["c"][8::8, s] = 0.0
    xt = rng.uniform(-1.0, 1.0, size=(n, nsys))
    f = synth.band_matvec(k, D["a"], D["b"], D["c"], D["d"], D["e"], xt)
    return D, f


def _run(band, method, schedule, layout, head, nsys, n, plant=None, seed=0):
    k = 1 if method in ("ntdm", "stdm") else 2
    D, f = _system(k, nsys, n, seed, plant)
    ss, es = _strides(layout, nsys, n)
    host = {}
    for q in "abcde":
        host[q], idx = _padded(D[q], head, ss, es, np.nan)
    host["f"], idx = _padded(f, head, ss, es, np.nan)
    view = lambda buf: buf.as_strided((n, nsys), (es, ss), head)
    dev = {q: torch.from_numpy(v).to(DEV) for q, v in host.items()}
    args = [view(dev[q]) if (k == 2 or q not in "ae") else None for q in "abcdef"]
    xbuf = torch.full_like(dev["f"], X_SENT)
    x = view(xbuf)
    sbuf = torch.full((nsys + 64,), ST_SENT, dtype=torch.int32, device=DEV)
    status = sbuf[32:32 + nsys]
    desc = band.desc_for(x, k, schedule)
    need = L.load().band_workspace_size(ct.byref(desc), L.OP_SOLVE, METHODS[method], 0)
    wbuf = torch.full((need + 2 * WS_PAD,), WS_SENT, dtype=torch.uint8, device=DEV)
    ws = wbuf[WS_PAD:WS_PAD + need]
    assert ws.data_ptr() % 256 == 0
    band.solve(*args, method=method, x=x, status=status, ws=ws, schedule=schedule)
    torch.cuda.synchronize()
    # every sentinel outside the arrays' elements is unchanged
    xh = xbuf.cpu().numpy()
    inside = np.zeros(xh.size, dtype=bool)
    inside[idx.reshape(-1)] = True
    assert (xh[~inside] == X_SENT).all(), "x written outside its elements"
    sh = sbuf.cpu().numpy()
    assert (sh[:32] == ST_SENT).all() and (sh[32 + nsys:] == ST_SENT).all(), "status overrun"
    wh = wbuf.cpu().numpy()
    assert (wh[:WS_PAD] == WS_SENT).all(), "workspace underrun"
    assert (wh[WS_PAD + need:] == WS_SENT).all(), "workspace overrun"
    # every system solved, and solved right
    assert (sh[32:32 + nsys] == 0).all(), sh[32:32 + nsys]
    diags = tuple(host[q][head:] for q in "abcde")
    ref, rst, _, _ = oracle.batch("gepp", k, diags, host["f"][head:], nsys, n, ss, es)
    assert (np.asarray(rst) == 0).all()
    rel = per_system_rel(xh[head:], ref, n, nsys, ss, es)
    return rel


LAYOUTS = ["interleaved", "contiguous"]
HEADS = [1, 2]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("schedule", ["auto", "thread", "two_sided", "partitioned"])
@pytest.mark.parametrize("method", ["npdm", "ntdm"])
def test_numeric_writes_stay_inside(band, method, schedule, layout, head):
    rel = _run(band, method, schedule, layout, head, nsys=70, n=600, seed=head)
    assert rel.max() <= 1e-12, rel.max()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("method", ["npdm", "ntdm"])
def test_grid_schedule_writes_stay_inside(band, method, layout, head):
    rel = _run(band, method, "grid", layout, head, nsys=3, n=6000, seed=10 + head)
    assert rel.max() <= 1e-12, rel.max()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
def test_redo_list_writes_stay_inside(band, layout, head):
    """The automatic schedule with systems whose partitioned elimination fails: the
    redo counter and list in the workspace, then the second launch."""
    rel = _run(band, "npdm", "auto", layout, head, nsys=70, n=600,
               plant=("chunk_starts", (3, 41, 69)), seed=20 + head)
    assert rel.max() <= 1e-10, rel.max()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("schedule", ["auto", "thread", "two_sided", "partitioned"])
@pytest.mark.parametrize("method", ["spdm", "stdm"])
def test_symbolic_writes_stay_inside(band, method, schedule, layout, head):
    """Zero pivots in three systems: the flagged list, the fix-up's slots and its
    series scratch in the workspace."""
    rel = _run(band, method, schedule, layout, head, nsys=70, n=600,
               plant=("zero_row", (0, 33, 69)), seed=30 + head)
    assert rel.max() <= 1e-10, rel.max()
