"""Writes stay inside their arrays, on every schedule and entry point.

Each output (x, the statuses, iteration counts, residuals, gradients, determinants,
stored factors) and the workspace sits inside a larger buffer whose other entries hold
a sentinel: a head before the first element, the gaps between systems that the strides
leave, and a tail after the last one.  The inputs sit the same way, their heads, gaps
and tails NaN.  Heads of one element put the FP64 arrays off the 16-byte boundary
(plain loads), heads of two on it (the 16-byte granule ring for contiguous systems).
After each call every sentinel is unchanged and the results match the oracle.  This is
the bounds evidence of the device code that a memory checker would otherwise give.
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
X_SENT = -3.0e299               # a finite double none of these calls produces
I_SENT = 0x5A5A5A5A             # int32 / int64 sentinel
WS_SENT = 0xA5                  # byte
TAIL = 40                       # entries after the last element
FLAT_HEAD = 32                  # entries before a per-system output
WS_PAD = 1024                   # bytes before and after a workspace (256-aligned)
LAYOUTS = ["interleaved", "contiguous"]
HEADS = [1, 2]


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
    strides with fill in the gaps, then TAIL fill entries; and the elements' indexes."""
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


class Guards:
    """Outputs made inside sentinel-filled buffers, checked together after a call."""

    def __init__(self):
        self.guards = []          # (name, buffer, check) of every output

    def padded_out(self, name, count, dtype, head=FLAT_HEAD):
        """count entries after `head` sentinels, TAIL sentinels after them."""
        sent = X_SENT if dtype == torch.float64 else I_SENT
        buf = torch.full((head + count + TAIL,), sent, dtype=dtype, device=DEV)
        self.guards.append((name, buf, lambda h: (h[:head] == sent).all() and
                            (h[head + count:] == sent).all()))
        return buf[head:head + count]

    def flat_out(self, name, count, dtype):
        return self.padded_out(name, count, dtype)

    def workspace(self, name, nbytes):
        buf = torch.full((nbytes + 2 * WS_PAD,), WS_SENT, dtype=torch.uint8, device=DEV)
        self.guards.append((name, buf, lambda h: (h[:WS_PAD] == WS_SENT).all() and
                            (h[WS_PAD + nbytes:] == WS_SENT).all()))
        ws = buf[WS_PAD:WS_PAD + nbytes]
        assert ws.data_ptr() % 256 == 0
        return ws

    def check_guards(self):
        torch.cuda.synchronize()
        for name, buf, ok in self.guards:
            assert ok(buf.cpu().numpy()), "%s written outside its elements" % name


class Case(Guards):
    """One batch's inputs in guarded strided storage on the device; guarded strided,
    per-system and workspace outputs made on request and checked together."""

    def __init__(self, k, nsys, n, layout, head, seed=0, plant=None, data=None):
        super().__init__()
        self.k, self.nsys, self.n, self.head = k, nsys, n, head
        self.ss, self.es = _strides(layout, nsys, n)
        D, f = data if data is not None else _system(k, nsys, n, seed, plant)
        self.host = {}
        for q in "abcde":
            self.host[q], self.idx = _padded(D[q], head, self.ss, self.es, np.nan)
        self.host["f"], _ = _padded(f, head, self.ss, self.es, np.nan)
        self.dev = {q: torch.from_numpy(v).to(DEV) for q, v in self.host.items()}
        self.inside = np.zeros(self.host["f"].size, dtype=bool)
        self.inside[self.idx.reshape(-1)] = True

    def view(self, buf):
        return buf.as_strided((self.n, self.nsys), (self.es, self.ss), self.head)

    def put(self, canon):
        """A strided device input holding canon (n, nsys), NaN outside its elements."""
        return self.view(torch.from_numpy(_padded(canon, self.head, self.ss, self.es,
                                                  np.nan)[0]).to(DEV))

    def diag5(self):
        keep = "abcde" if self.k == 2 else "bcd"
        return L.DIAG5(*[(self.view(self.dev[q]).data_ptr() if q in keep else None)
                         for q in "abcde"])

    def system(self, q, s):
        return self.host[q][self.idx[:, s]]

    def strided_out(self, name):
        """A strided output in the inputs' layout, the sentinel outside its elements."""
        buf = torch.full_like(self.dev["f"], X_SENT)
        self.guards.append((name, buf, lambda h: (h[~self.inside] == X_SENT).all()))
        return self.view(buf)

    def desc(self, schedule="auto", chunks=0):
        sched = {"auto": L.SCHED_AUTO, "thread": L.SCHED_THREAD, "two_sided": L.SCHED_TWO_SIDED,
                 "partitioned": L.SCHED_PARTITIONED, "grid": L.SCHED_GRID}[schedule]
        return L.BandDesc(half_bw=self.k, dtype=L.F64, nsys=self.nsys, n=self.n,
                          sys_stride=self.ss, elem_stride=self.es, offsets=None, hbw=None,
                          total_rows=0, schedule=sched, chunks=chunks)

    def gepp(self):
        """The oracle's banded GEPP solution, canonical (n, nsys)."""
        diags = tuple(self.host[q][self.head:] for q in "abcde")
        ref, st, _, _ = oracle.batch("gepp", self.k, diags, self.host["f"][self.head:],
                                     self.nsys, self.n, self.ss, self.es)
        assert (np.asarray(st) == 0).all()
        return np.asarray(ref)[self.idx - self.head]

    def rel(self, x_view, canon):
        """Per-system relative error of a strided device output against canon."""
        got = x_view.cpu().numpy()
        return per_system_rel(got.reshape(-1), canon.reshape(-1), self.n, self.nsys,
                              1, self.nsys)


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _solve(C, method, schedule):
    lib = L.load()
    desc = C.desc(schedule)
    x = C.strided_out("x")
    status = C.flat_out("status", C.nsys, torch.int32)
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE,
                                                          METHODS[method], 0))
    code = lib.band_solve(ct.byref(desc), METHODS[method], None, C.diag5(),
                          C.view(C.dev["f"]).data_ptr(), x.data_ptr(), status.data_ptr(),
                          ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    return C.rel(x, C.gepp())


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("schedule", ["auto", "thread", "two_sided", "partitioned"])
@pytest.mark.parametrize("method", ["npdm", "ntdm"])
def test_numeric_writes_stay_inside(band, method, schedule, layout, head):
    C = Case(2 if method == "npdm" else 1, 70, 600, layout, head, seed=head)
    assert _solve(C, method, schedule).max() <= 1e-12


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("method", ["npdm", "ntdm"])
def test_grid_schedule_writes_stay_inside(band, method, layout, head):
    C = Case(2 if method == "npdm" else 1, 3, 6000, layout, head, seed=10 + head)
    assert _solve(C, method, "grid").max() <= 1e-12


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
def test_redo_list_writes_stay_inside(band, layout, head):
    """The automatic schedule with systems whose partitioned elimination fails: the
    redo counter and list in the workspace, then the second launch."""
    C = Case(2, 70, 600, layout, head, seed=20 + head, plant=("chunk_starts", (3, 41, 69)))
    assert _solve(C, "npdm", "auto").max() <= 1e-10


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("schedule", ["auto", "thread", "two_sided", "partitioned"])
@pytest.mark.parametrize("method", ["spdm", "stdm"])
def test_symbolic_writes_stay_inside(band, method, schedule, layout, head):
    """Zero pivots in three systems: the flagged list, the fix-up's slots and its
    series scratch in the workspace."""
    C = Case(2 if method == "spdm" else 1, 70, 600, layout, head, seed=30 + head,
             plant=("zero_row", (0, 33, 69)))
    assert _solve(C, method, schedule).max() <= 1e-10


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("width", [0, 5])
def test_sip_writes_stay_inside(band, width, layout, head):
    """band_sip: x, iteration counts, residuals, statuses and the workspace (the ILU(0)
    factors, or the Hotelling-Bodewig band inverses for width 5)."""
    lib = L.load()
    C = Case(2, 70, 600, layout, head, seed=40 + head)
    desc = C.desc()
    x = C.strided_out("x")
    iters = C.flat_out("iters", C.nsys, torch.int32)
    resid = C.flat_out("resid", C.nsys, torch.float64)
    status = C.flat_out("status", C.nsys, torch.int32)
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), L.OP_SIP, 0, width))
    code = lib.band_sip(ct.byref(desc), C.diag5(), C.view(C.dev["f"]).data_ptr(), x.data_ptr(),
                        1e-12, 50, width, 30, 1e-12, iters.data_ptr(), resid.data_ptr(),
                        status.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    assert C.rel(x, C.gepp()).max() <= 1e-9


# slots of each diagonal outside the matrix (never part of a gradient)
_OUTSIDE = {"a": slice(0, 2), "b": slice(0, 1), "c": slice(0, 0), "d": slice(-1, None),
            "e": slice(-2, None)}


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("stored", [False, True])
@pytest.mark.parametrize("k", [1, 2])
def test_adjoint_writes_stay_inside(band, k, stored, layout, head):
    """band_adjoint, without factors (the transposed system solved as a band system)
    and with factors that band_factor wrote into a guarded buffer: the diagonals'
    gradients, the right-hand side's, the statuses and the workspace."""
    lib = L.load()
    m = L.NPDM if k == 2 else L.NTDM
    C = Case(k, 70, 600, layout, head, seed=50 + 2 * head + k)
    desc = C.desc()
    xc = C.gepp()
    wc = np.random.default_rng(60 + head).uniform(-1.0, 1.0, (C.n, C.nsys))
    x_d, w_d = C.put(xc), C.put(wc)
    factors = None
    if stored:
        factors = C.workspace("factors", lib.band_workspace_size(ct.byref(desc), L.OP_FACTOR,
                                                                 m, 0))
        fst = C.flat_out("factor status", C.nsys, torch.int32)
        assert lib.band_factor(ct.byref(desc), m, C.diag5(), factors.data_ptr(), factors.numel(),
                               fst.data_ptr(), _stream()) == L.OK
    keep = "abcde" if k == 2 else "bcd"
    grads = {q: C.strided_out("grad " + q) for q in keep}
    gf = C.strided_out("grad f")
    status = C.flat_out("status", C.nsys, torch.int32)
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), L.OP_ADJOINT, m, 0))
    G = L.DIAG5(*[(grads[q].data_ptr() if q in grads else None) for q in "abcde"])
    code = lib.band_adjoint(ct.byref(desc), m, factors.data_ptr() if stored else None,
                            C.diag5(), x_d.data_ptr(), w_d.data_ptr(), G, gf.data_ptr(),
                            status.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    got = {q: grads[q].cpu().numpy() for q in grads}
    gfh = gf.cpu().numpy()
    for s in range(0, C.nsys, 7):
        go, gfo, so = oracle.adjoint(k, *[C.system(q, s) for q in "abcde"], xc[:, s], wc[:, s])
        assert so == "OK"
        assert np.abs(gfh[:, s] - gfo).max() <= 1e-10 * np.abs(gfo).max(), s
        for j, q in enumerate("abcde"):
            if q in got:
                mask = np.ones(C.n, dtype=bool)
                mask[_OUTSIDE[q]] = False
                ref = go[j][mask]
                assert np.abs(got[q][mask, s] - ref).max() <= 1e-10 * np.abs(ref).max(), (q, s)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("k", [1, 2])
def test_det_writes_stay_inside(band, k, layout, head):
    """band_det with zero pivots in three systems (the flagged list and the series pass
    in the workspace): mantissas, exponents, statuses."""
    lib = L.load()
    C = Case(k, 70, 600, layout, head, seed=70 + head, plant=("zero_row", (2, 40, 69)))
    desc = C.desc()
    mant = C.flat_out("det_mant", C.nsys, torch.float64)
    ex = C.flat_out("det_exp", C.nsys, torch.int64)
    status = C.flat_out("status", C.nsys, torch.int32)
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), L.OP_DET, 0, 0))
    code = lib.band_det(ct.byref(desc), C.diag5(), mant.data_ptr(), ex.data_ptr(),
                        status.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    mant, ex = mant.cpu().numpy(), ex.cpu().numpy()
    for s in range(C.nsys):
        _, so, dm, dex, _ = oracle.symbolic(k, *[C.system(q, s) for q in "abcdef"])
        assert so == "OK"
        assert np.sign(mant[s]) == np.sign(dm)
        assert abs(np.log2(abs(mant[s])) + ex[s] - (np.log2(abs(dm)) + dex)) <= 1e-12 * C.n, s


@pytest.mark.parametrize("head", HEADS)
def test_batch_writes_stay_inside(band, head):
    """band_solve_batch over four problems of different layouts, methods and schedules
    (NPDM contiguous, NTDM partitioned, SPDM two-sided with zero pivots, SIP), every
    output and workspace guarded."""
    lib = L.load()
    specs = [(Case(2, 70, 600, "contiguous", head, seed=80), L.OP_SOLVE, L.NPDM, "auto"),
             (Case(1, 45, 900, "interleaved", head, seed=81), L.OP_SOLVE, L.NTDM, "partitioned"),
             (Case(2, 100, 300, "interleaved", head, seed=82, plant=("zero_row", (1, 99))),
              L.OP_SOLVE, L.SPDM, "two_sided"),
             (Case(2, 33, 500, "contiguous", head, seed=83), L.OP_SIP, 0, "auto")]
    arr = (L.BandProblem * len(specs))()
    outs = []
    for P, (C, op, m, sched) in zip(arr, specs):
        desc = C.desc(sched)
        x = C.strided_out("x")
        status = C.flat_out("status", C.nsys, torch.int32)
        ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), op, m, 0))
        P.op, P.method, P.desc = op, m, ct.pointer(desc)
        P.diag = C.diag5()
        P.f, P.x, P.sys_status = C.view(C.dev["f"]).data_ptr(), x.data_ptr(), status.data_ptr()
        P.ws, P.ws_bytes = ws.data_ptr(), ws.numel()
        if op == L.OP_SIP:
            iters = C.flat_out("iters", C.nsys, torch.int32)
            resid = C.flat_out("resid", C.nsys, torch.float64)
            P.tol, P.max_it = 1e-12, 50
            P.iters, P.resid = iters.data_ptr(), resid.data_ptr()
        outs.append((desc, x, status))
    assert lib.band_solve_batch(arr, len(specs), _stream()) == L.OK
    for (C, op, m, sched), (desc, x, status) in zip(specs, outs):
        C.check_guards()
        assert (status.cpu() == 0).all(), (m, sched)
        tol = 1e-9 if op == L.OP_SIP else (1e-10 if m == L.SPDM else 1e-12)
        assert C.rel(x, C.gepp()).max() <= tol, (op, m, sched)


@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("method", ["numeric", "symbolic"])
def test_ragged_single_call_writes_stay_inside(band, method, head):
    """band_solve on a ragged packing (n in [16, 3000], TD and PD mixed, one thread per
    system): x, statuses and the workspace guarded; zero pivots planted in three
    systems for the symbolic methods."""
    lib = L.load()
    B = synth.cfg2(nsys=300, nmin=16, nmax=3000, seed_salt=90 + head)
    offs, hbw, total, nsys = B["offsets"], B["hbw"], int(B["offsets"][-1]), B["nsys"]
    if method == "symbolic":
        for s in (0, 150, 299):
            j = int(offs[s]) + 5
            B["a"][j] = B["b"][j] = B["c"][j] = 0.0
        B["f"] = None
        x_true = B["x_true"]
        f = B["c"] * x_true
        for q, sh in (("b", 1), ("d", -1), ("a", 2), ("e", -2)):
            f += B[q] * np.roll(x_true, sh)     # zero slots stop the spill-over
        B["f"] = f
    guard = lambda v: np.concatenate((np.full(head, np.nan), v, np.full(TAIL, np.nan)))
    dev = {q: torch.from_numpy(guard(B[q])).to(DEV) for q in "abcdef"}
    C = Guards()
    x = C.padded_out("x", total, torch.float64, head)
    status = C.flat_out("status", nsys, torch.int32)
    offs_d = torch.from_numpy(offs).to(DEV)
    hbw_d = torch.from_numpy(hbw).to(DEV)
    desc = L.BandDesc(half_bw=2, dtype=L.F64, nsys=nsys, n=int(B["sizes"].max()), sys_stride=0,
                      elem_stride=1, offsets=offs_d.data_ptr(), hbw=hbw_d.data_ptr(),
                      total_rows=total, schedule=L.SCHED_AUTO, chunks=0)
    m = L.AUTO_NUMERIC if method == "numeric" else L.AUTO_SYMBOLIC
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE, m, 0))
    D = L.DIAG5(*[dev[q][head:].data_ptr() for q in "abcde"])
    code = lib.band_solve(ct.byref(desc), m, None, D, dev["f"][head:].data_ptr(),
                          x.data_ptr(), status.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    ref, st, _, _ = oracle.batch("gepp", 2, tuple(B[q] for q in "abcde"), B["f"], nsys, 0, 0, 1,
                                 offsets=offs, hbw=hbw)
    assert (np.asarray(st) == 0).all()
    xg = x.cpu().numpy()
    for s in range(nsys):
        lo, hi = int(offs[s]), int(offs[s + 1])
        rel = np.abs(xg[lo:hi] - ref[lo:hi]).max() / np.abs(ref[lo:hi]).max()
        assert rel <= (1e-12 if method == "numeric" else 1e-10), (s, rel)


@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("schedule", ["thread", "two_sided", "partitioned"])
def test_ragged_plan_writes_stay_inside(band, schedule, head):
    """A ragged packing as size buckets in one band_solve_batch (id lists per bucket):
    the packed x and the per-id statuses guarded."""
    B = synth.cfg2(nsys=300, nmin=16, nmax=3000, seed_salt=95 + head)
    offs, total, nsys = B["offsets"], int(B["offsets"][-1]), B["nsys"]
    guard = lambda v: np.concatenate((np.full(head, np.nan), v, np.full(TAIL, np.nan)))
    dev = {q: torch.from_numpy(guard(B[q])).to(DEV) for q in "abcdef"}
    C = Guards()
    x = C.padded_out("x", total, torch.float64, head)
    status = C.flat_out("status", nsys, torch.int32)
    plan = band.RaggedPlan(*(dev[q][head:head + total] for q in "abcdef"), offs, B["hbw"],
                           schedule=schedule, x=x, status=status)
    plan.run()
    C.check_guards()
    assert (status.cpu() == 0).all()
    xg = x.cpu().numpy()
    err = np.maximum.reduceat(np.abs(xg - B["x_true"]), offs[:-1])
    assert err.max() <= 1e-12


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", [1, 4])
@pytest.mark.parametrize("flags", [0, L.REFINE_PAIRS])
def test_refine_writes_stay_inside(band, flags, layout, head):
    """band_refine_solve_ex (FP32 factorisation, FP64 or pair residuals): x, the step
    counts, statuses and the workspace guarded; FP32 diagonals with heads of one and
    four elements (off and on the 16-byte boundary)."""
    lib = L.load()
    nsys, n = 70, 600
    rng = np.random.default_rng(100 + head + flags)
    D = synth.dominant(rng, nsys, n, k=2)
    D = {q: np.asarray(D[q], dtype=np.float32).astype(np.float64) for q in "abcde"}
    xt = rng.uniform(-1.0, 1.0, size=(n, nsys))
    f = synth.band_matvec(2, D["a"], D["b"], D["c"], D["d"], D["e"], xt)
    C = Case(2, nsys, n, layout, head, data=(D, f))
    d32 = {q: torch.from_numpy(C.host[q].astype(np.float32)).to(DEV) for q in "abcde"}
    diag32 = L.DIAG5(*[C.view(d32[q]).data_ptr() for q in "abcde"])
    desc = C.desc()
    desc.dtype = L.F32
    x = C.strided_out("x")
    steps = C.flat_out("steps", nsys, torch.int32)
    status = C.flat_out("status", nsys, torch.int32)
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), L.OP_REFINE, 0, 0))
    code = lib.band_refine_solve_ex(ct.byref(desc), diag32, C.view(C.dev["f"]).data_ptr(),
                                    x.data_ptr(), 1e-11, 10, flags, steps.data_ptr(),
                                    status.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    assert C.rel(x, C.gepp()).max() <= 1e-10


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("nx,ny", [(16, 12), (40, 6)])
def test_sip2d_writes_stay_inside(band, nx, ny, layout, head):
    """band_sip2d (a warp per system for nx <= 32, a thread per system beyond): x,
    iteration counts, residuals, statuses and the workspace guarded."""
    lib = L.load()
    nsys, N = 40, nx * ny
    rng = np.random.default_rng(110 + nx + head)
    r = rng.uniform(0.5, 4.0, nsys)[None, :]
    G = {q: -r * rng.uniform(0.5, 1.5, (N, nsys)) for q in "swet"}
    G["c"] = 1 + 4 * r + rng.uniform(0, 0.1, (N, nsys))
    f = rng.uniform(-1, 1, (N, nsys))
    # the five diagonals in the order band_sip2d takes them: s, w, c, e, t
    C = Case(2, nsys, N, layout, head, data=(dict(zip("abcde", (G[q] for q in "swcet"))), f))
    desc = C.desc()
    x = C.strided_out("x")
    iters = C.flat_out("iters", nsys, torch.int32)
    resid = C.flat_out("resid", nsys, torch.float64)
    status = C.flat_out("status", nsys, torch.int32)
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), L.OP_SIP2D, 0, 0))
    code = lib.band_sip2d(ct.byref(desc), nx, C.diag5(), C.view(C.dev["f"]).data_ptr(),
                          x.data_ptr(), 1e-10, 500, iters.data_ptr(), resid.data_ptr(),
                          status.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    xg = x.cpu().numpy()
    for s in range(0, nsys, 5):
        R = oracle.sip2d(nx, ny, *[G[q][:, s] for q in "swcet"], f[:, s], tol=1e-10, max_it=500)
        assert R["status"] == "OK"
        assert np.abs(xg[:, s] - R["x"]).max() <= 1e-9 * np.abs(R["x"]).max(), s


@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("n", [40, 129])
@pytest.mark.parametrize("k", [1, 2])
def test_adi_step_writes_stay_inside(band, k, n, head):
    """band_adi_step (its right-hand side and diagonal kernels and both sweeps' solves on
    the automatic schedule): u, the 2n line statuses and the workspace guarded."""
    lib = L.load()
    rng = np.random.default_rng(120 + n + k + head)
    u0 = rng.uniform(0, 1, (n, n))
    src = rng.uniform(-1, 1, (n, n))
    guard = lambda v, fill: np.concatenate((np.full(head, fill), v.reshape(-1),
                                            np.full(TAIL, fill)))
    C = Guards()
    u = C.padded_out("u", n * n, torch.float64, head)
    u.copy_(torch.from_numpy(u0.reshape(-1)))
    sbuf = torch.from_numpy(guard(src, np.nan)).to(DEV)
    status = C.flat_out("status", 2 * n, torch.int32)
    grid = L.BandDesc(half_bw=k, dtype=L.F64, nsys=n, n=n, sys_stride=1, elem_stride=1,
                      offsets=None, hbw=None, total_rows=0, schedule=0, chunks=0)
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(grid), L.OP_ADI, 0, 0))
    tau, lam = 0.01, 2.0
    code = lib.band_adi_step(ct.byref(grid), tau, lam, sbuf[head:].data_ptr(), u.data_ptr(),
                             status.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    uo, st = oracle.adi_step(u0, tau, lam, src, k=k)
    assert (np.asarray(st) == 0).all()
    ug = u.cpu().numpy().reshape(n, n)
    assert np.abs(ug - uo).max() <= 1e-12 * np.abs(uo).max()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("head", HEADS)
@pytest.mark.parametrize("schedule", ["auto", "thread"])
def test_mnpdm_writes_stay_inside(band, schedule, layout, head):
    """MNPDM on PD systems whose outer diagonals are nonzero on 5 % of the rows: the
    row-parallel path (its copies of the diagonals, the skip list and NTDM's workspace)
    and one thread per system."""
    lib = L.load()
    nsys, n = 70, 600
    rng = np.random.default_rng(130 + head)
    D = synth.dominant(rng, nsys, n, k=2)
    keep = rng.random((n, nsys)) < 0.05
    keep[2, :] = keep[n - 3, :] = True
    D["a"] = np.where(keep, D["a"], 0.0)
    D["e"] = np.where(keep, D["e"], 0.0)
    D["a"][:2] = 0.0
    D["e"][n - 2:] = 0.0
    D["c"] = 1.0 + sum(np.abs(D[q]) for q in "abde")
    xt = rng.uniform(-1.0, 1.0, size=(n, nsys))
    f = synth.band_matvec(2, D["a"], D["b"], D["c"], D["d"], D["e"], xt)
    C = Case(2, nsys, n, layout, head, data=(D, f))
    desc = C.desc(schedule)
    x = C.strided_out("x")
    status = C.flat_out("status", nsys, torch.int32)
    ws = C.workspace("workspace", lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE, L.MNPDM, 0))
    code = lib.band_solve(ct.byref(desc), L.MNPDM, None, C.diag5(),
                          C.view(C.dev["f"]).data_ptr(), x.data_ptr(), status.data_ptr(),
                          ws.data_ptr(), ws.numel(), _stream())
    assert code == L.OK
    C.check_guards()
    assert (status.cpu() == 0).all()
    assert C.rel(x, C.gepp()).max() <= 1e-11
