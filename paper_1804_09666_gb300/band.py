"""Python API over torch CUDA tensors; marshals arguments to libband's C ABI.

Uniform batches: every per-row array is a tensor of shape (n, nsys) whose element
[i, s] is row i of system s; all arrays of one call share the same strides, so a
contiguous (n, nsys) tensor is the interleaved layout and ``t.T`` of a contiguous
(nsys, n) tensor is the contiguous-systems layout.  Ragged batches use 1-D packed
tensors plus device offsets (see ``solve_ragged``).

The workspaces are torch tensors allocated here; the C library allocates nothing.
Calls run on torch's current CUDA stream and return without synchronising.
"""
import ctypes as ct

import torch

from . import _lib as L

_METHODS = {"ntdm": L.NTDM, "npdm": L.NPDM, "stdm": L.STDM, "spdm": L.SPDM,
            "auto": L.AUTO_NUMERIC, "auto_symbolic": L.AUTO_SYMBOLIC, "mnpdm": L.MNPDM}


def status_names(status):
    """Map a status tensor / list of codes to names."""
    vals = status.tolist() if hasattr(status, "tolist") else list(status)
    return [L.STATUS_NAMES.get(int(v), str(v)) for v in vals]


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None else ct.c_void_p(0)


def _dtype_code(t):
    if t.dtype == torch.float64:
        return L.F64
    if t.dtype == torch.float32:
        return L.F32
    raise TypeError("band arrays must be float64 or float32, got %s" % t.dtype)


_SCHEDULES = {"auto": L.SCHED_AUTO, "thread": L.SCHED_THREAD, "two_sided": L.SCHED_TWO_SIDED,
              "partitioned": L.SCHED_PARTITIONED, "grid": L.SCHED_GRID}


def desc_for(ref, half_bw, schedule="auto", chunks=0):
    """BandDesc for (n, nsys)-shaped tensors with ref's strides."""
    if ref.dim() != 2:
        raise ValueError("expected a (n, nsys) tensor")
    n, nsys = ref.shape
    return L.BandDesc(half_bw=half_bw, dtype=_dtype_code(ref), nsys=nsys, n=n,
                      sys_stride=ref.stride(1) if nsys > 1 else max(n, 1),
                      elem_stride=ref.stride(0) if n > 1 else max(nsys, 1),
                      offsets=None, hbw=None, total_rows=0, schedule=_SCHEDULES[schedule],
                      chunks=chunks)


def _check_same(ref, *ts):
    """ref and every given array share shape, strides, dtype and CUDA device."""
    for t in ts:
        if t is None:
            continue
        if t.shape != ref.shape or t.stride() != ref.stride() or t.dtype != ref.dtype:
            raise ValueError("all band arrays must share shape, strides and dtype")
    if not ref.is_cuda:
        raise ValueError("band arrays must be CUDA tensors")
    _on_device(ref.device, **{"band array %d" % i: t for i, t in enumerate(ts)})


def _on_device(dev, **named):
    """Every given tensor is a CUDA tensor on device dev: the kernels take raw device
    pointers, and a host pointer would fault on the GPU instead of failing here."""
    for name, t in named.items():
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device != dev:
            raise ValueError("%s must be a CUDA tensor on %s" % (name, dev))


def _status_out(status, nsys, dev):
    """The per-system status output: given (int32, contiguous, at least nsys entries) or
    allocated."""
    if status is None:
        return torch.empty(nsys, dtype=torch.int32, device=dev)
    _on_device(dev, status=status)
    if status.dtype != torch.int32 or not status.is_contiguous() or status.numel() < nsys:
        raise ValueError("status must be a contiguous int32 tensor of at least nsys entries")
    return status


def _bytes(t):
    return t.numel() * t.element_size()


def _diag5(a, b, c, d, e):
    return L.DIAG5(*[(t.data_ptr() if t is not None else None) for t in (a, b, c, d, e)])


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def solve(a, b, c, d, e, f, method="npdm", x=None, status=None, factors=None, ws=None,
          schedule="auto", chunks=0):
    """Solve A x = f for a uniform batch.  Returns (x, status int32[nsys]).

    method: "npdm", "ntdm", "spdm", "stdm", "mnpdm" (PD systems with few nonzero outer
    entries).  a, e are ignored (may be None) for TD.
    factors: a buffer from ``factor`` to reuse a factorisation (numeric methods).
    schedule: "auto", "thread" (one thread per system), "two_sided" (two threads per
    system meeting in the middle), "partitioned" (``chunks`` lanes per system, 8, 16,
    32, 64, 128 or 256, 0 = chosen by the library) or "grid" (one system, or a few,
    over the whole GPU; numeric methods); the last three without factors.
    """
    lib = L.load()
    m = _METHODS[method]
    half_bw = 1 if method in ("ntdm", "stdm") else 2
    _check_same(c, a if half_bw == 2 else None, b, d, e if half_bw == 2 else None, f)
    _on_device(c.device, factors=factors, ws=ws)
    desc = desc_for(c, half_bw, schedule, chunks)
    if x is None:
        x = torch.empty_strided(c.shape, c.stride(), dtype=c.dtype, device=c.device)
    _check_same(c, x)
    status = _status_out(status, c.shape[1], c.device)
    if factors is not None and _bytes(factors) < lib.band_workspace_size(ct.byref(desc),
                                                                         L.OP_FACTOR, m, 0):
        raise ValueError("factors is smaller than this batch's factorisation")
    need = lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE, m, 0)
    if ws is None or _bytes(ws) < need:
        ws = _workspace(need, c.device)
    code = lib.band_solve(ct.byref(desc), m, _ptr(factors), _diag5(a, b, c, d, e), _ptr(f), _ptr(x),
                          _ptr(status), _ptr(ws), _bytes(ws), _stream())
    L.check(code, "band_solve")
    return x, status


def det(a, b, c, d, e, half_bw=2, status=None):
    """Determinant of every system of a uniform FP64 batch (Sec. 3.2, Remark 1).

    Returns (mant float64[nsys], exp int64[nsys], status int32[nsys]) with
    det = mant * 2**exp; systems whose factorisation meets an exact zero pivot take the
    symbolic limit (status SINGULAR when it is 0).  a, e are ignored for half_bw 1.
    """
    lib = L.load()
    _check_same(c, a if half_bw == 2 else None, b, d, e if half_bw == 2 else None)
    if c.dtype != torch.float64:
        raise ValueError("band_det takes float64 diagonals")
    desc = desc_for(c, half_bw)
    nsys = c.shape[1]
    mant = torch.empty(nsys, dtype=torch.float64, device=c.device)
    ex = torch.empty(nsys, dtype=torch.int64, device=c.device)
    status = _status_out(status, nsys, c.device)
    ws = _workspace(lib.band_workspace_size(ct.byref(desc), L.OP_DET, 0, 0), c.device)
    code = lib.band_det(ct.byref(desc), _diag5(a, b, c, d, e), _ptr(mant), _ptr(ex), _ptr(status),
                        _ptr(ws), _bytes(ws), _stream())
    L.check(code, "band_det")
    return mant, ex, status


def slogdet(a, b, c, d, e, half_bw=2):
    """(sign, log|det|, status) of every system, as torch.linalg.slogdet reports it
    (sign 0 and log|det| = -inf for a singular system)."""
    mant, ex, status = det(a, b, c, d, e, half_bw)
    sign = torch.sign(mant)
    logabs = torch.log(mant.abs()) + ex.to(torch.float64) * 0.6931471805599453
    return sign, logabs, status


def sip2d(s, w, c, e, t, f, nx, tol=1e-10, max_it=500, x=None):
    """Stone's method on a batch of 2-D five-point systems (band_sip2d): (n, nsys)
    float64 tensors with n = nx * ny, unknown k = y nx + x; s, w, c, e, t the entries at
    columns k - nx, k - 1, k, k + 1, k + nx.  Returns (x, iters, resid, status)."""
    lib = L.load()
    _check_same(c, s, w, e, t, f)
    if c.dtype != torch.float64:
        raise ValueError("band_sip2d takes float64 arrays")
    desc = desc_for(c, 2)
    if x is None:
        x = torch.empty_strided(c.shape, c.stride(), dtype=c.dtype, device=c.device)
    _check_same(c, x)
    nsys = c.shape[1]
    iters = torch.empty(nsys, dtype=torch.int32, device=c.device)
    resid = torch.empty(nsys, dtype=torch.float64, device=c.device)
    status = torch.empty(nsys, dtype=torch.int32, device=c.device)
    ws = _workspace(lib.band_workspace_size(ct.byref(desc), L.OP_SIP2D, 0, 0), c.device)
    code = lib.band_sip2d(ct.byref(desc), int(nx), _diag5(s, w, c, e, t), _ptr(f), _ptr(x),
                          float(tol), int(max_it), _ptr(iters), _ptr(resid), _ptr(status),
                          _ptr(ws), _bytes(ws), _stream())
    L.check(code, "band_sip2d")
    return x, iters, resid, status


class AdiStepper:
    """Time steps of u_t = u_xx + u_yy + lam u (1 - u) + s on an n x n grid (Peaceman-
    Rachford ADI; band_adi_step): u is an (n, n) float64 CUDA tensor, u[y, x], updated
    in place.  half_bw 1: 3-point stencil (NTDM lines), 2: fourth-order 5-point stencil
    (NPDM lines).  The workspace is allocated once here, so ``step`` only launches and a
    number of steps can be captured in a CUDA graph.  ``status`` holds the 2n line
    statuses of the last step (rows, then columns)."""

    def __init__(self, n, tau, lam=1.0, source=None, half_bw=2, device=None):
        lib = L.load()
        self.lib = lib
        self.desc = L.BandDesc(half_bw=half_bw, dtype=L.F64, nsys=n, n=n, sys_stride=1,
                               elem_stride=1, offsets=None, hbw=None, total_rows=0,
                               schedule=0, chunks=0)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        if source is not None:
            _on_device(dev, source=source)
            if source.dtype != torch.float64 or not source.is_contiguous() or \
                    source.numel() != n * n:
                raise ValueError("source must be a contiguous float64 (n, n) tensor")
        self.n, self.tau, self.lam, self.source = n, float(tau), float(lam), source
        need = lib.band_workspace_size(ct.byref(self.desc), L.OP_ADI, 0, 0)
        if need == 0:
            raise ValueError("bad grid for band_adi_step")
        self.ws = _workspace(need, dev)
        self.status = torch.empty(2 * n, dtype=torch.int32, device=dev)
        self.device = dev

    def step(self, u, steps=1):
        if not (u.is_cuda and u.device == self.device and u.dtype == torch.float64 and
                u.is_contiguous() and u.numel() == self.n * self.n):
            raise ValueError("u must be a contiguous float64 (n, n) tensor on the stepper's device")
        for _ in range(steps):
            code = self.lib.band_adi_step(ct.byref(self.desc), self.tau, self.lam,
                                          _ptr(self.source), _ptr(u), _ptr(self.status),
                                          _ptr(self.ws), _bytes(self.ws), _stream())
            L.check(code, "band_adi_step")
        return u


def factor(a, b, c, d, e, method="npdm", status=None):
    """LU factors (opaque uint8 buffer) for repeated solves and the adjoint."""
    lib = L.load()
    m = _METHODS[method]
    half_bw = 1 if method == "ntdm" else 2
    _check_same(c, a if half_bw == 2 else None, b, d, e if half_bw == 2 else None)
    desc = desc_for(c, half_bw)
    need = lib.band_workspace_size(ct.byref(desc), L.OP_FACTOR, m, 0)
    buf = _workspace(need, c.device)
    status = _status_out(status, c.shape[1], c.device)
    code = lib.band_factor(ct.byref(desc), m, _diag5(a, b, c, d, e), _ptr(buf), buf.numel(),
                           _ptr(status), _stream())
    L.check(code, "band_factor")
    return buf, status


def solve_ragged(a, b, c, d, e, f, offsets, hbw, n_max, total_rows, method="auto", x=None,
                 status=None, ws=None):
    """Ragged batch: 1-D packed arrays, system s in rows offsets[s]..offsets[s+1]-1.

    offsets: int64 CUDA tensor (nsys+1); hbw: int8 CUDA tensor of 1/2 per system (or None
    with method "npdm"/"ntdm"); n_max: an upper bound on the system sizes; total_rows:
    offsets[-1] as a Python int.
    """
    lib = L.load()
    m = _METHODS[method]
    dev = c.device
    _on_device(dev, a=a, b=b, c=c, d=d, e=e, f=f, offsets=offsets, hbw=hbw, x=x, ws=ws)
    for name, t in (("a", a), ("b", b), ("d", d), ("e", e), ("f", f), ("x", x)):
        if t is not None and (t.dtype != c.dtype or t.dim() != 1 or not t.is_contiguous()
                              or t.numel() < int(total_rows)):
            raise ValueError("%s must be a contiguous 1-D tensor of c's dtype with at least "
                             "total_rows entries" % name)
    if c.dim() != 1 or not c.is_contiguous() or c.numel() < int(total_rows):
        raise ValueError("c must be a contiguous 1-D tensor with at least total_rows entries")
    if offsets.dtype != torch.int64 or hbw is not None and hbw.dtype != torch.int8:
        raise ValueError("offsets must be int64 and hbw int8")
    nsys = offsets.numel() - 1
    desc = L.BandDesc(half_bw=1 if method in ("ntdm", "stdm") else 2, dtype=_dtype_code(c),
                      nsys=nsys, n=int(n_max), sys_stride=0, elem_stride=1,
                      offsets=offsets.data_ptr(), hbw=hbw.data_ptr() if hbw is not None else None,
                      total_rows=int(total_rows))
    if x is None:
        x = torch.empty_like(f)
    status = _status_out(status, nsys, dev)
    need = lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE, m, 0)
    if ws is None or _bytes(ws) < need:
        ws = _workspace(need, dev)
    code = lib.band_solve(ct.byref(desc), m, None, _diag5(a, b, c, d, e), _ptr(f), _ptr(x),
                          _ptr(status), _ptr(ws), _bytes(ws), _stream())
    L.check(code, "band_solve")
    return x, status


def sip(a, b, c, d, e, f, tol=1e-10, max_it=200, width=5, hb_max_it=30, hb_tol=1e-12, x=None,
        schedule="auto"):
    """SIP / Stone method (FP64).  Returns (x, iters, resid, status).

    schedule applies to width 0 (Algorithm 1 with exact substitutions): "two_sided" runs
    the first update with two threads per system, "thread" with one, "auto" picks.
    """
    lib = L.load()
    _check_same(c, a, b, d, e, f)
    desc = desc_for(c, 2, schedule)
    if x is None:
        x = torch.empty_strided(c.shape, c.stride(), dtype=c.dtype, device=c.device)
    _check_same(c, x)
    nsys = c.shape[1]
    iters = torch.empty(nsys, dtype=torch.int32, device=c.device)
    resid = torch.empty(nsys, dtype=torch.float64, device=c.device)
    status = torch.empty(nsys, dtype=torch.int32, device=c.device)
    need = lib.band_workspace_size(ct.byref(desc), L.OP_SIP, 0, width)
    ws = _workspace(need, c.device)
    code = lib.band_sip(ct.byref(desc), _diag5(a, b, c, d, e), _ptr(f), _ptr(x), tol, max_it,
                        width, hb_max_it, hb_tol, _ptr(iters), _ptr(resid), _ptr(status), _ptr(ws),
                        ws.numel(), _stream())
    L.check(code, "band_sip")
    return x, iters, resid, status


def refine_solve(a32, b32, c32, d32, e32, f, rel_stop=1e-11, max_steps=10, x=None,
                 schedule="auto", chunks=0, pairs=False):
    """FP32 solve + refinement to FP64 accuracy; f, x float64 with the diagonals'
    strides.  The residual and the update are FP64 (pairs=False; x must not be f) or
    FP32 pairs (pairs=True).  The FP32 solves run on `schedule` / `chunks` as in
    ``solve``."""
    lib = L.load()
    _check_same(c32, a32, b32, d32, e32)
    if c32.dtype != torch.float32:
        raise ValueError("the diagonals must be float32")
    desc = desc_for(c32, 2 if a32 is not None else 1, schedule, chunks)
    if x is None:
        x = torch.empty_strided(c32.shape, c32.stride(), dtype=torch.float64, device=c32.device)
    for name, t in (("f", f), ("x", x)):
        _on_device(c32.device, **{name: t})
        if t.shape != c32.shape or t.stride() != c32.stride() or t.dtype != torch.float64:
            raise ValueError("%s must be float64 with the diagonals' shape and strides" % name)
    nsys = c32.shape[1]
    steps = torch.empty(nsys, dtype=torch.int32, device=c32.device)
    status = torch.empty(nsys, dtype=torch.int32, device=c32.device)
    need = lib.band_workspace_size(ct.byref(desc), L.OP_REFINE, 0, 0)
    ws = _workspace(need, c32.device)
    code = lib.band_refine_solve_ex(ct.byref(desc), _diag5(a32, b32, c32, d32, e32), _ptr(f),
                                    _ptr(x), rel_stop, max_steps, L.REFINE_PAIRS if pairs else 0,
                                    _ptr(steps), _ptr(status), _ptr(ws), ws.numel(), _stream())
    L.check(code, "band_refine_solve")
    return x, steps, status


def adjoint(a, b, c, d, e, x, w, factors=None, method="npdm", schedule="auto", chunks=0):
    """Gradients (ga, gb, gc, gd, ge), gf of sum(w * x) with x = A^{-1} f.  Without
    factors the transposed system is solved on `schedule` / `chunks` as in ``solve``."""
    lib = L.load()
    m = _METHODS[method]
    half_bw = 1 if method == "ntdm" else 2
    _check_same(c, a if half_bw == 2 else None, b, d, e if half_bw == 2 else None, x, w)
    _on_device(c.device, factors=factors)
    desc = desc_for(c, half_bw, schedule, chunks)
    if factors is not None and _bytes(factors) < lib.band_workspace_size(ct.byref(desc),
                                                                         L.OP_FACTOR, m, 0):
        raise ValueError("factors is smaller than this batch's factorisation")
    mk = lambda: torch.empty_strided(c.shape, c.stride(), dtype=c.dtype, device=c.device)
    grads = [mk() if (half_bw == 2 or k in (1, 2, 3)) else None for k in range(5)]
    gf = mk()
    status = torch.empty(c.shape[1], dtype=torch.int32, device=c.device)
    need = lib.band_workspace_size(ct.byref(desc), L.OP_ADJOINT, m, 0)
    ws = _workspace(need, c.device)
    code = lib.band_adjoint(ct.byref(desc), m, _ptr(factors), _diag5(a, b, c, d, e), _ptr(x), _ptr(w),
                            L.DIAG5(*[(g.data_ptr() if g is not None else None) for g in grads]),
                            _ptr(gf), _ptr(status), _ptr(ws), ws.numel(), _stream())
    L.check(code, "band_adjoint")
    return tuple(grads), gf, status


class BatchPlan:
    """Several independent solves in one batched launch (band_solve_batch).

    specs: list of dicts with keys
      op      "solve" (default) or "sip" (Algorithm 1, exact substitutions)
      method  for "solve": "npdm", "ntdm", "spdm", "stdm"
      a, b, c, d, e, f   (n, nsys) tensors with equal strides (a, e None for TD)
      x       optional output tensor
      tol, max_it        for "sip"
      schedule           "auto" (default), "thread", "two_sided", "partitioned" (for
                         "sip": the first update of Algorithm 1, not partitioned)
      chunks             lanes per system on the partitioned schedule (0: the library's)
    Outputs, statuses and workspaces are allocated once here; ``run()`` only launches,
    so a run can be captured in a CUDA graph.  results[i] holds x, status (and iters,
    resid for "sip").  tune: band_autotune picks thread or two-sided for every "solve"
    spec left on "auto", then moves diagonally dominant problems to the partitioned
    schedule while that shortens the whole launch (BAND_TUNE_JOINT); the trial runs
    overwrite the outputs.  ``schedules`` / ``chunks`` hold the schedules in use.
    """

    def __init__(self, specs, tune=False, reps=3):
        lib = L.load()
        if len(specs) > L.MAX_BATCH:
            raise ValueError("at most %d problems per batch" % L.MAX_BATCH)
        self.lib = lib
        self.keep = []
        self.results = []
        self.arr = (L.BandProblem * max(len(specs), 1))()
        for i, sp in enumerate(specs):
            op = sp.get("op", "solve")
            a, b, c, d, e, f = (sp.get(k) for k in "abcdef")
            if op == "solve":
                m = _METHODS[sp.get("method", "npdm")]
                half_bw = 1 if sp.get("method") in ("ntdm", "stdm") else 2
                opc = L.OP_SOLVE
            elif op == "sip":
                m, half_bw, opc = 0, 2, L.OP_SIP
            else:
                raise ValueError(op)
            _check_same(c, a if half_bw == 2 else None, b, d, e if half_bw == 2 else None, f)
            desc = desc_for(c, half_bw, sp.get("schedule", "auto"), sp.get("chunks", 0))
            x = sp.get("x")
            if x is None:
                x = torch.empty_strided(c.shape, c.stride(), dtype=c.dtype, device=c.device)
            _check_same(c, x)
            status = torch.empty(c.shape[1], dtype=torch.int32, device=c.device)
            need = lib.band_workspace_size(ct.byref(desc), opc, m, 0)
            if tune and op == "solve" and desc.schedule == L.SCHED_AUTO:
                dp = L.BandDesc.from_buffer_copy(desc)      # room for the partitioned schedule
                dp.schedule, dp.chunks = L.SCHED_PARTITIONED, 0
                need = max(need, lib.band_workspace_size(ct.byref(dp), opc, m, 0))
            ws = _workspace(need, c.device)
            res = dict(x=x, status=status)
            P = self.arr[i]
            P.op, P.method = opc, m
            P.desc = ct.pointer(desc)
            P.diag = _diag5(a, b, c, d, e)
            P.f, P.x, P.sys_status = f.data_ptr(), x.data_ptr(), status.data_ptr()
            P.ws, P.ws_bytes = ws.data_ptr(), ws.numel()
            if op == "sip":
                iters = torch.empty(c.shape[1], dtype=torch.int32, device=c.device)
                resid = torch.empty(c.shape[1], dtype=torch.float64, device=c.device)
                P.tol, P.max_it = sp.get("tol", 1e-10), sp.get("max_it", 200)
                P.iters, P.resid = iters.data_ptr(), resid.data_ptr()
                res.update(iters=iters, resid=resid)
            self.keep.append((desc, a, b, c, d, e, f, ws))
            self.results.append(res)
        self.count = len(specs)
        self.descs = [k[0] for k in self.keep]
        if tune and self.count > 0:
            out = (ct.c_int32 * self.count)()
            outc = (ct.c_int32 * self.count)()
            code = lib.band_autotune(self.arr, self.count, reps, L.TUNE_JOINT, out, outc, _stream())
            L.check(code, "band_autotune")
            for desc, v, pc in zip(self.descs, out, outc):
                desc.schedule, desc.chunks = v, pc
        self.schedules = [d.schedule for d in self.descs]
        self.chunks = [d.chunks for d in self.descs]

    def run(self):
        code = self.lib.band_solve_batch(self.arr, self.count, _stream())
        L.check(code, "band_solve_batch")
        return self.results


class RaggedPlan:
    """A ragged packing solved as size buckets in one batched launch (band_plan_ragged).

    a, b, c, d, e, f: 1-D device tensors of the packed rows (system s in rows
    offsets[s] .. offsets[s+1]-1; the a, e rows of TD systems are not read).
    offsets: host int64 array (nsys + 1); hbw: host int8 array of 1/2 per system, or None
    with half_bw for all.  method: "numeric" (NTDM/NPDM per bucket) or "symbolic"
    (STDM/SPDM).  schedule: "auto", "thread", "two_sided", "partitioned" (``chunks``
    lanes per system, 0 = the library's choice), or "tune": band_autotune picks thread
    or two-sided per bucket, then moves the buckets of the longest systems to the
    partitioned schedule while that shortens the whole launch (BAND_TUNE_JOINT).  The
    buckets' workspaces are allocated here; run() only launches (graph-capturable).  x is
    packed like f; status holds one entry per system id.
    """

    def __init__(self, a, b, c, d, e, f, offsets, hbw=None, half_bw=2, method="numeric",
                 schedule="auto", x=None, status=None, reps=3, chunks=0):
        import numpy as np
        lib = L.load()
        self.lib = lib
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        nsys = len(offs) - 1
        hb = None if hbw is None else np.ascontiguousarray(np.asarray(hbw, dtype=np.int8))
        order = np.empty(max(nsys, 1), dtype=np.int64)
        buckets = (L.BandBucket * L.MAX_BATCH)()
        nb = lib.band_plan_ragged(offs.ctypes.data, hb.ctypes.data if hb is not None else None,
                                  half_bw, nsys, order.ctypes.data, buckets, L.MAX_BATCH)
        if nb < 0:
            raise ValueError("band_plan_ragged: bad sizes or bandwidths, or more than %d buckets"
                             % L.MAX_BATCH)
        dev = f.device
        _on_device(dev, a=a, b=b, c=c, d=d, e=e, f=f, x=x)
        rows = int(offs[-1]) if nsys > 0 else 0
        for name, t in (("a", a), ("b", b), ("c", c), ("d", d), ("e", e), ("f", f), ("x", x)):
            if t is not None and (t.dtype != f.dtype or t.dim() != 1 or not t.is_contiguous()
                                  or t.numel() < rows):
                raise ValueError("%s must be a contiguous 1-D tensor of f's dtype with at "
                                 "least offsets[-1] entries" % name)
        self.order = torch.from_numpy(order[:nsys].copy()).to(dev)
        self.offsets = torch.from_numpy(offs).to(dev)
        self.buckets = [(bk.first, bk.count, bk.n_max, bk.half_bw) for bk in buckets[:nb]]
        self.x = x if x is not None else torch.empty_like(f)
        self.status = _status_out(status, nsys, dev)
        sched = "auto" if schedule == "tune" else schedule
        self.descs, self.keep = [], [a, b, c, d, e, f]
        self.arr = (L.BandProblem * max(nb, 1))()
        for i, (first, count, n_max, k) in enumerate(self.buckets):
            desc = L.BandDesc(half_bw=k, dtype=_dtype_code(f), nsys=count, n=n_max, sys_stride=0,
                              elem_stride=1, offsets=self.offsets.data_ptr(), hbw=None,
                              total_rows=int(offs[-1]), schedule=_SCHEDULES[sched],
                              chunks=chunks if sched == "partitioned" else 0,
                              systems=self.order.data_ptr() + 8 * first)
            name = ("npdm" if k == 2 else "ntdm") if method == "numeric" else \
                   ("spdm" if k == 2 else "stdm")
            m = _METHODS[name]
            need = lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE, m, 0)
            if schedule == "tune":      # room for the partitioned schedule too
                dp = L.BandDesc.from_buffer_copy(desc)
                dp.schedule, dp.chunks = L.SCHED_PARTITIONED, 0
                need = max(need, lib.band_workspace_size(ct.byref(dp), L.OP_SOLVE, m, 0))
            ws = _workspace(need, dev)
            P = self.arr[i]
            P.op, P.method = L.OP_SOLVE, m
            P.desc = ct.pointer(desc)
            P.diag = _diag5(a if k == 2 else None, b, c, d, e if k == 2 else None)
            P.f, P.x, P.sys_status = f.data_ptr(), self.x.data_ptr(), self.status.data_ptr()
            P.ws, P.ws_bytes = ws.data_ptr(), ws.numel()
            self.descs.append(desc)
            self.keep.append(ws)
        self.count = nb
        self.schedules = [d.schedule for d in self.descs]
        self.chunks = [d.chunks for d in self.descs]
        if schedule == "tune" and nb > 0:
            out = (ct.c_int32 * nb)()
            outc = (ct.c_int32 * nb)()
            code = lib.band_autotune(self.arr, nb, reps, L.TUNE_JOINT, out, outc, _stream())
            L.check(code, "band_autotune")
            for desc, v, pc in zip(self.descs, out, outc):
                desc.schedule, desc.chunks = v, pc
            self.schedules = list(out)
            self.chunks = list(outc)

    def run(self):
        code = self.lib.band_solve_batch(self.arr, self.count, _stream())
        L.check(code, "band_solve_batch")
        return self.x, self.status


def solve_batch(specs):
    """One-shot batched solve; see BatchPlan.  Returns the list of results."""
    return BatchPlan(specs).run()


class BandSolve(torch.autograd.Function):
    """x = A^{-1} f for a batch of PD systems (NPDM forward, hand-written adjoint backward).

    Inputs: a, b, c, d, e, f of shape (n, nsys), float64 CUDA, equal strides.
    """

    @staticmethod
    def forward(ctx, a, b, c, d, e, f):
        x, status = solve(a, b, c, d, e, f, method="npdm")
        ctx.save_for_backward(a, b, c, d, e, x)
        ctx.mark_non_differentiable(status)
        return x, status

    @staticmethod
    def backward(ctx, gx, gstatus=None):
        a, b, c, d, e, x = ctx.saved_tensors
        w = gx
        if w.stride() != c.stride():
            w = torch.empty_strided(c.shape, c.stride(), dtype=c.dtype, device=c.device).copy_(gx)
        (ga, gb, gc, gd, ge), gf, _ = adjoint(a, b, c, d, e, x, w)
        return ga, gb, gc, gd, ge, gf
