"""FP64 CPU oracle for the batched band solvers -- TEST INFRASTRUCTURE ONLY.

(FP64 throughout, except the Laurent-series pass of STDM/SPDM, whose coefficients are
double-double so that exact cancellations can be told from rounding residue.)

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It is independent of the CUDA library: it shares no code,
header, table or constant with it, and neither side imports the other.  Its
arithmetic lives in ``band_oracle.c`` (plain C, compiled ``-O2
-ffp-contract=off``) and, for exact rational checks on tiny systems, in
``exact.py``.

Method names and readings follow Veneva & Ayriyan, arXiv:1804.09666:
NTDM/NPDM (R1/R2, Sec. 1, Table 7), MNPDM (R2m, Sec. 1 and Sec. 3.2 Remark 2),
STDM/SPDM (R3, Sec. 1 and Sec. 3.2
Remark 1), ILU(0) (R4, Sec. 2), Hotelling-Bodewig (R5, Eq. (1)), SIP
(R6, Algorithm 1), FP32 + refinement (R7) and the adjoint (R8).

Arrays: one system = 1-D float64 arrays of length n (diagonals a, b, c, d, e as
A[i][i-2], A[i][i-1], A[i][i], A[i][i+1], A[i][i+2]; right-hand side f).
"""
import ctypes as _ct
import os as _os

import numpy as _np

from . import build as _build

STATUS = {
    0: "OK",
    1: "ARG",
    3: "ZERO_PIVOT",
    4: "SINGULAR",
    5: "NONFINITE",
    6: "NOT_CONVERGED",
    7: "SYMBOLIC_RANGE",
    10: "NOMEM",
}

_lib = None
_D = _ct.POINTER(_ct.c_double)
_F = _ct.POINTER(_ct.c_float)
_I64 = _ct.POINTER(_ct.c_int64)
_I32 = _ct.POINTER(_ct.c_int32)
_I8 = _ct.POINTER(_ct.c_int8)
_LL = _ct.POINTER(_ct.c_longlong)


def _load():
    global _lib
    if _lib is None:
        # BAND_ORACLE_LIB lets the mutation test load a deliberately broken copy
        path = _os.environ.get("BAND_ORACLE_LIB") or _build.build()
        lib = _ct.CDLL(path)
        i64, c_int, dbl = _ct.c_int64, _ct.c_int, _ct.c_double
        lib.orc_ntdm.argtypes = [i64, _D, _D, _D, _D, _D, _LL]
        lib.orc_npdm.argtypes = [i64, _D, _D, _D, _D, _D, _D, _D, _D, _LL]
        lib.orc_mnpdm.argtypes = [i64, _D, _D, _D, _D, _D, _D, _D, _LL]
        lib.orc_sip2d.argtypes = [i64, i64, _D, _D, _D, _D, _D, _D, _D, dbl, c_int,
                                  _ct.POINTER(c_int), _D]
        lib.orc_ilu0_2d.argtypes = [i64, i64, _D, _D, _D, _D, _D, _D, _D, _D]
        lib.orc_gepp_band.argtypes = [i64, c_int, _D, _D, _D, _D, _D, _D, _D, _D]
        lib.orc_symbolic.argtypes = [i64, c_int, _D, _D, _D, _D, _D, _D, _D, _D, _LL,
                                     _ct.POINTER(c_int)]
        lib.orc_ilu0.argtypes = [i64, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        lib.orc_lu_minus_a.argtypes = [i64] + [_D] * 15
        lib.orc_lu_minus_a.restype = None
        lib.orc_hb.argtypes = [i64, c_int, c_int, _D, _D, _D, _D, c_int, dbl,
                               _ct.POINTER(c_int)]
        lib.orc_sip.argtypes = [i64, _D, _D, _D, _D, _D, _D, _D, dbl, c_int, c_int, c_int,
                                dbl, _ct.POINTER(c_int), _D, _ct.POINTER(c_int), _LL]
        lib.orc_refine.argtypes = [i64, _F, _F, _F, _F, _F, _D, _D, dbl, c_int,
                                   _ct.POINTER(c_int)]
        lib.orc_adjoint.argtypes = [i64, c_int, _D, _D, _D, _D, _D, _D, _D,
                                    _D, _D, _D, _D, _D, _D]
        lib.orc_cond1.argtypes = [i64, c_int, _D, _D, _D, _D, _D]
        lib.orc_cond1.restype = dbl
        lib.orc_batch.argtypes = [c_int, c_int, i64, i64, i64, i64, _I64, _I8,
                                  _D, _D, _D, _D, _D, _D, _D, _I32, dbl, c_int, c_int, c_int,
                                  dbl, _I32, _D, c_int]
        for name in ("orc_ntdm", "orc_npdm", "orc_mnpdm", "orc_sip2d", "orc_ilu0_2d", "orc_gepp_band", "orc_symbolic", "orc_ilu0",
                     "orc_hb", "orc_sip", "orc_refine", "orc_adjoint", "orc_batch"):
            getattr(lib, name).restype = c_int
        _lib = lib
    return _lib


def _d(arr):
    """float64 C-contiguous view (copy if needed) and its pointer."""
    a = _np.ascontiguousarray(arr, dtype=_np.float64)
    return a, a.ctypes.data_as(_D)


def _f(arr):
    a = _np.ascontiguousarray(arr, dtype=_np.float32)
    return a, a.ctypes.data_as(_F)


def _zeros_like_n(n):
    return _np.zeros(n, dtype=_np.float64)


def ntdm(b, c, d, f, count_ops=False):
    """R1 NTDM.  Returns (x, status[, ops])."""
    lib = _load()
    n = len(c)
    (b, pb), (c, pc), (d, pd), (f, pf) = _d(b), _d(c), _d(d), _d(f)
    x = _zeros_like_n(n)
    ops = _ct.c_longlong(0)
    st = lib.orc_ntdm(n, pb, pc, pd, pf, x.ctypes.data_as(_D), _ct.byref(ops) if count_ops else None)
    return (x, STATUS[st], ops.value) if count_ops else (x, STATUS[st])


def npdm(a, b, c, d, e, f, count_ops=False, factors=False):
    """R2 NPDM.  Returns (x, status[, ops][, (gamma, mu, alpha, beta)])."""
    lib = _load()
    n = len(c)
    (a, pa), (b, pb), (c, pc), (d, pd), (e, pe), (f, pf) = map(_d, (a, b, c, d, e, f))
    x = _zeros_like_n(n)
    fac = _np.zeros(4 * n) if factors else None
    ops = _ct.c_longlong(0)
    st = lib.orc_npdm(n, pa, pb, pc, pd, pe, pf, x.ctypes.data_as(_D),
                      fac.ctypes.data_as(_D) if factors else None,
                      _ct.byref(ops) if count_ops else None)
    out = [x, STATUS[st]]
    if count_ops:
        out.append(ops.value)
    if factors:
        out.append(tuple(fac.reshape(4, n)))
    return tuple(out)


def _diags(k, a, b, c, d, e, n):
    z = _np.zeros(n)
    if a is None:
        a = z
    if e is None:
        e = z
    return a, b, c, d, e


def mnpdm(a, b, c, d, e, f, count_ops=False):
    """R2m MNPDM: the PD -> TD elimination of the nonzero outer entries, then R1.
    Returns (x, status[, ops])."""
    lib = _load()
    n = len(c)
    (a, pa), (b, pb), (c, pc), (d, pd), (e, pe), (f, pf) = map(_d, (a, b, c, d, e, f))
    x = _zeros_like_n(n)
    ops = _ct.c_longlong(0)
    st = lib.orc_mnpdm(n, pa, pb, pc, pd, pe, pf, x.ctypes.data_as(_D),
                       _ct.byref(ops) if count_ops else None)
    return (x, STATUS[st], ops.value) if count_ops else (x, STATUS[st])


def sip2d(nx, ny, s, w, c, e, t, f, tol=1e-10, max_it=500):
    """R6b Stone's method on a 2-D five-point matrix (unknown y nx + x; s, w, c, e, t at
    columns k - nx, k - 1, k, k + 1, k + nx).  Returns dict(x, iters, resid, status)."""
    lib = _load()
    (s, ps), (w, pw), (c, pc), (e, pe), (t, pt), (f, pf) = map(_d, (s, w, c, e, t, f))
    x = _zeros_like_n(nx * ny)
    it, rs = _ct.c_int(0), _ct.c_double(0)
    st = lib.orc_sip2d(nx, ny, ps, pw, pc, pe, pt, pf, x.ctypes.data_as(_D), tol, max_it,
                       _ct.byref(it), _ct.byref(rs))
    return dict(x=x, iters=it.value, resid=rs.value, status=STATUS[st])


def ilu0_2d(nx, ny, s, w, c, e, t):
    """R6b's ILU(0) factors (ls, lw, uc) of a 2-D five-point matrix, and the status."""
    lib = _load()
    (s, ps), (w, pw), (c, pc), (e, pe), (t, pt) = map(_d, (s, w, c, e, t))
    N = nx * ny
    ls, lw, uc = _zeros_like_n(N), _zeros_like_n(N), _zeros_like_n(N)
    st = lib.orc_ilu0_2d(nx, ny, ps, pw, pc, pe, pt, ls.ctypes.data_as(_D), lw.ctypes.data_as(_D),
                         uc.ctypes.data_as(_D))
    return (ls, lw, uc), STATUS[st]


def gepp_band(k, a, b, c, d, e, f):
    """R0 banded GEPP (the truth).  Returns (x, status, det)."""
    lib = _load()
    n = len(c)
    a, b, c, d, e = _diags(k, a, b, c, d, e, n)
    (a, pa), (b, pb), (c, pc), (d, pd), (e, pe), (f, pf) = map(_d, (a, b, c, d, e, f))
    x = _zeros_like_n(n)
    det = _ct.c_double(0)
    st = lib.orc_gepp_band(n, k, pa, pb, pc, pd, pe, pf, x.ctypes.data_as(_D), _ct.byref(det))
    return x, STATUS[st], det.value


def symbolic(k, a, b, c, d, e, f):
    """R3 SPDM (k=2) / STDM (k=1).  Returns (x, status, det_mant, det_exp2, nflag)."""
    lib = _load()
    n = len(c)
    a, b, c, d, e = _diags(k, a, b, c, d, e, n)
    (a, pa), (b, pb), (c, pc), (d, pd), (e, pe), (f, pf) = map(_d, (a, b, c, d, e, f))
    x = _zeros_like_n(n)
    dm, de, nf = _ct.c_double(0), _ct.c_longlong(0), _ct.c_int(0)
    st = lib.orc_symbolic(n, k, pa, pb, pc, pd, pe, pf, x.ctypes.data_as(_D), _ct.byref(dm),
                          _ct.byref(de), _ct.byref(nf))
    return x, STATUS[st], dm.value, de.value, nf.value


def ilu0(a, b, c, d, e):
    """R4 ILU(0).  Returns ((l2, l1, u0, u1, u2), status)."""
    lib = _load()
    n = len(c)
    (a, pa), (b, pb), (c, pc), (d, pd), (e, pe) = map(_d, (a, b, c, d, e))
    out = [_zeros_like_n(n) for _ in range(5)]
    st = lib.orc_ilu0(n, pa, pb, pc, pd, pe, *[o.ctypes.data_as(_D) for o in out])
    return tuple(out), STATUS[st]


def lu_minus_a(lu, a, b, c, d, e):
    """K = LU - A on five diagonals (Algorithm 1)."""
    lib = _load()
    n = len(c)
    lu = [_d(v) for v in lu]
    A = [_d(v) for v in (a, b, c, d, e)]
    out = [_zeros_like_n(n) for _ in range(5)]
    lib.orc_lu_minus_a(n, *[p for _, p in lu], *[p for _, p in A],
                       *[o.ctypes.data_as(_D) for o in out])
    return tuple(out)


def hb(w, lower, m0, m1, m2, max_it=30, tol=1e-12):
    """R5 band Hotelling-Bodewig.  Returns (X[w, n], iters, status)."""
    lib = _load()
    n = len(m1)
    m0 = _np.ones(n) if m0 is None else m0
    (m0, p0), (m1, p1), (m2, p2) = _d(m0), _d(m1), _d(m2)
    X = _np.zeros((w, n))
    it = _ct.c_int(0)
    st = lib.orc_hb(n, w, 1 if lower else 0, p0, p1, p2, X.ctypes.data_as(_D), max_it, tol,
                    _ct.byref(it))
    return X, it.value, STATUS[st]


def sip(a, b, c, d, e, f, tol=1e-10, max_it=200, hb_width=5, hb_max_it=30, hb_tol=1e-12,
        count_ops=False):
    """R6 SIP.  Returns dict(x, iters, resid, hb_iters, status[, ops])."""
    lib = _load()
    n = len(c)
    (a, pa), (b, pb), (c, pc), (d, pd), (e, pe), (f, pf) = map(_d, (a, b, c, d, e, f))
    x = _zeros_like_n(n)
    it, rs = _ct.c_int(0), _ct.c_double(0)
    hbi = (_ct.c_int * 2)(0, 0)
    ops = _ct.c_longlong(0)
    st = lib.orc_sip(n, pa, pb, pc, pd, pe, pf, x.ctypes.data_as(_D), tol, max_it, hb_width,
                     hb_max_it, hb_tol, _ct.byref(it), _ct.byref(rs), hbi,
                     _ct.byref(ops) if count_ops else None)
    out = dict(x=x, iters=it.value, resid=rs.value, hb_iters=(hbi[0], hbi[1]), status=STATUS[st])
    if count_ops:
        out["ops"] = ops.value
    return out


def refine(a32, b32, c32, d32, e32, f, rel_stop=1e-11, max_steps=10):
    """R7 FP32 solve + FP64 refinement.  Returns (x, steps, status)."""
    lib = _load()
    n = len(c32)
    A = [_f(v) for v in (a32, b32, c32, d32, e32)]
    f, pf = _d(f)
    x = _zeros_like_n(n)
    steps = _ct.c_int(0)
    st = lib.orc_refine(n, *[p for _, p in A], pf, x.ctypes.data_as(_D), rel_stop, max_steps,
                        _ct.byref(steps))
    return x, steps.value, STATUS[st]


def adjoint(k, a, b, c, d, e, x, w):
    """R8 adjoint.  Returns ((ga, gb, gc, gd, ge), gf, status)."""
    lib = _load()
    n = len(c)
    a, b, c, d, e = _diags(k, a, b, c, d, e, n)
    A = [_d(v) for v in (a, b, c, d, e)]
    (x, px), (w, pw) = _d(x), _d(w)
    g = [_zeros_like_n(n) for _ in range(6)]
    st = lib.orc_adjoint(n, k, *[p for _, p in A], px, pw, *[v.ctypes.data_as(_D) for v in g])
    return tuple(g[:5]), g[5], STATUS[st]


def cond1(k, a, b, c, d, e):
    """Hager/Higham estimate of kappa_1(A) (a lower bound, usually exact)."""
    lib = _load()
    n = len(c)
    a, b, c, d, e = _diags(k, a, b, c, d, e, n)
    A = [_d(v) for v in (a, b, c, d, e)]
    return lib.orc_cond1(n, k, *[p for _, p in A])


def cond1_batch(k, diags, nsys, n, sys_stride, elem_stride):
    """cond1 of every system of a uniform strided batch (numpy array)."""
    out = _np.empty(nsys)
    idx = _np.arange(n) * elem_stride
    for s in range(nsys):
        sel = s * sys_stride + idx
        out[s] = cond1(k, *[None if v is None else _np.asarray(v)[sel] for v in diags])
    return out


METHOD = {"direct": 0, "symbolic": 1, "gepp": 2, "sip": 3}


def batch(method, k, diags, f, nsys, n, sys_stride, elem_stride, offsets=None, hbw=None,
          nthreads=None, tol=1e-10, max_it=200, hb_width=5, hb_max_it=30, hb_tol=1e-12):
    """Solve a batch of independent systems stored with the given strides.

    diags = (a, b, c, d, e) flat float64 arrays (a, e may be None for TD);
    element i of system s sits at s*sys_stride + i*elem_stride, or at
    offsets[s] + i*elem_stride for ragged batches (per-system half bandwidth
    hbw[s]).  Returns (x, status[nsys] as ints, iters, resid).
    """
    lib = _load()
    if nthreads is None:
        nthreads = _os.cpu_count() or 1
    a, b, c, d, e = diags
    keep = []

    def p(v):
        if v is None:
            return None
        arr, ptr = _d(_np.asarray(v).reshape(-1))
        keep.append(arr)
        return ptr

    f_arr = _np.ascontiguousarray(_np.asarray(f, dtype=_np.float64).reshape(-1))
    x = _np.zeros_like(f_arr)
    # the C driver trusts the strides: check that every element it touches exists
    if offsets is None:
        last = (nsys - 1) * sys_stride + (n - 1) * elem_stride if nsys > 0 and n > 0 else -1
    else:
        last = int(_np.asarray(offsets)[-1]) - 1 if nsys > 0 else -1
    for v in (a, b, c, d, e, f_arr):
        if v is not None and last >= _np.asarray(v).size:
            raise ValueError("batch layout reaches element %d of an array of %d"
                             % (last, _np.asarray(v).size))
    status = _np.zeros(nsys, dtype=_np.int32)
    iters = _np.zeros(nsys, dtype=_np.int32)
    resid = _np.zeros(nsys, dtype=_np.float64)
    offs = None
    if offsets is not None:
        offs = _np.ascontiguousarray(offsets, dtype=_np.int64)
        keep.append(offs)
    hb_arr = None
    if hbw is not None:
        hb_arr = _np.ascontiguousarray(hbw, dtype=_np.int8)
        keep.append(hb_arr)
    lib.orc_batch(METHOD[method], k, nsys, n, sys_stride, elem_stride,
                  offs.ctypes.data_as(_I64) if offs is not None else None,
                  hb_arr.ctypes.data_as(_I8) if hb_arr is not None else None,
                  p(a), p(b), p(c), p(d), p(e), f_arr.ctypes.data_as(_D), x.ctypes.data_as(_D),
                  status.ctypes.data_as(_I32), tol, max_it, hb_width, hb_max_it, hb_tol,
                  iters.ctypes.data_as(_I32), resid.ctypes.data_as(_D), nthreads)
    return x.reshape(_np.shape(f)), status, iters, resid


def _second_difference(v, axis, k, h):
    """D v along `axis` of a square grid with u = 0 on the boundary: the 3-point stencil
    (1, -2, 1) / h^2 (k = 1) or the fourth-order 5-point (-1, 16, -30, 16, -1) / (12 h^2)
    (k = 2), whose point beyond the boundary is the odd reflection of the first interior
    point (u(-h) = -u(h), u(1 + h) = -u(1 - h))."""
    pad = [(0, 0), (0, 0)]
    pad[axis] = (2, 2)
    vp = _np.pad(v, pad)
    n = v.shape[axis]

    def sh(o):
        sl = [slice(None), slice(None)]
        sl[axis] = slice(2 + o, 2 + o + n)
        return vp[tuple(sl)]
    if k == 1:
        return (sh(-1) - 2.0 * sh(0) + sh(1)) / (h * h)
    # the reflected points beyond the boundary
    lo = [slice(None), slice(None)]
    lo[axis] = 0
    hi = [slice(None), slice(None)]
    hi[axis] = n + 3
    first = [slice(None), slice(None)]
    first[axis] = 2
    last = [slice(None), slice(None)]
    last[axis] = n + 1
    vp[tuple(lo)] = -vp[tuple(first)]
    vp[tuple(hi)] = -vp[tuple(last)]
    return (-sh(-2) + 16.0 * sh(-1) - 30.0 * sh(0) + 16.0 * sh(1) - sh(2)) / (12.0 * h * h)


def adi_step(u, tau, lam, source=None, k=2, nthreads=None):
    """One Peaceman-Rachford ADI step of u_t = u_xx + u_yy + lam u (1 - u) + s on the
    n x n interior grid of the unit square (u = 0 on the boundary, h = 1 / (n + 1),
    u[y, x]; second differences as in _second_difference), the nonlinear term and s on
    the right-hand side (theta = tau / 2):
      (I - theta D_x) u* = u + theta (D_y u + g(u) + s),
      (I - theta D_y) u' = u* + theta (D_x u* + g(u*) + s),
    every line system solved by R1 (k = 1) / R2 (k = 2).  Returns (u', statuses)."""
    u = _np.asarray(u, dtype=_np.float64)
    n = u.shape[0]
    h = 1.0 / (n + 1)
    theta = 0.5 * tau
    r = theta / (h * h)
    s = _np.zeros_like(u) if source is None else _np.asarray(source, dtype=_np.float64)
    g = lambda v: lam * v * (1.0 - v)
    if k == 1:
        vals = (0.0, -r, 1.0 + 2.0 * r, -r, 0.0)
    else:
        vals = (r / 12.0, -4.0 * r / 3.0, 1.0 + 2.5 * r, -4.0 * r / 3.0, r / 12.0)
    diags = [_np.full(n * n, v) for v in vals]
    # the 5-point stencil's reflected point makes the first and last rows' diagonal
    # 1 + 29 r / 12: per sweep, by the position along the system
    cx = _np.full((n, n), vals[2])
    cy = _np.full((n, n), vals[2])
    if k == 2:
        cx[:, 0] = cx[:, -1] = 1.0 + 29.0 * r / 12.0      # rows: position = x
        cy[0, :] = cy[-1, :] = 1.0 + 29.0 * r / 12.0      # columns: position = y
    F = u + theta * (_second_difference(u, 0, k, h) + g(u) + s)
    # rows (systems y, elements x): system stride n, element stride 1
    dx = diags[:2] + [cx.reshape(-1)] + diags[3:]
    ustar, st1, _, _ = batch("direct", k, dx, F.reshape(-1), n, n, n, 1, nthreads=nthreads)
    ustar = ustar.reshape(n, n)
    F2 = ustar + theta * (_second_difference(ustar, 1, k, h) + g(ustar) + s)
    # columns (systems x, elements y): system stride 1, element stride n
    dy = diags[:2] + [cy.reshape(-1)] + diags[3:]
    unew, st2, _, _ = batch("direct", k, dy, F2.reshape(-1), n, n, 1, n, nthreads=nthreads)
    return unew.reshape(n, n), _np.concatenate([st1, st2])
