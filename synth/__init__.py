"""Seeded synthetic inputs for the batched band solvers.

This module only draws numbers and lays them out; it holds none of the solvers'
arithmetic.  The one product it forms, ``f = A x_true`` (a manufactured right-hand
side), is how an input is built, and both the CUDA path and the CPU oracle receive
its result as input.

Shapes and distributions follow the workloads of Veneva & Ayriyan (arXiv:1804.09666):
independent systems "one per grid line" of an ADI sweep of a parabolic PDE (Sec. 1),
solved for sizes up to N = 10^8 (Tables 3, 5).

Canonical shape of every per-row array is (n, nsys): row i of system s at [i, s].
Layouts (element i of system s at flat index):
  interleaved  i * nsys + s        -> array.reshape(-1) of the canonical array
  contiguous   s * n + i           -> canonical.T.copy().reshape(-1)
  ragged       offsets[s] + i      -> packed contiguous systems of different n
Diagonals: a = A[i][i-2], b = A[i][i-1], c = A[i][i], d = A[i][i+1], e = A[i][i+2].
Out-of-matrix slots (a[0], a[1], b[0], d[n-1], e[n-2], e[n-1]) hold whatever the
generator says; the solvers never use them.
"""
import math

import numpy as np

SEED_BASE = 180409666


def rng_for(config_id: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_id + 1000 * salt))


def out_of_matrix_mask(n: int):
    """Boolean masks (n,) of the in-matrix slots of a, b, d, e."""
    i = np.arange(n)
    return dict(a=i >= 2, b=i >= 1, d=i <= n - 2, e=i <= n - 3)


def band_matvec(k, a, b, c, d, e, x):
    """y = A x for canonical (n, nsys) diagonals and x; out-of-matrix slots skipped."""
    n = c.shape[0]
    y = c * x
    if n >= 2:
        y[1:] += b[1:] * x[:-1]
        y[:-1] += d[:-1] * x[1:]
    if k == 2 and n >= 3:
        y[2:] += a[2:] * x[:-2]
        y[:-2] += e[:-2] * x[2:]
    return y


def _mask_outside(k, diags, fill=0.0):
    n = diags["b"].shape[0]
    m = out_of_matrix_mask(n)
    for key in ("b", "d") + (("a", "e") if k == 2 else ()):
        diags[key][~m[key]] = fill
    return diags


def dominant(rng, nsys, n, k=2, dtype=np.float64, ratio=None, flip_frac=0.0):
    """Diagonally dominant band systems, canonical shape.

    Off-diagonals uniform in [-1, 1].  Main diagonal = 1 + sum |off-diagonals| of the
    row (ratio None), or ratio * sum |off| with the sign flipped on a random
    ``flip_frac`` of rows.  ``ratio`` may be a per-system array.
    """
    shape = (n, nsys)
    diags = {}
    for key in ("b", "d") + (("a", "e") if k == 2 else ()):
        diags[key] = rng.uniform(-1.0, 1.0, size=shape).astype(dtype)
    if k == 1:
        diags["a"] = np.zeros(shape, dtype=dtype)
        diags["e"] = np.zeros(shape, dtype=dtype)
    _mask_outside(k, diags)
    off = sum(np.abs(diags[key]).astype(np.float64) for key in ("a", "b", "d", "e"))
    if ratio is None:
        cdiag = 1.0 + off
    else:
        cdiag = np.asarray(ratio, dtype=np.float64) * off
        if flip_frac > 0.0:
            flip = rng.random(shape) < flip_frac
            cdiag = np.where(flip, -cdiag, cdiag)
    diags["c"] = cdiag.astype(dtype)
    return diags


def manufactured(rng, k, diags, nsys, n):
    """x_true uniform in [-1, 1] and f = A x_true in FP64 (canonical shape)."""
    x_true = rng.uniform(-1.0, 1.0, size=(n, nsys))
    d64 = {key: np.asarray(v, dtype=np.float64) for key, v in diags.items()}
    f = band_matvec(k, d64["a"], d64["b"], d64["c"], d64["d"], d64["e"], x_true)
    return x_true, f


def to_layout(arr, layout):
    """Canonical (n, nsys) -> flat array in the given layout."""
    if layout == "interleaved":
        return np.ascontiguousarray(arr).reshape(-1)
    if layout == "contiguous":
        return np.ascontiguousarray(arr.T).reshape(-1)
    raise ValueError(layout)


def strides(layout, nsys, n):
    """(sys_stride, elem_stride) in elements."""
    if layout == "interleaved":
        return 1, nsys
    if layout == "contiguous":
        return n, 1
    raise ValueError(layout)


def batch(diags, f, k, nsys, n, layout="interleaved", **extra):
    """Pack canonical arrays into a batch dict in the requested layout."""
    ss, es = strides(layout, nsys, n)
    out = dict(k=k, nsys=nsys, n=n, layout=layout, sys_stride=ss, elem_stride=es)
    for key in ("a", "b", "c", "d", "e"):
        out[key] = to_layout(diags[key], layout)
    out["f"] = to_layout(f, layout)
    for key, v in extra.items():
        out[key] = to_layout(v, layout) if isinstance(v, np.ndarray) and v.shape == (n, nsys) else v
    return out


# ----------------------------------------------------------------- workloads
def cfg0(nsys=1024, n=128, layout="interleaved", k=2, seed_salt=0):
    """Plain NPDM, FP64: dominant PD systems (1 + sum|off| on the diagonal)."""
    rng = rng_for(0, seed_salt)
    diags = dominant(rng, nsys, n, k=k)
    x_true, f = manufactured(rng, k, diags, nsys, n)
    return batch(diags, f, k, nsys, n, layout, x_true=x_true)


def adi_rows(r, n, g, k=2):
    """Diagonals of one ADI sweep for canonical field g (n, nsys).

    PD (second-order scheme): a = e = -r/12, b = d = 4r/3, c = 1 - 5r/2 + h g.
    TD analogue: b = d = -r, c = 1 + 2r + h g.  h = 1/(n+1).  Out-of-matrix slots
    keep the stencil values (the solvers must ignore them).
    """
    h = 1.0 / (n + 1)
    shape = g.shape
    if k == 2:
        diags = dict(a=np.full(shape, -r / 12.0), b=np.full(shape, 4.0 * r / 3.0),
                     c=1.0 - 2.5 * r + h * g, d=np.full(shape, 4.0 * r / 3.0),
                     e=np.full(shape, -r / 12.0))
    else:
        diags = dict(a=np.zeros(shape), b=np.full(shape, -r), c=1.0 + 2.0 * r + h * g,
                     d=np.full(shape, -r), e=np.zeros(shape))
    return diags


ADI_R = (0.5, 2.0, 10.0)


def cfg1(r=0.5, k=2, sweep="x", grid=2048, nsys=None):
    """ADI-shaped sweep of a grid x grid field: grid systems of n = grid.

    The field g (source term) is uniform in [-1, 1] on the grid, stored row-major
    G[y][x].  The x-sweep solves along x (system = row y: contiguous layout); the
    y-sweep solves along y (system = column x, read at row stride: interleaved
    layout).  The right-hand side is f = A x_true with x_true uniform in [-1, 1].
    ``nsys`` (<= grid) keeps only the first nsys lines (smaller parity cases).
    """
    rng = rng_for(1, salt=int(ADI_R.index(r)) if r in ADI_R else 7)
    G = rng.uniform(-1.0, 1.0, size=(grid, grid))
    Xt = rng.uniform(-1.0, 1.0, size=(grid, grid))
    n = grid
    ns = grid if nsys is None else nsys
    if sweep == "x":
        g = G[:ns, :].T      # canonical (n = x, nsys = y)
        xt = Xt[:ns, :].T
        layout = "contiguous"
    else:
        g = G[:, :ns]        # canonical (n = y, nsys = x)
        xt = Xt[:, :ns]
        layout = "interleaved"
    diags = adi_rows(r, n, g, k)
    f = band_matvec(k, diags["a"], diags["b"], diags["c"], diags["d"], diags["e"], xt)
    return batch(diags, f, k, ns, n, layout, x_true=np.ascontiguousarray(xt), r=r, sweep=sweep)


def cfg2(nsys=65536, nmin=16, nmax=8192, seed_salt=0):
    """Ragged batch: n log-uniform in [nmin, nmax], half TD / half PD, dominant.

    Packed contiguous systems: system s occupies [offsets[s], offsets[s+1]) of every
    array; TD systems leave their a/e slots zero.  hbw[s] is 1 (TD) or 2 (PD).
    """
    rng = rng_for(2, seed_salt)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=nsys))).astype(np.int64)
    hbw = np.array([1] * (nsys // 2) + [2] * (nsys - nsys // 2), dtype=np.int8)
    rng.shuffle(hbw)
    offsets = np.zeros(nsys + 1, dtype=np.int64)
    np.cumsum(ns, out=offsets[1:])
    total = int(offsets[-1])
    a = np.zeros(total)
    b = rng.uniform(-1.0, 1.0, size=total)
    d = rng.uniform(-1.0, 1.0, size=total)
    e = np.zeros(total)
    pd_rows = np.repeat(hbw == 2, ns)
    npd = int(pd_rows.sum())
    a[pd_rows] = rng.uniform(-1.0, 1.0, size=npd)
    e[pd_rows] = rng.uniform(-1.0, 1.0, size=npd)
    # row index within its system
    row = np.arange(total) - np.repeat(offsets[:-1], ns)
    nrow = np.repeat(ns, ns)
    a[row < 2] = 0.0
    b[row < 1] = 0.0
    d[row > nrow - 2] = 0.0
    e[row > nrow - 3] = 0.0
    c = 1.0 + np.abs(a) + np.abs(b) + np.abs(d) + np.abs(e)
    x_true = rng.uniform(-1.0, 1.0, size=total)
    f = c * x_true
    prev1 = np.concatenate(([0.0], x_true[:-1]))
    prev2 = np.concatenate(([0.0, 0.0], x_true[:-2]))
    next1 = np.concatenate((x_true[1:], [0.0]))
    next2 = np.concatenate((x_true[2:], [0.0, 0.0]))
    f += b * prev1 + d * next1 + a * prev2 + e * next2   # zero slots stop spill-over
    return dict(k=0, nsys=nsys, n=0, layout="ragged", sys_stride=0, elem_stride=1,
                offsets=offsets, hbw=hbw, sizes=ns, a=a, b=b, c=c, d=d, e=e, f=f,
                x_true=x_true)


CFG3_RATIOS = (1.01, 1.1, 2.0)


def cfg3(nsys=16384, n=4096, layout="interleaved", seed_salt=0):
    """Precision workload: PD systems stored in FP32 (exactly representable), with
    dominance ratio |c| / sum|off| per system in {1.01, 1.1, 2.0} and the diagonal's
    sign flipped on 5% of rows.  f = A x_true in FP64 with A the FP64 values of the
    FP32 diagonals."""
    rng = rng_for(3, seed_salt)
    ratio = rng.choice(np.array(CFG3_RATIOS), size=nsys)
    diags = dominant(rng, nsys, n, k=2, dtype=np.float32, ratio=ratio[None, :], flip_frac=0.05)
    x_true, f = manufactured(rng, 2, diags, nsys, n)
    out = batch(diags, f, 2, nsys, n, layout, x_true=x_true)
    out["ratio"] = ratio
    return out


def cfg4(nsys=4096, n=1024, layout="interleaved", seed_salt=0):
    """Differentiation workload: cfg0-style systems plus loss weights w in [-1, 1]."""
    rng = rng_for(4, seed_salt)
    diags = dominant(rng, nsys, n, k=2)
    x_true, f = manufactured(rng, 2, diags, nsys, n)
    w = rng.uniform(-1.0, 1.0, size=(n, nsys))
    return batch(diags, f, 2, nsys, n, layout, x_true=x_true, w=w)


def system(batch_dict, s):
    """Extract system s of a strided batch as contiguous 1-D arrays (a..e, f)."""
    B = batch_dict
    if B["layout"] == "ragged":
        lo, hi = int(B["offsets"][s]), int(B["offsets"][s + 1])
        return {key: B[key][lo:hi] for key in ("a", "b", "c", "d", "e", "f")}
    n, ss, es = B["n"], B["sys_stride"], B["elem_stride"]
    idx = s * ss + np.arange(n) * es
    return {key: B[key][idx] for key in ("a", "b", "c", "d", "e", "f")}
