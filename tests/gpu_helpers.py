"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def strided_view(flat, n, nsys, ss, es, dtype=torch.float64):
    """Device tensor (n, nsys) viewing a flat host array laid out with the given strides."""
    t = torch.from_numpy(np.ascontiguousarray(flat)).to(DEV, dtype=dtype)
    return t.as_strided((n, nsys), (es, ss))


def to_dev(B, keys="abcdef", dtype=torch.float64):
    n, ns, ss, es = B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]
    return {k: strided_view(B[k], n, ns, ss, es, dtype) for k in keys}


def flat_of(t):
    """The storage of a strided device tensor as a flat host array."""
    n, ns = t.shape
    es, ss = t.stride()
    size = (n - 1) * es + (ns - 1) * ss + 1
    return t.as_strided((size,), (1,)).cpu().numpy()


def per_system_rel(x, ref, n, nsys, ss, es):
    """max_i |x - ref| / max_i |ref| per system, for flat arrays in a strided layout."""
    idx = (np.arange(nsys)[None, :] * ss + np.arange(n)[:, None] * es)
    xs, rs = x[idx], ref[idx]
    den = np.abs(rs).max(0)
    den[den == 0] = 1.0
    return np.abs(xs - rs).max(0) / den
