"""The Python binding rejects arguments the kernels cannot take before any CUDA call
(no GPU needed): host tensors (a kernel would be handed host pointers), mismatched
shapes, strides or dtypes, and malformed ragged packings."""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _host(n=16, nsys=4, dtype=torch.float64):
    return [torch.ones(n, nsys, dtype=dtype) for _ in range(6)]


def test_host_tensors_are_rejected(band):
    a, b, c, d, e, f = _host()
    calls = [
        lambda: band.solve(a, b, c, d, e, f),
        lambda: band.solve(None, b, c, d, None, f, method="ntdm"),
        lambda: band.factor(a, b, c, d, e),
        lambda: band.sip(a, b, c, d, e, f),
        lambda: band.adjoint(a, b, c, d, e, f, f),
        lambda: band.refine_solve(*_host(dtype=torch.float32)[:5], f),
        lambda: band.BatchPlan([dict(a=a, b=b, c=c, d=d, e=e, f=f)]),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="CUDA"):
            call()


def test_host_ragged_packings_are_rejected(band):
    offs = np.array([0, 5, 12], dtype=np.int64)
    a, b, c, d, e, f = (torch.ones(12, dtype=torch.float64) for _ in range(6))
    with pytest.raises(ValueError, match="CUDA"):
        band.solve_ragged(a, b, c, d, e, f, torch.from_numpy(offs), None, n_max=7,
                          total_rows=12, method="npdm")
    with pytest.raises(ValueError, match="CUDA"):
        band.RaggedPlan(a, b, c, d, e, f, offs, half_bw=2)


def test_mismatched_arrays_are_rejected(band):
    a, b, c, d, e, f = _host()
    with pytest.raises(ValueError, match="shape, strides and dtype"):
        band.solve(a, b, c, d, e, f[:8])
    with pytest.raises(ValueError, match="shape, strides and dtype"):
        band.solve(a, b, c, d, e, f.float())
    with pytest.raises(ValueError, match="shape, strides and dtype"):
        band.solve(a, b, c, d, e, f.T.contiguous().T)     # same shape, other strides
    with pytest.raises(ValueError, match="shape, strides and dtype"):
        band.adjoint(a, b, c, d, e, f, f[:, :2])
    with pytest.raises(ValueError, match="shape, strides and dtype"):
        band.refine_solve(*_host(dtype=torch.float32)[:4], torch.ones(16, 4, dtype=torch.float64), f)
