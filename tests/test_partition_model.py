"""The partitioned schedule's algorithm on the CPU (tests/partition_model.py, a numpy
model of what the kernels compute), against the oracle.

What the GPU tests cannot show alone: that the SPIKE partition with the two-ended
interface (mirrored slots included) is LU without pivoting reordered, for every chunk
count from 4 to 256 and ragged chunk lengths; and, on the indefinite ADI rows, that
the pivot guard is what holds the partition to NPDM's accuracy (pivot growth in the
restarted chunks), for four chunks as for eight and sixteen."""
import numpy as np
import pytest

import oracle
import partition_model as model
import synth


def _columns(B):
    n, ns, ss, es = B["n"], B["nsys"], B["sys_stride"], B["elem_stride"]
    idx = np.arange(ns)[None, :] * ss + np.arange(n)[:, None] * es
    return idx, {q: B[q][idx] for q in "abcdef"}


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("n,P", [(32, 4), (33, 4), (64, 8), (257, 8), (300, 32), (1000, 16),
                                 (520, 64), (1031, 128), (2048, 256)])
def test_model_is_lu_reordered(k, n, P):
    B = synth.cfg0(nsys=9, n=n, k=k, seed_salt=90 + n)
    idx, A = _columns(B)
    x, failed = model.solve(A, k, P)
    assert not failed.any()
    xo, so, _, _ = oracle.batch("direct", k, [B[q] for q in "abcde"], B["f"], B["nsys"], n,
                                B["sys_stride"], B["elem_stride"])
    xo = xo[idx]
    assert (so == 0).all()
    assert (np.abs(x - xo).max(0) / np.abs(xo).max(0)).max() <= 1e-13


@pytest.mark.parametrize("sweep", ["x", "y"])
def test_pivot_guard_on_indefinite_adi_rows(sweep):
    B = synth.cfg1(r=2.0, k=2, sweep=sweep, grid=2048, nsys=40)
    idx, A = _columns(B)
    args = (B["nsys"], B["n"], B["sys_stride"], B["elem_stride"])
    xt = oracle.batch("gepp", 2, [B[q] for q in "abcde"], B["f"], *args)[0][idx]
    xo = oracle.batch("direct", 2, [B[q] for q in "abcde"], B["f"], *args)[0][idx]
    den = np.abs(xt).max(0)
    bound = np.maximum(1e-10, 10 * np.abs(xo - xt).max(0) / den)
    unguarded_worst = 0.0
    for P in (4, 8, 16, 32):
        x, failed = model.solve(A, 2, P, guard=True)
        err = np.abs(x - xt).max(0) / den
        assert (err[~failed] <= bound[~failed]).all(), (P, err[~failed].max())
        assert failed.any() == (P < 32), P          # chunks of 64 rows never trip it here
        x, failed = model.solve(A, 2, P, guard=False)
        assert not failed.any()
        unguarded_worst = max(unguarded_worst, (np.abs(x - xt).max(0) / den).max())
    assert unguarded_worst > 1e-10                   # without the guard: pivot growth
