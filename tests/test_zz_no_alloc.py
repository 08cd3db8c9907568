"""band_solve_static: the NTDM / NPDM solve for callers that cannot allocate device
memory -- code that must not block on cudaMalloc's device-wide synchronisation, hosts
whose own pool owns all device memory, C callers without an allocator.  It uses the
library's fixed per-GPU scratch array (BAND_STATIC_SCRATCH_BYTES) instead of a
workspace.

Checked through the C ABI against band_solve on two calls in a row with different
inputs, so the second call cannot lean on what the first left in the shared array.
This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09666_gb300 import build
    from paper_1804_09666_gb300 import _lib as L
    build.build()
    lib = L.load()
    lib.band_solve_static.argtypes = [ct.POINTER(L.BandDesc), ct.c_int32, L.DIAG5, ct.c_void_p,
                                      ct.c_void_p, ct.c_void_p, ct.c_void_p]
    lib.band_solve_static.restype = ct.c_int
    return lib


STATIC_SCRATCH_BYTES = 32 << 20     # BAND_STATIC_SCRATCH_BYTES in include/band.h


def _batch(k, nsys, n, salt):
    B = synth.cfg0(nsys=nsys, n=n, k=k, seed_salt=salt)
    dev = torch.device("cuda:0")
    return {q: torch.from_numpy(B[q]).to(dev) for q in "abcdef"}


def _call(lib, fn, k, nsys, n, T, dtype, schedule=0, chunks=0):
    from paper_1804_09666_gb300 import _lib as L
    T = {q: v.to(dtype) for q, v in T.items()}
    desc = L.BandDesc(half_bw=k, dtype=L.F64 if dtype == torch.float64 else L.F32, nsys=nsys, n=n,
                      sys_stride=1, elem_stride=nsys, offsets=None, hbw=None, total_rows=0,
                      schedule=schedule, chunks=chunks)
    x = torch.empty_like(T["f"])
    st = torch.full((nsys,), -1, dtype=torch.int32, device=x.device)
    diag = L.DIAG5(*[T[q].data_ptr() if (k == 2 or q in "bcd") else None for q in "abcde"])
    method = L.NPDM if k == 2 else L.NTDM
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if fn == "static":
        code = lib.band_solve_static(ct.byref(desc), method, diag, T["f"].data_ptr(), x.data_ptr(),
                                     st.data_ptr(), stream)
    else:
        need = lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE, method, 0)
        ws = torch.empty(need, dtype=torch.uint8, device=x.device)
        code = lib.band_solve(ct.byref(desc), method, None, diag, T["f"].data_ptr(), x.data_ptr(),
                              st.data_ptr(), ws.data_ptr(), need, stream)
    torch.cuda.synchronize()
    assert code == 0
    return x, st


@pytest.mark.parametrize("k", [2, 1])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("schedule,chunks", [(0, 0), (1, 0), (2, 0), (3, 8), (3, 64)])
def test_static_scratch_matches_band_solve_twice(lib, k, dtype, schedule, chunks):
    """The same kernels as band_solve on every schedule: bitwise equal results."""
    for salt, (nsys, n) in enumerate(((1000, 300), (2048, 129))):
        T = _batch(k, nsys, n, salt + 40)
        xs, sts = _call(lib, "static", k, nsys, n, T, dtype, schedule, chunks)
        xw, stw = _call(lib, "ws", k, nsys, n, T, dtype, schedule, chunks)
        assert (sts == 0).all() and (stw == 0).all()
        assert torch.equal(xs, xw)


def test_static_scratch_rejects_oversized_batches(lib):
    from paper_1804_09666_gb300 import _lib as L
    cap = STATIC_SCRATCH_BYTES
    nsys = 4096
    n = cap // (8 * nsys)          # alpha alone fills the array: alpha + beta do not fit
    desc = L.BandDesc(half_bw=2, dtype=L.F64, nsys=nsys, n=n, sys_stride=1, elem_stride=nsys,
                      offsets=None, hbw=None, total_rows=0)
    diag = L.DIAG5(8, 8, 8, 8, 8)
    code = lib.band_solve_static(ct.byref(desc), L.NPDM, diag, 8, 8, None, None)
    assert code == L.ERR_WORKSPACE
    code = lib.band_solve_static(ct.byref(desc), L.SPDM, diag, 8, 8, None, None)
    assert code == L.ERR_ARG


def test_static_scratch_ragged_packing(lib):
    """A whole ragged packing (offsets, per-system bandwidths): the workspace rule is
    band_workspace_size's for the same descriptor; bitwise equal to band_solve, twice."""
    from paper_1804_09666_gb300 import _lib as L
    dev = torch.device("cuda:0")
    for salt in (0, 1):
        B = synth.cfg2(nsys=300, nmin=16, nmax=512, seed_salt=30 + salt)
        T = {q: torch.from_numpy(B[q]).to(dev) for q in "abcdef"}
        offs = torch.from_numpy(B["offsets"]).to(dev)
        hbw = torch.from_numpy(B["hbw"]).to(dev)
        total = int(B["offsets"][-1])
        desc = L.BandDesc(half_bw=2, dtype=L.F64, nsys=300, n=int(B["sizes"].max()),
                          sys_stride=0, elem_stride=1, offsets=offs.data_ptr(),
                          hbw=hbw.data_ptr(), total_rows=total)
        need = lib.band_workspace_size(ct.byref(desc), L.OP_SOLVE, L.AUTO_NUMERIC, 0)
        assert 0 < need <= STATIC_SCRATCH_BYTES
        diag = L.DIAG5(*[T[q].data_ptr() for q in "abcde"])
        stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
        xs = torch.empty_like(T["f"])
        xw = torch.empty_like(T["f"])
        ss = torch.full((300,), -1, dtype=torch.int32, device=dev)
        sw = torch.full((300,), -1, dtype=torch.int32, device=dev)
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        assert lib.band_solve_static(ct.byref(desc), L.AUTO_NUMERIC, diag, T["f"].data_ptr(),
                                     xs.data_ptr(), ss.data_ptr(), stream) == 0
        assert lib.band_solve(ct.byref(desc), L.AUTO_NUMERIC, None, diag, T["f"].data_ptr(),
                              xw.data_ptr(), sw.data_ptr(), ws.data_ptr(), need, stream) == 0
        torch.cuda.synchronize()
        assert (ss == 0).all() and (sw == 0).all()
        assert torch.equal(xs, xw)
        err = (xs.cpu().numpy() - B["x_true"])
        assert np.abs(err).max() <= 1e-12 * np.abs(B["x_true"]).max()
