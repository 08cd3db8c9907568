"""CPU checks of the C ABI: the library loads, exports what include/band.h declares,
and rejects bad arguments before touching the GPU.  No compute calls."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "band.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09666_gb300 import build
    from paper_1804_09666_gb300 import _lib as L
    build.build()
    return L.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(band_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("band_solve", "band_factor", "band_sip", "band_refine_solve", "band_adjoint",
                 "band_workspace_size", "band_status_str"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_exports_match_binding_list(lib):
    from paper_1804_09666_gb300 import _lib as L
    assert sorted(L.EXPORTS) == sorted(n for n in declared_functions() if n in L.EXPORTS)
    for name in L.EXPORTS:
        assert hasattr(lib, name)


def test_desc_layout():
    from paper_1804_09666_gb300 import _lib as L
    # int32, int32, 4 x int64, 2 pointers, int64, int32, int32, pointer
    assert ct.sizeof(L.BandDesc) == 8 + 4 * 8 + 2 * 8 + 8 + 8 + 8


def test_status_strings(lib):
    from paper_1804_09666_gb300 import _lib as L
    for code, name in L.STATUS_NAMES.items():
        assert lib.band_status_str(code).decode() == "BAND_" + ("OK" if name == "OK" else "ERR_" + name)
    assert b"sm_103a" in lib.band_version()


def _desc(**kw):
    from paper_1804_09666_gb300 import _lib as L
    base = dict(half_bw=2, dtype=L.F64, nsys=64, n=128, sys_stride=1, elem_stride=64, offsets=None,
                hbw=None, total_rows=0)
    base.update(kw)
    return L.BandDesc(**base)


def test_workspace_sizes(lib):
    from paper_1804_09666_gb300 import _lib as L
    d = _desc()
    rows = 64 * 128 * 8
    assert lib.band_workspace_size(ct.byref(d), L.OP_SOLVE, L.NPDM, 0) >= 2 * rows
    # partitioned: alpha, beta, z and the two coupling columns, chunk-major
    dp = _desc(schedule=L.SCHED_PARTITIONED, chunks=8)
    assert lib.band_workspace_size(ct.byref(dp), L.OP_SOLVE, L.NPDM, 0) >= 5 * rows
    dt = _desc(half_bw=1, schedule=L.SCHED_PARTITIONED)
    assert lib.band_workspace_size(ct.byref(dt), L.OP_SOLVE, L.NTDM, 0) >= 4 * rows
    # chunks = 0 leaves the library the choice: its workspace covers every chunk count
    for nsys, n in ((64, 128), (37, 1031), (3, 5000), (1000, 40)):
        auto = lib.band_workspace_size(ct.byref(_desc(nsys=nsys, n=n, elem_stride=nsys,
                                                      schedule=L.SCHED_PARTITIONED)),
                                       L.OP_SOLVE, L.NPDM, 0)
        for P in (4, 8, 16, 32, 64, 128, 256):
            fixed = lib.band_workspace_size(
                ct.byref(_desc(nsys=nsys, n=n, elem_stride=nsys, schedule=L.SCHED_PARTITIONED,
                               chunks=P)), L.OP_SOLVE, L.NPDM, 0)
            assert 0 < fixed <= auto, (nsys, n, P, fixed, auto)
            # ceil(n / P) * P rows for nsys rounded up to 32 / P systems, five arrays
            np_ = nsys if P >= 32 else -(-nsys // (32 // P)) * (32 // P)
            assert fixed >= 5 * (-(-n // P)) * P * np_ * 8
    assert lib.band_workspace_size(ct.byref(d), L.OP_SOLVE, L.SPDM, 0) > \
        lib.band_workspace_size(ct.byref(d), L.OP_SOLVE, L.NPDM, 0)
    assert lib.band_workspace_size(ct.byref(d), L.OP_FACTOR, L.NPDM, 0) >= 4 * rows
    assert lib.band_workspace_size(ct.byref(d), L.OP_SIP, 0, 5) > \
        lib.band_workspace_size(ct.byref(d), L.OP_SIP, 0, 0)
    assert lib.band_workspace_size(ct.byref(d), L.OP_SIP, 0, 9) == 0       # width > 8
    assert lib.band_workspace_size(ct.byref(_desc(n=0)), L.OP_SOLVE, L.NPDM, 0) == 0
    for v in (lib.band_workspace_size(ct.byref(d), op, L.NPDM, 5) for op in range(5)):
        assert v % 256 == 0


def test_bad_arguments_are_rejected_without_gpu(lib):
    from paper_1804_09666_gb300 import _lib as L
    nul = L.DIAG5(None, 1, 2, 3, None)
    full = L.DIAG5(8, 16, 24, 32, 40)
    cases = [
        (_desc(n=0), L.NPDM, full),               # n < 1
        (_desc(half_bw=3), L.NPDM, full),         # bad bandwidth
        (_desc(dtype=7), L.NPDM, full),           # bad dtype
        (_desc(nsys=-1), L.NPDM, full),
        (_desc(elem_stride=0), L.NPDM, full),
        (_desc(sys_stride=1, elem_stride=10), L.NPDM, full),   # overlapping systems
        (_desc(half_bw=2), L.NTDM, full),         # method / bandwidth mismatch
        (_desc(half_bw=1), L.NPDM, full),
        (_desc(half_bw=2), L.NPDM, nul),          # PD without a, e
        (_desc(), 17, full),                      # unknown method
        (_desc(dtype=L.F32), L.SPDM, full),       # symbolic path is FP64 only
        (_desc(schedule=5), L.NPDM, full),        # unknown schedule
        (_desc(schedule=L.SCHED_GRID), L.SPDM, full),          # grid: numeric methods only
        (_desc(schedule=L.SCHED_GRID, chunks=8), L.NPDM, full),
        (_desc(schedule=L.SCHED_GRID, offsets=8, total_rows=100), L.NPDM, full),  # uniform only
        (_desc(schedule=-1), L.NPDM, full),
        (_desc(chunks=8), L.NPDM, full),          # chunks without the partitioned schedule
        (_desc(schedule=L.SCHED_PARTITIONED, chunks=6), L.NPDM, full),   # not 4/8/16/32
        (_desc(schedule=L.SCHED_PARTITIONED, chunks=512), L.NPDM, full),
        (_desc(schedule=L.SCHED_PARTITIONED, chunks=2), L.NPDM, full),
        (_desc(schedule=L.SCHED_PARTITIONED, chunks=48), L.NPDM, full),
    ]
    for d, m, diag in cases:
        code = lib.band_solve(ct.byref(d), m, None, diag, 8, 8, None, 8, 1 << 30, None)
        assert code == L.ERR_ARG, (d.half_bw, d.dtype, d.nsys, d.n, m)
    # workspace too small
    d = _desc()
    assert lib.band_solve(ct.byref(d), L.NPDM, None, full, 8, 8, None, 8, 16, None) == L.ERR_WORKSPACE
    assert lib.band_solve(ct.byref(d), L.NPDM, None, full, 8, 8, None, None, 0, None) == L.ERR_WORKSPACE
    # empty batch is a no-op that succeeds
    d0 = _desc(nsys=0)
    assert lib.band_solve(ct.byref(d0), L.NPDM, None, full, 8, 8, None, 8, 1 << 20, None) == L.OK
    # SIP argument checks
    assert lib.band_sip(ct.byref(d), full, 8, 8, 1e-10, 10, 9, 30, 1e-12, None, None, None, 8,
                        1 << 30, None) == L.ERR_ARG
    assert lib.band_sip(ct.byref(_desc(dtype=L.F32)), full, 8, 8, 1e-10, 10, 5, 30, 1e-12, None,
                        None, None, 8, 1 << 30, None) == L.ERR_ARG
    assert lib.band_sip(ct.byref(d), full, 8, 8, float("nan"), 10, 5, 30, 1e-12, None, None, None,
                        8, 1 << 30, None) == L.ERR_ARG
    # refinement wants an FP32 descriptor
    assert lib.band_refine_solve(ct.byref(d), full, 8, 8, 1e-11, 10, None, None, 8, 1 << 30,
                                 None) == L.ERR_ARG
    # adjoint rejects symbolic methods and missing gradient buffers
    g = L.DIAG5(8, 16, 24, 32, 40)
    assert lib.band_adjoint(ct.byref(d), L.SPDM, None, full, 8, 8, g, 8, None, 8, 1 << 30,
                            None) == L.ERR_ARG
    assert lib.band_adjoint(ct.byref(d), L.NPDM, None, full, 8, 8, L.DIAG5(None, 1, 2, 3, None), 8,
                            None, 8, 1 << 30, None) == L.ERR_ARG
    # the grid schedule is band_solve's alone
    dg = _desc(schedule=L.SCHED_GRID)
    assert lib.band_sip(ct.byref(dg), full, 8, 8, 1e-10, 10, 0, 30, 1e-12, None, None, None, 8,
                        1 << 30, None) == L.ERR_ARG
    assert lib.band_workspace_size(ct.byref(dg), L.OP_SOLVE, L.NPDM, 0) >= 5 * 64 * 128 * 8
    # determinant: FP64 only, every output required, PD needs a and e, workspace checked
    assert lib.band_det(ct.byref(_desc(dtype=L.F32)), full, 8, 8, 8, 8, 1 << 30, None) == L.ERR_ARG
    assert lib.band_det(ct.byref(d), full, 8, 8, None, 8, 1 << 30, None) == L.ERR_ARG
    assert lib.band_det(ct.byref(d), full, None, 8, 8, 8, 1 << 30, None) == L.ERR_ARG
    assert lib.band_det(ct.byref(d), nul, 8, 8, 8, 8, 1 << 30, None) == L.ERR_ARG
    assert lib.band_det(ct.byref(d), full, 8, 8, 8, 8, 16, None) == L.ERR_WORKSPACE
    assert lib.band_det(ct.byref(_desc(nsys=0)), full, 8, 8, 8, 8, 0, None) == L.OK
    # the ADI step: a grid descriptor (strides ignored), n >= 3, tau > 0
    grid = _desc(nsys=64, n=64, sys_stride=1, elem_stride=1)
    assert lib.band_workspace_size(ct.byref(grid), L.OP_ADI, 0, 0) >= 8 * 64 * 64 * 8
    assert lib.band_workspace_size(ct.byref(_desc(nsys=2, n=2)), L.OP_ADI, 0, 0) == 0
    assert lib.band_workspace_size(ct.byref(_desc(nsys=64, n=63)), L.OP_ADI, 0, 0) == 0
    assert lib.band_adi_step(ct.byref(grid), 0.0, 1.0, None, 8, None, 8, 1 << 40, None) == L.ERR_ARG
    assert lib.band_adi_step(ct.byref(grid), 0.1, 1.0, None, None, None, 8, 1 << 40, None) == L.ERR_ARG
    assert lib.band_adi_step(ct.byref(grid), 0.1, 1.0, None, 8, None, 8, 64, None) == L.ERR_WORKSPACE
    # 2-D SIP: nx must divide n, x must not alias f, FP64 uniform only
    d2 = _desc(nsys=64, n=120)
    assert lib.band_sip2d(ct.byref(d2), 7, full, 8, 16, 1e-10, 10, None, None, None, 8, 1 << 30,
                          None) == L.ERR_ARG
    assert lib.band_sip2d(ct.byref(d2), 12, full, 8, 8, 1e-10, 10, None, None, None, 8, 1 << 30,
                          None) == L.ERR_ARG
    assert lib.band_sip2d(ct.byref(_desc(nsys=64, n=120, dtype=L.F32)), 12, full, 8, 16, 1e-10, 10,
                          None, None, None, 8, 1 << 30, None) == L.ERR_ARG
    assert lib.band_sip2d(ct.byref(d2), 12, full, 8, 16, 1e-10, 10, None, None, None, 8, 64,
                          None) == L.ERR_WORKSPACE
    assert lib.band_workspace_size(ct.byref(d2), L.OP_SIP2D, 0, 0) >= 4 * 64 * 120 * 8
    # its workspace is the flagged-system counter and list
    assert lib.band_workspace_size(ct.byref(d), L.OP_DET, 0, 0) >= 8 + 64 * 8


def test_misaligned_pointers_are_rejected_without_gpu(lib):
    """A pointer off its boundary (element size for arrays, 256 bytes for workspaces and
    factor buffers) is refused before anything is launched, so these calls with fake
    addresses never reach the GPU."""
    from paper_1804_09666_gb300 import _lib as L
    ws = 1 << 20                   # a 256-byte aligned stand-in address
    full = L.DIAG5(8, 16, 24, 32, 40)
    odd = L.DIAG5(8, 16, 28, 32, 40)                       # c off the 8-byte boundary
    d, d32 = _desc(), _desc(dtype=L.F32)
    assert lib.band_solve(ct.byref(d), L.NPDM, None, odd, 8, 8, None, ws, 1 << 30, None) == L.ERR_ARG
    assert lib.band_solve(ct.byref(d), L.NPDM, None, full, 12, 8, None, ws, 1 << 30, None) == L.ERR_ARG
    assert lib.band_solve(ct.byref(d), L.NPDM, None, full, 8, 4, None, ws, 1 << 30, None) == L.ERR_ARG
    assert lib.band_solve(ct.byref(d), L.NPDM, None, full, 8, 8, 6, ws, 1 << 30, None) == L.ERR_ARG
    assert lib.band_solve(ct.byref(d), L.NPDM, 4096 + 8, full, 8, 8, None, ws, 1 << 30,
                          None) == L.ERR_WORKSPACE
    for w in (ws + 8, ws + 128):   # workspace off the 256-byte boundary
        assert lib.band_solve(ct.byref(d), L.NPDM, None, full, 8, 8, None, w, 1 << 30,
                              None) == L.ERR_WORKSPACE
        for s in ("auto", "thread", "two_sided", "partitioned", "grid"):
            ds = _desc(schedule={"auto": L.SCHED_AUTO, "thread": L.SCHED_THREAD,
                                 "two_sided": L.SCHED_TWO_SIDED,
                                 "partitioned": L.SCHED_PARTITIONED, "grid": L.SCHED_GRID}[s])
            assert lib.band_solve(ct.byref(ds), L.NPDM, None, full, 8, 8, None, w, 1 << 30,
                                  None) == L.ERR_WORKSPACE, s
        assert lib.band_sip(ct.byref(d), full, 8, 8, 1e-10, 10, 5, 30, 1e-12, None, None, None, w,
                            1 << 30, None) == L.ERR_WORKSPACE
        assert lib.band_det(ct.byref(d), full, 8, 8, 8, w, 1 << 30, None) == L.ERR_WORKSPACE
    # FP32 arrays need 4 bytes: 4 is on the boundary, 2 is not
    assert lib.band_solve(ct.byref(d32), L.NPDM, None, L.DIAG5(4, 12, 20, 28, 36), 4, 4, None,
                          ws + 8, 1 << 30, None) == L.ERR_WORKSPACE   # arrays fine, ws not
    assert lib.band_solve(ct.byref(d32), L.NPDM, None, L.DIAG5(4, 12, 22, 28, 36), 4, 4, None,
                          ws, 1 << 30, None) == L.ERR_ARG
    # the other entry points
    assert lib.band_factor(ct.byref(d), L.NPDM, odd, ws, 1 << 30, None, None) == L.ERR_ARG
    assert lib.band_factor(ct.byref(d), L.NPDM, full, ws + 64, 1 << 30, None, None) == L.ERR_WORKSPACE
    assert lib.band_sip(ct.byref(d), odd, 8, 8, 1e-10, 10, 5, 30, 1e-12, None, None, None, ws,
                        1 << 30, None) == L.ERR_ARG
    assert lib.band_sip(ct.byref(d), full, 8, 8, 1e-10, 10, 5, 30, 1e-12, 2, None, None, ws,
                        1 << 30, None) == L.ERR_ARG               # int32 iters off 4 bytes
    assert lib.band_refine_solve(ct.byref(d32), L.DIAG5(4, 12, 20, 28, 36), 12, 8, 1e-11, 10,
                                 None, None, ws, 1 << 30, None) == L.ERR_ARG
    assert lib.band_adjoint(ct.byref(d), L.NPDM, None, full, 8, 8, odd, 8, None, ws, 1 << 30,
                            None) == L.ERR_ARG
    assert lib.band_adjoint(ct.byref(d), L.NPDM, 4096 + 16, full, 8, 8, full, 8, None, ws,
                            1 << 30, None) == L.ERR_WORKSPACE
    assert lib.band_det(ct.byref(d), full, 12, 8, 8, ws, 1 << 30, None) == L.ERR_ARG
    grid = _desc(nsys=64, n=64, sys_stride=1, elem_stride=1)
    assert lib.band_adi_step(ct.byref(grid), 0.1, 1.0, None, 12, None, ws, 1 << 40, None) == L.ERR_ARG
    assert lib.band_adi_step(ct.byref(grid), 0.1, 1.0, None, 8, None, ws + 8, 1 << 40,
                             None) == L.ERR_WORKSPACE
    d2 = _desc(nsys=64, n=120)
    assert lib.band_sip2d(ct.byref(d2), 12, full, 8, 20, 1e-10, 10, None, None, None, ws, 1 << 30,
                          None) == L.ERR_ARG
    # ragged offsets and id lists are device int64 arrays
    assert lib.band_workspace_size(ct.byref(_desc(offsets=12, total_rows=100)), L.OP_SOLVE,
                                   L.NPDM, 0) == 0


def test_package_refuses_to_run_without_library(tmp_path):
    from paper_1804_09666_gb300 import _lib as L
    with pytest.raises(RuntimeError):
        L.load(str(tmp_path / "missing.so"))
