"""Host-side batch runtime (no GPU): band_plan_ragged cuts a ragged packing into size
buckets of one half bandwidth and one power-of-two size range."""
import ctypes as ct

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09666_gb300 import build
    from paper_1804_09666_gb300 import _lib as L
    build.build()
    return L.load()


def _plan(lib, sizes, hbw=None, half_bw=2, max_buckets=64):
    from paper_1804_09666_gb300 import _lib as L
    sizes = np.asarray(sizes, dtype=np.int64)
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    hb = None if hbw is None else np.ascontiguousarray(np.asarray(hbw, dtype=np.int8))
    order = np.full(max(len(sizes), 1), -1, dtype=np.int64)
    bk = (L.BandBucket * max(max_buckets, 1))()
    nb = lib.band_plan_ragged(offs.ctypes.data, hb.ctypes.data if hb is not None else None,
                              half_bw, len(sizes), order.ctypes.data, bk, max_buckets)
    return nb, order[:len(sizes)], [(b.first, b.count, b.n_max, b.half_bw) for b in bk[:max(nb, 0)]]


def test_buckets_partition_the_batch(lib):
    rng = np.random.default_rng(0)
    nsys = 5000
    sizes = np.rint(np.exp(rng.uniform(np.log(16), np.log(8192), nsys))).astype(np.int64)
    hbw = rng.integers(1, 3, nsys).astype(np.int8)
    nb, order, buckets = _plan(lib, sizes, hbw)
    assert nb == len(buckets) > 0
    assert sorted(order.tolist()) == list(range(nsys))          # a permutation
    pos = 0
    for first, count, n_max, k in buckets:
        assert first == pos and count > 0
        ids = order[first:first + count]
        n = sizes[ids]
        assert (hbw[ids] == k).all()                              # one bandwidth
        assert n.max() == n_max and n_max < 2 * (1 << int(np.log2(n.min())))   # one octave
        assert (np.diff(n) <= 0).all()                            # longest first
        assert (np.floor(np.log2(n)) == np.floor(np.log2(n_max))).all()
        pos += count
    assert pos == nsys
    # every (bandwidth, octave) pair present in the data is one bucket
    pairs = {(int(k), int(np.log2(n))) for k, n in zip(hbw, sizes)}
    assert len(pairs) == nb


def test_uniform_bandwidth_and_edge_cases(lib):
    nb, order, buckets = _plan(lib, [5, 1, 64, 63, 32], hbw=None, half_bw=1)
    assert [b[3] for b in buckets] == [1, 1, 1, 1]
    # octaves: 64 | 63, 32 | 5 | 1, larger octaves first, longest first within one
    assert [b[2] for b in buckets] == [64, 63, 5, 1]
    assert [b[1] for b in buckets] == [1, 2, 1, 1]
    assert order.tolist() == [2, 3, 4, 0, 1]
    assert _plan(lib, [])[0] == 0
    assert _plan(lib, [3, 0, 4])[0] == -1                 # a system of size 0
    assert _plan(lib, [3, 4], hbw=[1, 3])[0] == -1        # bad bandwidth
    assert _plan(lib, [3, 4], half_bw=5)[0] == -1
    assert _plan(lib, [2, 4, 8, 16], max_buckets=2)[0] == -1   # too many buckets


def test_autotune_rejects_bad_arguments(lib):
    from paper_1804_09666_gb300 import _lib as L
    out = (ct.c_int32 * 2)()
    outc = (ct.c_int32 * 2)()
    assert lib.band_autotune(None, 0, 3, 0, out, outc, None) == L.OK
    assert lib.band_autotune(None, 0, 3, L.TUNE_JOINT, out, None, None) == L.OK
    assert lib.band_autotune(None, 0, 3, 2, out, outc, None) == L.ERR_ARG   # unknown flag
    arr = (L.BandProblem * 1)()
    assert lib.band_autotune(arr, 1, 3, 0, out, outc, None) == L.ERR_ARG     # desc NULL
    assert lib.band_autotune(arr, 65, 3, 0, out, outc, None) == L.ERR_ARG
    assert lib.band_autotune(arr, 1, 0, 0, out, outc, None) == L.ERR_ARG     # reps < 1


def test_batch_warps_default(lib):
    lib.band_autotune_reset()
    assert lib.band_batch_warps(0) == 2
    assert lib.band_batch_warps(63) == 2
    assert lib.band_batch_warps(64) == -1
    assert lib.band_batch_warps(-1) == -1
