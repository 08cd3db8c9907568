"""The FP64 reciprocal every pivot goes through (rcp64: an FP32 seed on a rebased
exponent, then one third-order Newton-Raphson step) against IEEE division, element by
element: within 1 ulp of the correctly rounded 1/m over the exponent window where the
rebasing applies, mantissas at 1, 1 + ulp, 2 - ulp and random, both signs; at the
window's edges and outside it (and for 0, Inf, NaN) the division itself, bit for bit."""
import ctypes as ct
import os
import subprocess

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("rcp") / "librcp.so")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
                    "-I" + os.path.join(ROOT, "paper_1804_09666_gb300", "csrc"),
                    os.path.join(HERE, "probes", "rcp_probe.cu"), "-o", out], check=True)
    lib = ct.CDLL(out)
    lib.rcp64_probe.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int64]
    lib.rcp64_probe.restype = ct.c_int
    return lib


def _run(probe, m):
    dev = torch.device("cuda:0")
    x = torch.from_numpy(np.ascontiguousarray(m, dtype=np.float64)).to(dev)
    y = torch.empty_like(x)
    assert probe.rcp64_probe(x.data_ptr(), y.data_ptr(), x.numel()) == 0
    return y.cpu().numpy()


def _with_exponent(mant, biased):
    """Doubles with the given mantissa fields (in [1, 2)) and biased exponents."""
    bits = (np.asarray(biased, dtype=np.uint64) << np.uint64(52)) | \
        (np.asarray(mant, dtype=np.float64).view(np.uint64) & np.uint64((1 << 52) - 1))
    return bits.view(np.float64)


def _ulps(got, want):
    """Distance in units in the last place of want."""
    return np.abs(got - want) / np.spacing(np.abs(want))


def test_rcp64_within_one_ulp_in_the_window(probe):
    rng = np.random.default_rng(64)
    mants = np.concatenate([[1.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 1.5],
                            rng.uniform(1.0, 2.0, 60)])
    exps = np.concatenate([np.arange(903, 911), np.arange(1016, 1032), np.arange(1136, 1144),
                           rng.integers(903, 1144, 40)])
    M = np.array([_with_exponent(mants, e) for e in exps]).reshape(-1)
    M = np.concatenate([M, -M])
    got = _run(probe, M)
    want = 1.0 / M
    u = _ulps(got, want)
    assert u.max() <= 1.0, (M[np.argmax(u)], u.max())
    assert (u == 0).mean() >= 0.9     # almost always the correctly rounded value


def test_rcp64_window_edges_and_specials_are_the_division(probe):
    """Outside the rebasing window (biased exponents 903 .. 1143, |m| in about
    [2^-120, 2^121)), and for zero, infinities, NaN and subnormals: exactly IEEE 1/m."""
    rng = np.random.default_rng(65)
    mants = np.concatenate([[1.0, np.nextafter(2.0, 1.0)], rng.uniform(1.0, 2.0, 20)])
    exps = np.concatenate([np.arange(1, 903), np.arange(1144, 2047)])
    M = np.array([_with_exponent(mants, e) for e in exps[::7]]).reshape(-1)
    M = np.concatenate([M, -M, [0.0, -0.0, np.inf, -np.inf, 5e-324, -1e-310]])
    with np.errstate(divide="ignore", over="ignore"):
        want = 1.0 / M
    got = _run(probe, M)
    same = (got.view(np.uint64) == want.view(np.uint64)) | (np.isnan(got) & np.isnan(want))
    assert same.all(), M[~same][:5]
    nan = _run(probe, np.array([np.nan]))
    assert np.isnan(nan).all()
