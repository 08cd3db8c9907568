"""GPU parity of the ADI time step (band_adi_step: Peaceman-Rachford steps of
u_t = Delta u + lam u (1 - u) + s with TD or PD line systems) against the oracle's
adi_step, element by element after several steps; the steps captured in one CUDA graph
give the same bits as launched one by one; the steady state matches the oracle's and
the manufactured solution's second-order accuracy."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def band():
    import paper_1804_09666_gb300 as band
    from paper_1804_09666_gb300 import build
    build.build()
    band.load()
    return band


def _manufactured(n, lam):
    h = 1.0 / (n + 1)
    xs = h * np.arange(1, n + 1)
    X, Y = np.meshgrid(xs, xs)
    sp = np.sin(np.pi * X) * np.sin(np.pi * Y)
    ue = sp * (1 + X * Y / 2)
    S_xx = -np.pi ** 2 * sp
    S_x = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
    S_y = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
    lap = 2 * S_xx * (1 + X * Y / 2) + 2 * (S_x * Y / 2 + S_y * X / 2)
    return ue, -lap - lam * ue * (1 - ue)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("n,tau", [(129, 0.01), (200, 0.002), (3, 0.1)])
def test_adi_steps_against_oracle(band, k, n, tau):
    rng = np.random.default_rng(n + k)
    u0 = rng.uniform(0, 1, (n, n))
    s = rng.uniform(-1, 1, (n, n))
    lam = 2.0
    stepper = band.AdiStepper(n, tau, lam, torch.tensor(s, device=DEV), half_bw=k)
    u = torch.tensor(u0, device=DEV)
    uo = u0.copy()
    for step in range(5):
        stepper.step(u)
        uo, st = oracle.adi_step(uo, tau, lam, s, k=k)
        torch.cuda.synchronize()
        assert (stepper.status.cpu() == 0).all() and (st == 0).all()
        err = np.abs(u.cpu().numpy() - uo).max() / np.abs(uo).max()
        assert err <= 1e-12, (step, err)


def test_adi_graph_capture_is_bitwise(band):
    n, k = 256, 2
    rng = np.random.default_rng(3)
    u0 = torch.tensor(rng.uniform(0, 1, (n, n)), device=DEV)
    stepper = band.AdiStepper(n, 0.005, 1.0, None, half_bw=k)
    eager = u0.clone()
    stepper.step(eager, steps=10)
    ug = u0.clone()
    stepper.step(ug)                      # warm-up outside capture
    ug.copy_(u0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            stepper.step(ug, steps=10)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ug, eager)


@pytest.mark.parametrize("k", [1, 2])
def test_adi_steady_state(band, k):
    """400 steps to steady state at n = 63: the oracle's result and the manufactured
    solution's second-order error (3-point 2.2e-4, 5-point 3.3e-5 at this n)."""
    n, lam = 63, 1.0
    ue, s = _manufactured(n, lam)
    stepper = band.AdiStepper(n, 0.02, lam, torch.tensor(s, device=DEV), half_bw=k)
    u = torch.zeros((n, n), dtype=torch.float64, device=DEV)
    stepper.step(u, steps=400)
    uo = np.zeros((n, n))
    for _ in range(400):
        uo, _ = oracle.adi_step(uo, 0.02, lam, s, k=k)
    ug = u.cpu().numpy()
    assert np.abs(ug - uo).max() <= 1e-11
    assert np.abs(ug - ue).max() <= (2.5e-4 if k == 1 else 4e-5)


def test_adi_rejects_bad_grids(band):
    from paper_1804_09666_gb300 import BandError
    with pytest.raises(ValueError):
        band.AdiStepper(2, 0.01)          # n >= 3
    stepper = band.AdiStepper(16, 0.01)
    with pytest.raises(ValueError):
        stepper.step(torch.zeros((15, 15), dtype=torch.float64, device=DEV))
    del BandError
